// probe.cu -- fused multiply-add throughput of the current GPU (the ALU
// roofline denominator of the stage kernels; see include/sbli_probe.h).
//
// Every thread runs CHAINS independent chains x <- x * a + b, so the FMA pipe
// always has independent work; the grid fills every SM to full occupancy.
// a and b come from the host and the final sum is stored only if it equals
// a value it can never reach, which the compiler cannot prove: the chains
// stay live and nothing is written.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include "../../include/sbli_probe.h"
#include "sbli_internal.cuh"

namespace sbli {
namespace {

constexpr int PROBE_CHAINS = 8;
constexpr int PROBE_BLOCK = 256;
constexpr int PROBE_ROUNDS = 2;  // chain steps per loop trip

template <typename T>
__global__ void __launch_bounds__(PROBE_BLOCK) fma_chain_kernel(long long iters, T a, T b, T* sink) {
  T x[PROBE_CHAINS];
#pragma unroll
  for (int i = 0; i < PROBE_CHAINS; ++i) x[i] = T(threadIdx.x & 7) + T(i);
  for (long long it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < PROBE_ROUNDS; ++u) {
#pragma unroll
      for (int i = 0; i < PROBE_CHAINS; ++i) x[i] = fma(x[i], a, b);
    }
  }
  T s = T(0);
#pragma unroll
  for (int i = 0; i < PROBE_CHAINS; ++i) s += x[i];
  if (s == T(-12345.0)) *sink = s;  // unreachable for the host's a, b (the chains stay positive)
}

int probe_fail(int code, const char* fmt, ...) {
  char buf[256];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  return set_last_error(code, buf);
}

template <typename T>
int probe_run(long long iters, T* sink, cudaStream_t s, double* rate, float* ms_out) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return probe_fail(SBLI_ECUDA, "no current CUDA device");
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_chain_kernel<T>, PROBE_BLOCK, 0) != cudaSuccess ||
      per_sm < 1)
    return probe_fail(SBLI_ECUDA, "occupancy query failed");
  const unsigned blocks = (unsigned)(sms * per_sm);
  // a < 1 and b > 0: every chain converges to b / (1 - a) and stays positive
  const T a = T(0.999), b = T(0.001);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return probe_fail(SBLI_ECUDA, "cudaEventCreate");
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return probe_fail(SBLI_ECUDA, "cudaEventCreate");
  }
  fma_chain_kernel<T><<<blocks, PROBE_BLOCK, 0, s>>>(1, a, b, sink);  // warm-up (module load, clocks)
  cudaError_t e = cudaEventRecord(e0, s);
  if (e == cudaSuccess) {
    fma_chain_kernel<T><<<blocks, PROBE_BLOCK, 0, s>>>(iters, a, b, sink);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return probe_fail(SBLI_ECUDA, "probe launch: %s", cudaGetErrorString(e));
  const double fmas = (double)blocks * PROBE_BLOCK * PROBE_CHAINS * PROBE_ROUNDS * (double)iters;
  *rate = 2.0 * fmas / (ms * 1e-3);
  if (ms_out) *ms_out = ms;
  return SBLI_OK;
}

}  // namespace
}  // namespace sbli

extern "C" SBLI_API int sbli_probe_fma_rate(int precision, long long iters, double* sink_dev, void* stream,
                                            double* flop_per_s, float* ms) {
  using namespace sbli;
  if (!sink_dev || !flop_per_s) return probe_fail(SBLI_EINVAL, "sink_dev and flop_per_s must not be null");
  if (iters < 1) return probe_fail(SBLI_EINVAL, "iters must be >= 1");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (precision == SBLI_FP64) return probe_run<double>(iters, sink_dev, s, flop_per_s, ms);
  if (precision == SBLI_FP32) return probe_run<float>(iters, reinterpret_cast<float*>(sink_dev), s, flop_per_s, ms);
  return probe_fail(SBLI_EINVAL, "precision %d: SBLI_FP64 or SBLI_FP32 only", precision);
}
