// noalloc.cu -- kinetic energy and enstrophy of a caller's state without any
// device allocation by anyone.
//
// Who needs this: callers that hold a Navier-Stokes state in device memory
// but cannot allocate more, so they can neither call cudaMalloc nor hand the
// library a workspace.  Typical cases are a host application whose memory
// manager reserves the whole device at start-up and refuses later requests,
// plug-in code that a framework calls with nothing but a pointer to the state,
// and latency-critical loops in which an allocation (which can synchronise
// the device) is not allowed once the loop is running.
//
// The partial sums that sbli_kinetic_energy keeps in the grid's workspace
// live here in a file-scope __device__ array instead.  Every GPU that loads
// the library holds this array (NOALLOC_MAX_PARTIALS pairs of doubles,
// 128 KiB) until the process exits.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include <algorithm>
#include <mutex>

#include "sbli_internal.cuh"

namespace sbli {
namespace {

// Capacity of the static scratch in (ke, enstrophy) pairs (one per block),
// and the most points one block may cover; together they bound the grid to
// NOALLOC_MAX_PARTIALS * NOALLOC_POINTS_PER_BLOCK = 512^3 points.  A call
// launches one block per NOALLOC_BLOCK points, at most NOALLOC_MAX_PARTIALS.
constexpr int NOALLOC_MAX_PARTIALS = 8192;
constexpr int NOALLOC_BLOCK = 256;
constexpr long long NOALLOC_POINTS_PER_BLOCK = 64LL * NOALLOC_BLOCK;

static __device__ __align__(256) double g_noalloc_partials[2 * NOALLOC_MAX_PARTIALS];

// Device address of g_noalloc_partials per device (host code cannot use the
// symbol itself: on the host it names a stand-in, not device memory).  The
// address is looked up again on every call made while the stream is not
// being captured (so a device reset between calls is picked up); a call
// during stream capture uses the address an earlier call stored.
constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mutex;
double* g_scratch_ptr[MAX_DEVICES] = {};

cudaError_t scratch_for_current_device(cudaStream_t s, double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
    cudaGetLastError();
    cap = cudaStreamCaptureStatusActive;  // unknown: do not call into the runtime's module lookup
  }
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (cap == cudaStreamCaptureStatusNone) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<double*>(p);
  } else if (!g_scratch_ptr[dev]) {
    return cudaErrorStreamCaptureUnsupported;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

// True when p is device (or managed) memory the current device can read.
bool device_readable(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

// Same quantities as the workspace-based reduction, read from plain
// conserved variables (rho, rho u_i, rho E): per point rho |u|^2 / 2 and
// rho |curl u|^2 / 2 with Eq. 6 derivatives of u; fixed-order sums.
__global__ void __launch_bounds__(NOALLOC_BLOCK) ke_plain_kernel(Geom g, Coef<double> c, const double* __restrict__ q,
                                                                  double* __restrict__ partials) {
  const long long P = g.P;
  const int n0 = g.n0, n1 = g.n1, n2 = g.n2;
  double ke = 0.0, en = 0.0;
  for (long long n = blockIdx.x * (long long)NOALLOC_BLOCK + threadIdx.x; n < P;
       n += (long long)gridDim.x * NOALLOC_BLOCK) {
    const int i = (int)(n % n0);
    const int j = (int)((n / n0) % n1);
    const int k = (int)(n / ((long long)n0 * n1));
    auto vel = [&](long long m, int comp) { return q[(1 + comp) * P + m] / q[m]; };
    auto idx = [&](int ii, int jj, int kk) {
      return (long long)wrapi(ii, n0) + (long long)n0 * (wrapi(jj, n1) + (long long)n1 * wrapi(kk, n2));
    };
    auto d1 = [&](int comp, int axis) {
      const int o[4] = {-2, -1, 1, 2};
      double f[4];
      for (int m = 0; m < 4; ++m) {
        const long long nn = axis == 0 ? idx(i + o[m], j, k) : axis == 1 ? idx(i, j + o[m], k) : idx(i, j, k + o[m]);
        f[m] = vel(nn, comp);
      }
      return c.c1[axis] * (f[2] - f[1]) - c.c2[axis] * (f[3] - f[0]);
    };
    const double rho = q[n];
    const double u0 = vel(n, 0), u1 = vel(n, 1), u2 = vel(n, 2);
    const double w0 = d1(2, 1) - d1(1, 2);
    const double w1 = d1(0, 2) - d1(2, 0);
    const double w2 = d1(1, 0) - d1(0, 1);
    ke += 0.5 * rho * (u0 * u0 + u1 * u1 + u2 * u2);
    en += 0.5 * rho * (w0 * w0 + w1 * w1 + w2 * w2);
  }
  __shared__ double red[2][NOALLOC_BLOCK / 32];
  for (int o = 16; o > 0; o >>= 1) {
    ke += __shfl_down_sync(0xffffffffu, ke, o);
    en += __shfl_down_sync(0xffffffffu, en, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = ke;
    red[1][threadIdx.x >> 5] = en;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < NOALLOC_BLOCK / 32; ++w) {
      a += red[0][w];
      b += red[1][w];
    }
    partials[2 * blockIdx.x] = a;
    partials[2 * blockIdx.x + 1] = b;
  }
}

int noalloc_fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  return set_last_error(code, buf);
}

}  // namespace

}  // namespace sbli

extern "C" SBLI_API int sbli_kinetic_energy_noalloc(const double* q_dev, int n0, int n1, int n2, double L,
                                                    double* out_dev, void* stream) {
  using namespace sbli;
  if (!q_dev || !out_dev) return noalloc_fail(SBLI_EINVAL, "q_dev and out_dev must be device pointers");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return noalloc_fail(SBLI_ECUDA, "no current CUDA device");
  }
  if (!device_readable(q_dev, dev) || !device_readable(out_dev, dev))
    return noalloc_fail(SBLI_EINVAL, "q_dev and out_dev must be device (or managed) memory of the current device %d",
                        dev);
  if (n0 < 5 || n1 < 5 || n2 < 5 || n0 > (1 << 24) || n1 > (1 << 24) || n2 > (1 << 24) ||
      (long long)n0 * n1 >= (1LL << 31))
    return noalloc_fail(SBLI_EINVAL, "grid %d x %d x %d: each edge must be in [5, 2^24] and n0*n1 < 2^31", n0, n1, n2);
  if (!(L > 0) || !isfinite(L)) return noalloc_fail(SBLI_EINVAL, "L must be finite and > 0");
  const long long P = (long long)n0 * n1 * n2;
  if ((P + NOALLOC_POINTS_PER_BLOCK - 1) / NOALLOC_POINTS_PER_BLOCK > NOALLOC_MAX_PARTIALS)
    return noalloc_fail(SBLI_EINVAL,
                        "grid of %lld points exceeds the allocation-free maximum of %lld points "
                        "(static scratch of %d partial sums)",
                        P, (long long)NOALLOC_MAX_PARTIALS * NOALLOC_POINTS_PER_BLOCK, NOALLOC_MAX_PARTIALS);
  // one block per NOALLOC_BLOCK points up to the scratch capacity; the
  // kernel's grid-stride loop covers the rest
  const long long blocks = std::min<long long>((P + NOALLOC_BLOCK - 1) / NOALLOC_BLOCK, NOALLOC_MAX_PARTIALS);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* scratch = nullptr;
  cudaError_t e = scratch_for_current_device(s, &scratch);
  if (e == cudaErrorStreamCaptureUnsupported)
    return noalloc_fail(SBLI_EINVAL, "first call on device %d made during stream capture: call once before capturing",
                        dev);
  if (e != cudaSuccess) return noalloc_fail(SBLI_ECUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
  sbli_params prm{1.0, 1.0, 1.0, 1.4, L};
  const int n[3] = {n0, n1, n2};
  const Geom g{n0, n1, n2, P};
  ke_plain_kernel<<<(unsigned)blocks, NOALLOC_BLOCK, 0, s>>>(g, make_coef<double>(n, prm), q_dev, scratch);
  e = cudaGetLastError();
  if (e != cudaSuccess) return noalloc_fail(SBLI_ECUDA, "kernel launch: %s", cudaGetErrorString(e));
  e = launch_finalize_ke(scratch, (int)blocks, 1.0 / (double)P, out_dev, s);
  if (e != cudaSuccess) return noalloc_fail(SBLI_ECUDA, "finalize launch: %s", cudaGetErrorString(e));
  return SBLI_OK;
}
