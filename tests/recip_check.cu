// Compiled by tests/test_gpu_recip.py: the stage kernels' binary64 reciprocal
// (sbli::recip<double>, a Newton-refined hardware approximation) against
// CUDA's correctly rounded reciprocal, as the largest difference in units in
// the last place over seeded inputs.
#include <cstdint>
#include <cstdio>

#include "fused_stage.cuh"

__global__ void compare(const double* x, long long n, unsigned long long* worst, unsigned long long* differ) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double a = sbli::recip<double>(x[i]), b = __drcp_rn(x[i]);
  long long d = (long long)__double_as_longlong(a) - (long long)__double_as_longlong(b);
  if (d < 0) d = -d;
  atomicMax(worst, (unsigned long long)d);
  if (d) atomicAdd(differ, 1ull);
}

int main() {
  const long long n = 1 << 22;
  double* h = new double[n];
  uint64_t s = 88172645463325252ull;  // xorshift64
  for (long long i = 0; i < n; ++i) {
    s ^= s << 13;
    s ^= s >> 7;
    s ^= s << 17;
    const double u = (double)(s >> 11) / 9007199254740992.0;
    // 1 + rho' of the stage kernels (density deviations), and a wide range
    h[i] = (i % 3 == 0) ? 0.5 + u : (i % 3 == 1) ? 1.0 + 1e-3 * (u - 0.5) : ldexp(1.0 + u, (int)(s % 400) - 200);
  }
  double* d = nullptr;
  unsigned long long* r = nullptr;
  if (cudaMalloc(&d, n * sizeof(double)) != cudaSuccess || cudaMalloc(&r, 2 * sizeof(unsigned long long)) != cudaSuccess)
    return 2;
  cudaMemcpy(d, h, n * sizeof(double), cudaMemcpyHostToDevice);
  cudaMemset(r, 0, 2 * sizeof(unsigned long long));
  compare<<<(unsigned)((n + 255) / 256), 256>>>(d, n, r, r + 1);
  if (cudaDeviceSynchronize() != cudaSuccess) return 3;
  unsigned long long out[2];
  cudaMemcpy(out, r, sizeof out, cudaMemcpyDeviceToHost);
  printf("%llu %llu %lld\n", out[0], out[1], n);
  return 0;
}
