// diag.cu -- Taylor-Green initial field, reference-state conversion and the
// binary64 kinetic-energy / enstrophy reduction.
#include <math.h>

#include "fpconv.cuh"
#include "sbli_internal.cuh"

namespace sbli {

template <typename T>
Coef<T> make_coef(const int n[3], const sbli_params& p) {
  Coef<T> c;
  for (int a = 0; a < 3; ++a) {
    const double h = 2.0 * M_PI * p.L / (double)n[a];
    c.c1[a] = T(2.0 / (3.0 * h));
    c.c2[a] = T(1.0 / (12.0 * h));
    c.e0[a] = T(-5.0 / (2.0 * h * h));
    c.e1[a] = T(4.0 / (3.0 * h * h));
    c.e2[a] = T(-1.0 / (12.0 * h * h));
  }
  const double inv_re = isinf(p.Re) ? 0.0 : 1.0 / p.Re;
  c.gm1 = T(p.gamma - 1.0);
  c.gM2 = T(p.gamma * p.Mach * p.Mach);
  c.gm1x2 = T(2.0 * (p.gamma - 1.0));
  c.hgM2 = T(0.5 * p.gamma * p.Mach * p.Mach);
  c.inv_re = T(inv_re);
  c.kappa = T(inv_re / ((p.gamma - 1.0) * p.Mach * p.Mach * p.Pr));
  c.H0 = T(1.0 / ((p.gamma - 1.0) * p.Mach * p.Mach));
  return c;
}
template Coef<double> make_coef<double>(const int[3], const sbli_params&);
template Coef<float> make_coef<float>(const int[3], const sbli_params&);
template Coef<dfloat> make_coef<dfloat>(const int[3], const sbli_params&);

RefState make_ref(const sbli_params& p) {
  RefState r;
  r.rho0 = 1.0;
  r.E0 = 1.0 / (p.gamma * (p.gamma - 1.0) * p.Mach * p.Mach);  // p_ref/(gamma-1)
  return r;
}

// §4, Eqs. 9-12 with amplitude A; T = 1 so rho = gamma M^2 p (Eq. 5), rho E
// from Eq. 4.  Written as deviations from the reference state:
//   rho - 1 = gamma M^2 (p - p_ref),  rho E - E_ref = (p - p_ref)/(gamma-1) + rho |u|^2/2.
__global__ void init_tgv_kernel(Geom g, double h0, double h1, double h2, double L, double A, double gM2,
                                double inv_gm1, double* __restrict__ q) {
  const long long P = g.P;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < P; n += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(n % g.n0);
    const int j = (int)((n / g.n0) % g.n1);
    const int k = (int)(n / ((long long)g.n0 * g.n1));
    const double x = i * h0, y = j * h1, z = k * h2;
    double sx, cx, sy, cy, sz, cz;
    sincos(x / L, &sx, &cx);
    sincos(y / L, &sy, &cy);
    sincos(z / L, &sz, &cz);
    (void)sz;
    const double u0 = A * sx * cy * cz;
    const double u1 = -A * cx * sy * cz;
    const double dp = A * A / 16.0 * (cos(2.0 * x / L) + cos(2.0 * y / L)) * (2.0 + cos(2.0 * z / L));
    const double rho_p = gM2 * dp;
    const double rho = 1.0 + rho_p;
    q[n] = rho_p;
    q[P + n] = rho * u0;
    q[2 * P + n] = rho * u1;
    q[3 * P + n] = 0.0;
    q[4 * P + n] = dp * inv_gm1 + 0.5 * rho * (u0 * u0 + u1 * u1);
  }
}

static unsigned grid_for(long long n, int block) {
  long long b = (n + block - 1) / block;
  return (unsigned)(b < 8192 ? (b < 1 ? 1 : b) : 8192);
}

cudaError_t launch_init_tgv(const Geom& g, const sbli_params& p, double amplitude, double* q, cudaStream_t s) {
  const double h0 = 2.0 * M_PI * p.L / g.n0, h1 = 2.0 * M_PI * p.L / g.n1, h2 = 2.0 * M_PI * p.L / g.n2;
  init_tgv_kernel<<<grid_for(g.P, 256), 256, 0, s>>>(g, h0, h1, h2, p.L, amplitude, p.gamma * p.Mach * p.Mach,
                                                     1.0 / (p.gamma - 1.0), q);
  return cudaGetLastError();
}

// sign = -1: plain -> deviation; +1: deviation -> plain.  Fields 0 and 4 only
// differ; momenta are copied.
__global__ void offset_kernel(long long P, double rho0, double E0, double sign, const double* __restrict__ src,
                              double* __restrict__ dst) {
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < 5 * P;
       n += (long long)gridDim.x * blockDim.x) {
    const long long f = n / P;
    double v = src[n];
    if (f == 0) v += sign * rho0;
    if (f == 4) v += sign * E0;
    dst[n] = v;
  }
}

cudaError_t launch_to_offset(const Geom& g, const RefState& r, const double* q_plain, double* q_off, cudaStream_t s) {
  offset_kernel<<<grid_for(5 * g.P, 256), 256, 0, s>>>(g.P, r.rho0, r.E0, -1.0, q_plain, q_off);
  return cudaGetLastError();
}

cudaError_t launch_from_offset(const Geom& g, const RefState& r, const double* q_off, double* q_plain,
                               cudaStream_t s) {
  offset_kernel<<<grid_for(5 * g.P, 256), 256, 0, s>>>(g.P, r.rho0, r.E0, 1.0, q_off, q_plain);
  return cudaGetLastError();
}

__global__ void widen_kernel(long long n, const float* __restrict__ src, double* __restrict__ dst) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = double(src[i]);
}

cudaError_t launch_widen(long long n, const float* src, double* dst, cudaStream_t s) {
  widen_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, src, dst);
  return cudaGetLastError();
}

// The binary32 copy of a binary64 state that stage 0 of the binary32 path
// reads: the same narrowing the stage kernels apply (narrow_f64_rna).
__global__ void narrow_kernel(long long n, const double* __restrict__ src, float* __restrict__ dst) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = narrow_f64_rna(src[i]);
}

cudaError_t launch_narrow(long long n, const double* src, float* dst, cudaStream_t s) {
  narrow_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, src, dst);
  return cudaGetLastError();
}

__global__ void df_split_kernel(long long n5, long long P, double rho0, double E0, const double* __restrict__ src,
                                float* __restrict__ dst) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n5; i += (long long)gridDim.x * blockDim.x) {
    const long long f = i / P;
    const double v = src[i] - (f == 0 ? rho0 : (f == 4 ? E0 : 0.0));
    const float hi = __double2float_rn(v);
    dst[i] = hi;
    dst[i + 5 * P] = __double2float_rn(v - (double)hi);
  }
}

__global__ void df_join_kernel(long long n5, long long P, double rho0, double E0, const float* __restrict__ src,
                               double* __restrict__ dst) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n5; i += (long long)gridDim.x * blockDim.x) {
    const long long f = i / P;
    dst[i] = ((double)src[i] + (double)src[i + 5 * P]) + (f == 0 ? rho0 : (f == 4 ? E0 : 0.0));
  }
}

cudaError_t launch_df_split(long long P, const RefState& r, const double* src, float* dst, cudaStream_t s) {
  df_split_kernel<<<grid_for(5 * P, 256), 256, 0, s>>>(5 * P, P, r.rho0, r.E0, src, dst);
  return cudaGetLastError();
}

cudaError_t launch_df_join(long long P, const RefState& r, const float* src, double* dst, cudaStream_t s) {
  df_join_kernel<<<grid_for(5 * P, 256), 256, 0, s>>>(5 * P, P, r.rho0, r.E0, src, dst);
  return cudaGetLastError();
}

// A binary64 field as interleaved double-float pairs, split as the stage
// kernels split a binary64 input (split_f64).
__global__ void pair_split_kernel(long long n, const double* __restrict__ src, float2* __restrict__ dst) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    float hi, lo;
    split_f64(src[i], hi, lo);
    dst[i] = make_float2(hi, lo);
  }
}

cudaError_t launch_pair_split(long long n, const double* src, float* dst, cudaStream_t s) {
  pair_split_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, src, reinterpret_cast<float2*>(dst));
  return cudaGetLastError();
}

// A stage field of interleaved double-float pairs as binary64 (the sum of two
// binary32 values is exact in binary64).
__global__ void pair_join_kernel(long long n, const float2* __restrict__ src, double* __restrict__ dst) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float2 v = src[i];
    dst[i] = (double)v.x + (double)v.y;
  }
}

cudaError_t launch_pair_join(long long n, const float* src, double* dst, cudaStream_t s) {
  pair_join_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, reinterpret_cast<const float2*>(src), dst);
  return cudaGetLastError();
}

// Plain conserved variables at listed points: out[f * count + i] for the
// point of linear index idx[i] (x0 fastest).  The binary64 state (q64) or the
// double-float state (qdf: hi fields, then lo fields) is in deviation form;
// the sums are those of the full-grid conversions, so a sample equals the
// corresponding entry of a full read-out bit for bit.  Indices outside
// [0, P) yield NaN in all five fields.
__global__ void sample_state_kernel(long long P, double rho0, double E0, const double* __restrict__ q64,
                                    const float* __restrict__ qdf, const long long* __restrict__ idx, int count,
                                    double* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    const long long n = idx[i];
    const bool inside = n >= 0 && n < P;
#pragma unroll
    for (int f = 0; f < 5; ++f) {
      double v = __longlong_as_double(0x7ff8000000000000LL);  // quiet NaN
      if (inside) {
        const long long m = (long long)f * P + n;
        if (q64) {  // as offset_kernel
          v = q64[m];
          if (f == 0) v += rho0;
          if (f == 4) v += E0;
        } else {  // as df_join_kernel
          v = ((double)qdf[m] + (double)qdf[m + 5 * P]) + (f == 0 ? rho0 : (f == 4 ? E0 : 0.0));
        }
      }
      out[(long long)f * count + i] = v;
    }
  }
}

cudaError_t launch_sample_state(long long P, const RefState& r, const double* q64, const float* qdf,
                                const long long* idx, int count, double* out, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  sample_state_kernel<<<grid_for(count, 256), 256, 0, s>>>(P, r.rho0, r.E0, q64, qdf, idx, count, out);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ KE
constexpr int KE_BLOCK = 256;
constexpr int KE_MAX_BLOCKS = 1024;

int ke_num_partials(const Geom& g) {
  long long b = (g.P + KE_BLOCK - 1) / KE_BLOCK;
  return (int)(b < KE_MAX_BLOCKS ? (b < 1 ? 1 : b) : KE_MAX_BLOCKS);
}

__device__ __forceinline__ double vel(const double* __restrict__ q, long long P, long long n, int i) {
  return q[(1 + i) * P + n] / (1.0 + q[n]);
}

// Per point: ke = rho |u|^2 / 2, enstrophy = rho |curl u|^2 / 2 with Eq. 6
// derivatives of u (u recomputed at the stencil points).  Each thread sums
// its points in a fixed order; blocks reduce in a fixed order.
__global__ void __launch_bounds__(KE_BLOCK) ke_kernel(Geom g, Coef<double> c, const double* __restrict__ q,
                                                      double* __restrict__ partials) {
  const long long P = g.P;
  const int n0 = g.n0, n1 = g.n1, n2 = g.n2;
  double ke = 0.0, en = 0.0;
  for (long long n = blockIdx.x * (long long)KE_BLOCK + threadIdx.x; n < P; n += (long long)gridDim.x * KE_BLOCK) {
    const int i = (int)(n % n0);
    const int j = (int)((n / n0) % n1);
    const int k = (int)(n / ((long long)n0 * n1));
    auto idx = [&](int ii, int jj, int kk) {
      return (long long)wrapi(ii, n0) + (long long)n0 * (wrapi(jj, n1) + (long long)n1 * wrapi(kk, n2));
    };
    auto d1 = [&](int comp, int axis) {
      const int o[4] = {-2, -1, 1, 2};
      double f[4];
      for (int m = 0; m < 4; ++m) {
        const long long nn = axis == 0 ? idx(i + o[m], j, k) : axis == 1 ? idx(i, j + o[m], k) : idx(i, j, k + o[m]);
        f[m] = vel(q, P, nn, comp);
      }
      return c.c1[axis] * (f[2] - f[1]) - c.c2[axis] * (f[3] - f[0]);
    };
    const double rho = 1.0 + q[n];
    const double u0 = vel(q, P, n, 0), u1 = vel(q, P, n, 1), u2 = vel(q, P, n, 2);
    const double w0 = d1(2, 1) - d1(1, 2);
    const double w1 = d1(0, 2) - d1(2, 0);
    const double w2 = d1(1, 0) - d1(0, 1);
    ke += 0.5 * rho * (u0 * u0 + u1 * u1 + u2 * u2);
    en += 0.5 * rho * (w0 * w0 + w1 * w1 + w2 * w2);
  }
  __shared__ double red[2][KE_BLOCK / 32];
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
    for (int w = 0; w < KE_BLOCK / 32; ++w) {
      a += red[0][w];
      b += red[1][w];
    }
    partials[2 * blockIdx.x] = a;
    partials[2 * blockIdx.x + 1] = b;
  }
}

// One block: thread t sums pairs t, t+256, ... in order, then a fixed tree.
__global__ void __launch_bounds__(256) finalize_ke_kernel(const double* __restrict__ partials, int n, double inv_p,
                                                          double* __restrict__ out) {
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) {
    a += partials[2 * i];
    b += partials[2 * i + 1];
  }
  __shared__ double red[2][256];
  red[0][threadIdx.x] = a;
  red[1][threadIdx.x] = b;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
      red[0][threadIdx.x] += red[0][threadIdx.x + s];
      red[1][threadIdx.x] += red[1][threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = red[0][0] * inv_p;
    out[1] = red[1][0] * inv_p;
  }
}

cudaError_t launch_finalize_ke(const double* partials, int n, double inv_p, double* out, cudaStream_t s) {
  finalize_ke_kernel<<<1, 256, 0, s>>>(partials, n, inv_p, out);
  return cudaGetLastError();
}

cudaError_t launch_ke(const Geom& g, const Coef<double>& c, const RefState& r, const double* q_off,
                      double* partials, double* out, cudaStream_t s) {
  (void)r;
  const int nb = ke_num_partials(g);
  ke_kernel<<<nb, KE_BLOCK, 0, s>>>(g, c, q_off, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_finalize_ke(partials, nb, 1.0 / (double)g.P, out, s);
}

}  // namespace sbli
