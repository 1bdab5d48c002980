// storeall.cu -- the store-all ("BL") variant of §2.3.1 on the GPU, kept as
// the paper's memory-intensive comparison point.
//
// Exactly as the paper describes BL: (a) primitives and every product that
// is differentiated go to full-grid temporary arrays; (b) one derivative
// kernel per (field, direction, order) writes each of the 60 distinct
// derivatives of Eqs. 1-3 to its own global array (Listing 1's derx, one
// launch each); (c) a residual kernel reads the arrays and assembles Eqs. 1-3;
// (d) the Runge-Kutta update of Fig. 1 runs as its own kernel.
//
// Variables are deviations from the reference state, as in the fused path.
#include "sbli_internal.cuh"

namespace sbli {

namespace {

// scratch array indices (each P elements)
enum {
  A_U = 0,             // u_i                         3
  A_P = 3,             // p'                          1
  A_T = 4,             // T'                          1
  A_MU = 5,            // m_i u_j, symmetric pairs    6 (00,01,02,11,12,22)
  A_EU = 11,           // E' u_j                      3
  A_PU = 14,           // p' u_j                      3
  A_DRHOU = 17,        // D_j m_i        [i][j]       9
  A_DU = 26,           // D_j u_i        [i][j]       9
  A_DRHOUU = 35,       // D_j (m_i u_j)  [i][j]       9
  A_D2U = 44,          // D2_j u_i       [i][j]       9
  A_DDU = 53,          // D_i D_j u_j, i != j         6 (01,02,10,12,20,21)
  A_DRHO = 59,         // D_j rho'                    3
  A_DP = 62,           // D_j p'                      3
  A_DE = 65,           // D_j E'                      3
  A_DEU = 68,          // D_j (E' u_j)                3
  A_DPU = 71,          // D_j (p' u_j)                3
  A_D2T = 74,          // D2_j T'                     3
  A_R = 77,            // residual                    5
  A_COUNT = 82
};

__host__ __device__ inline int sym(int i, int j) {
  const int a = i < j ? i : j, b = i < j ? j : i;
  return a == 0 ? b : (a == 1 ? 2 + b : 5);  // (0,0)0 (0,1)1 (0,2)2 (1,1)3 (1,2)4 (2,2)5
}
__host__ __device__ inline int offd(int i, int j) { return 2 * i + (j > i ? j - 1 : j); }  // i != j -> 0..5

template <typename T, typename TIN>
__global__ void bl_primitives(Geom g, Coef<T> c, const TIN* __restrict__ q, T* __restrict__ s) {
  const long long P = g.P;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < P; n += (long long)gridDim.x * blockDim.x) {
    const T rho_p = T(q[n]);
    const T m[3] = {T(q[P + n]), T(q[2 * P + n]), T(q[3 * P + n])};
    const T E_p = T(q[4 * P + n]);
    const T rho = T(1) + rho_p;
    T u[3];
    for (int i = 0; i < 3; ++i) u[i] = m[i] / rho;
    const T p_p = c.gm1 * (E_p - T(0.5) * rho * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]));  // Eq. 4
    const T T_p = (c.gM2 * p_p - rho_p) / rho;                                              // Eq. 5
    for (int i = 0; i < 3; ++i) s[(A_U + i) * P + n] = u[i];
    s[A_P * P + n] = p_p;
    s[A_T * P + n] = T_p;
    for (int i = 0; i < 3; ++i)
      for (int j = i; j < 3; ++j) s[(A_MU + sym(i, j)) * P + n] = m[i] * u[j];
    for (int j = 0; j < 3; ++j) {
      s[(A_EU + j) * P + n] = E_p * u[j];
      s[(A_PU + j) * P + n] = p_p * u[j];
    }
  }
}

// One derivative of one array along one axis (Listing 1): order 1 is Eq. 6,
// order 2 is Eq. 7.
template <typename T, typename TS, int AXIS, int ORDER>
__global__ void __launch_bounds__(256) bl_derivative(Geom g, const TS* __restrict__ f, T* __restrict__ df, T k0, T k1,
                                                     T k2) {
  const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y, k = blockIdx.z;
  if (i >= g.n0 || j >= g.n1) return;
  const long long n0 = g.n0, pl = (long long)g.n0 * g.n1;
  auto at = [&](int s) -> T {
    if (AXIS == 0) return T(f[wrapi(i + s, g.n0) + n0 * j + pl * k]);
    if (AXIS == 1) return T(f[i + n0 * wrapi(j + s, g.n1) + pl * k]);
    return T(f[i + n0 * j + pl * wrapi(k + s, g.n2)]);
  };
  T v;
  if (ORDER == 1)
    v = k1 * (at(1) - at(-1)) - k2 * (at(2) - at(-2));
  else
    v = k0 * at(0) + k1 * (at(1) + at(-1)) + k2 * (at(2) + at(-2));
  df[i + n0 * j + pl * k] = v;
}

template <typename T>
__global__ void bl_residual(Geom g, Coef<T> c, const T* __restrict__ qrho, const T* __restrict__ qm,
                            const T* __restrict__ qE, long long qstride, T* __restrict__ s) {
  const long long P = g.P;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < P; n += (long long)gridDim.x * blockDim.x) {
    auto A = [&](int a) { return s[(long long)a * P + n]; };
    const T rho = T(1) + qrho[n];
    T m[3], u[3];
    for (int i = 0; i < 3; ++i) {
      m[i] = qm[i * qstride + n];
      u[i] = A(A_U + i);
    }
    const T E = qE[n];
    T du[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) du[i][j] = A(A_DU + 3 * i + j);
    auto dd = [&](int i, int j) { return i == j ? A(A_D2U + 3 * i + i) : A(A_DDU + offd(i, j)); };
    const T div = du[0][0] + du[1][1] + du[2][2];
    // Eq. 1
    T conv = T(0);
    for (int j = 0; j < 3; ++j) conv += A(A_DRHOU + 3 * j + j) + rho * du[j][j] + u[j] * A(A_DRHO + j);
    s[(A_R + 0) * P + n] = T(-0.5) * conv;
    // Eq. 2
    T sd[3];
    for (int i = 0; i < 3; ++i) {
      conv = T(0);
      for (int j = 0; j < 3; ++j) conv += A(A_DRHOUU + 3 * i + j) + m[i] * du[j][j] + u[j] * A(A_DRHOU + 3 * i + j);
      T lap = T(0), cross = T(0);
      for (int j = 0; j < 3; ++j) {
        lap += A(A_D2U + 3 * i + j);
        cross += dd(i, j);
      }
      sd[i] = lap + cross - T(2.0 / 3.0) * cross;
      s[(A_R + 1 + i) * P + n] = T(-0.5) * conv - A(A_DP + i) + c.inv_re * sd[i];
    }
    // Eq. 3 (reference enthalpy carries the constant parts of rho E and p)
    conv = T(0);
    T pw = T(0), heat = T(0), vw = T(0), diss = T(0);
    for (int j = 0; j < 3; ++j) {
      conv += A(A_DEU + j) + E * du[j][j] + u[j] * A(A_DE + j);
      pw += A(A_DPU + j);
      heat += A(A_D2T + j);
    }
    for (int i = 0; i < 3; ++i) {
      vw += u[i] * c.inv_re * sd[i];
      for (int j = 0; j < 3; ++j) diss += du[i][j] * (du[i][j] + du[j][i] - (i == j ? T(2.0 / 3.0) * div : T(0)));
    }
    s[(A_R + 4) * P + n] = T(-0.5) * conv - c.H0 * div - pw + vw + c.inv_re * diss + c.kappa * heat;
  }
}

template <typename T, typename TS>
cudaError_t launch_der(const Geom& g, const Coef<T>& c, const TS* f, T* df, int axis, int order, cudaStream_t s) {
  dim3 blk(32, 8), grd((g.n0 + 31) / 32, (g.n1 + 7) / 8, g.n2);
  const T k0 = c.e0[axis];
  const T k1 = order == 1 ? c.c1[axis] : c.e1[axis];
  const T k2 = order == 1 ? c.c2[axis] : c.e2[axis];
#define SBLI_DER(A, O) bl_derivative<T, TS, A, O><<<grd, blk, 0, s>>>(g, f, df, k0, k1, k2)
  if (order == 1) {
    if (axis == 0) SBLI_DER(0, 1);
    else if (axis == 1) SBLI_DER(1, 1);
    else SBLI_DER(2, 1);
  } else {
    if (axis == 0) SBLI_DER(0, 2);
    else if (axis == 1) SBLI_DER(1, 2);
    else SBLI_DER(2, 2);
  }
#undef SBLI_DER
  return cudaGetLastError();
}

unsigned pgrid(long long n) {
  long long b = (n + 255) / 256;
  return (unsigned)(b < 4096 ? (b < 1 ? 1 : b) : 4096);
}

template <typename T, typename TIN>
cudaError_t storeall_rhs(const Geom& g, const Coef<T>& c, const TIN* q, T* s, cudaStream_t st) {
  const long long P = g.P;
  auto arr = [&](int a) { return s + (long long)a * P; };
  cudaError_t e;
#define SBLI_CK(x)                      \
  do {                                  \
    e = (x);                            \
    if (e != cudaSuccess) return e;     \
  } while (0)
  bl_primitives<T, TIN><<<pgrid(P), 256, 0, st>>>(g, c, q, s);
  SBLI_CK(cudaGetLastError());
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      SBLI_CK((launch_der<T, TIN>(g, c, q + (1 + i) * P, arr(A_DRHOU + 3 * i + j), j, 1, st)));
      SBLI_CK((launch_der<T, T>(g, c, arr(A_U + i), arr(A_DU + 3 * i + j), j, 1, st)));
      SBLI_CK((launch_der<T, T>(g, c, arr(A_MU + sym(i, j)), arr(A_DRHOUU + 3 * i + j), j, 1, st)));
      SBLI_CK((launch_der<T, T>(g, c, arr(A_U + i), arr(A_D2U + 3 * i + j), j, 2, st)));
    }
  for (int j = 0; j < 3; ++j) {
    SBLI_CK((launch_der<T, TIN>(g, c, q, arr(A_DRHO + j), j, 1, st)));
    SBLI_CK((launch_der<T, T>(g, c, arr(A_P), arr(A_DP + j), j, 1, st)));
    SBLI_CK((launch_der<T, TIN>(g, c, q + 4 * P, arr(A_DE + j), j, 1, st)));
    SBLI_CK((launch_der<T, T>(g, c, arr(A_EU + j), arr(A_DEU + j), j, 1, st)));
    SBLI_CK((launch_der<T, T>(g, c, arr(A_PU + j), arr(A_DPU + j), j, 1, st)));
    SBLI_CK((launch_der<T, T>(g, c, arr(A_T), arr(A_D2T + j), j, 2, st)));
  }
  // mixed derivatives D_i (D_j u_j), i != j, from the stored diagonal gradients
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      if (i != j) SBLI_CK((launch_der<T, T>(g, c, arr(A_DU + 3 * j + j), arr(A_DDU + offd(i, j)), i, 1, st)));
  // conserved variables in the arithmetic type (callers pass T == TIN)
  static_assert(sizeof(TIN) == sizeof(T), "storeall_rhs reads conserved fields in the arithmetic type");
  const T* qrho = reinterpret_cast<const T*>(q);
  const T* qm = qrho + P;
  const T* qE = qrho + 4 * P;
  const long long qstride = P;
  bl_residual<T><<<pgrid(P), 256, 0, st>>>(g, c, qrho, qm, qE, qstride, s);
  SBLI_CK(cudaGetLastError());
#undef SBLI_CK
  return cudaSuccess;
}

template <typename TIN>
__global__ void to_float_kernel(long long n, const TIN* __restrict__ a, float* __restrict__ b) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = float(a[i]);
}

template <typename TR, typename TOUT>
__global__ void rk_update_kernel(long long n, const TR* __restrict__ r, const double* __restrict__ acc_in,
                                 double* __restrict__ acc_out, TOUT* __restrict__ q_out, double a_dt, double b_dt) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double rr = double(r[i]);
    const double a = acc_in[i];
    acc_out[i] = fma(b_dt, rr, a);
    if (q_out) q_out[i] = TOUT(fma(a_dt, rr, a));
  }
}

}  // namespace

cudaError_t launch_derivative_fp64(const Geom& g, const Coef<double>& c, const double* f, double* df, int axis,
                                   int order, cudaStream_t s) {
  return launch_der<double, double>(g, c, f, df, axis, order, s);
}

size_t storeall_scratch_doubles(const Geom& g, int elem_bytes) {
  // A_COUNT arrays of the arithmetic type, plus (binary32 only) a binary32
  // copy of the 5 conserved fields for a binary64 stage-0 input.
  const size_t elems = (size_t)A_COUNT * g.P + (elem_bytes == 4 ? 5 * (size_t)g.P : 0);
  return (elems * elem_bytes + 7) / 8;
}

long long storeall_r_offset(const Geom& g) { return (long long)A_R * g.P; }

cudaError_t launch_storeall_rhs_fp64(const Geom& g, const Coef<double>& c, const double* q_off, double* scratch,
                                     double* r_out, cudaStream_t s) {
  cudaError_t e = storeall_rhs<double, double>(g, c, q_off, scratch, s);
  if (e != cudaSuccess) return e;
  if (r_out) return cudaMemcpyAsync(r_out, scratch + (long long)A_R * g.P, 5 * g.P * sizeof(double),
                                    cudaMemcpyDeviceToDevice, s);
  return cudaSuccess;
}

cudaError_t launch_storeall_rhs_fp32(const Geom& g, const Coef<float>& c, const void* q_off, bool in_fp64,
                                     float* scratch, float* r_out, cudaStream_t s) {
  const float* q = static_cast<const float*>(q_off);
  if (in_fp64) {
    float* conv = scratch + (long long)A_COUNT * g.P;
    to_float_kernel<double><<<pgrid(5 * g.P), 256, 0, s>>>(5 * g.P, static_cast<const double*>(q_off), conv);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    q = conv;
  }
  cudaError_t e = storeall_rhs<float, float>(g, c, q, scratch, s);
  if (e != cudaSuccess) return e;
  if (r_out) return cudaMemcpyAsync(r_out, scratch + (long long)A_R * g.P, 5 * g.P * sizeof(float),
                                    cudaMemcpyDeviceToDevice, s);
  return cudaSuccess;
}

// R -> stage update of Fig. 1: acc_out = acc_in + b dt R; q_out = acc_in + a dt R.
cudaError_t launch_rk_update(const Geom& g, const void* r, bool r_fp64, const double* acc_in, double* acc_out,
                             void* q_out, bool out_fp64, double a_dt, double b_dt, cudaStream_t s) {
  const long long n = 5 * g.P;
  if (r_fp64) {
    if (out_fp64)
      rk_update_kernel<double, double><<<pgrid(n), 256, 0, s>>>(n, static_cast<const double*>(r), acc_in, acc_out,
                                                                static_cast<double*>(q_out), a_dt, b_dt);
    else
      rk_update_kernel<double, float><<<pgrid(n), 256, 0, s>>>(n, static_cast<const double*>(r), acc_in, acc_out,
                                                               static_cast<float*>(q_out), a_dt, b_dt);
  } else {
    if (out_fp64)
      rk_update_kernel<float, double><<<pgrid(n), 256, 0, s>>>(n, static_cast<const float*>(r), acc_in, acc_out,
                                                               static_cast<double*>(q_out), a_dt, b_dt);
    else
      rk_update_kernel<float, float><<<pgrid(n), 256, 0, s>>>(n, static_cast<const float*>(r), acc_in, acc_out,
                                                              static_cast<float*>(q_out), a_dt, b_dt);
  }
  return cudaGetLastError();
}

}  // namespace sbli
