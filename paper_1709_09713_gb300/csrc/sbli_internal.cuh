// sbli_internal.cuh -- shared definitions of the CUDA library (not part of
// the public ABI).  Kernels and launchers for one grid are declared here and
// defined in the per-precision translation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/sbli.h"
#include "dfloat.cuh"

namespace sbli {

// Number of fields of the state Q = (rho, rho u0, rho u1, rho u2, rho E).
constexpr int NF = 5;

// Per-grid constants in the arithmetic type T of the kernel.  All
// divisions by the grid spacing and by physical constants are folded here
// once (as the paper's generated code does, §2.6).
template <typename T>
struct Coef {
  // Eq. 6: D1 f = c1 (f[+1] - f[-1]) - c2 (f[+2] - f[-2]),
  //   c1 = 2/(3h), c2 = 1/(12h)
  T c1[3], c2[3];
  // Eq. 7: D2 f = e0 f[0] + e1 (f[+1] + f[-1]) + e2 (f[+2] + f[-2]),
  //   e0 = -5/(2h^2), e1 = 4/(3h^2), e2 = -1/(12h^2)
  T e0[3], e1[3], e2[3];
  T gm1;    // gamma - 1                    (Eq. 4)
  T gM2;    // gamma M^2                    (Eq. 5)
  T gm1x2;  // 2 (gamma - 1): the fused kernels keep 2 p' (both uses of p in Eqs. 2-3 carry a factor 2)
  T hgM2;   // gamma M^2 / 2: T' from 2 p'  (Eq. 5)
  T inv_re; // 1/Re (0 for Re = inf)        (Eqs. 2-3)
  T kappa;  // 1/((gamma-1) M^2 Pr Re)      (Eq. 3 heat flux)
  T H0;     // (rho E)_ref + p_ref = 1/((gamma-1) M^2): enthalpy of the reference state
};

// Reference state the stored variables are measured from:
//   rho_ref = 1, (rho u)_ref = 0, (rho E)_ref = p_ref/(gamma-1),
//   p_ref = 1/(gamma M^2)  (so T_ref = 1 by Eq. 5).
struct RefState {
  double rho0, E0;
};

template <typename T>
Coef<T> make_coef(const int n[3], const sbli_params& p);

RefState make_ref(const sbli_params& p);

// Runge-Kutta coefficients of the two-register three-stage scheme (§2.2):
// stage a_k and accumulator b_k, third order (a_2 = b_2).
constexpr double RK_A[3] = {2.0 / 3.0, 5.0 / 12.0, 3.0 / 5.0};
constexpr double RK_B[3] = {1.0 / 4.0, 3.0 / 20.0, 3.0 / 5.0};

// Geometry passed to every kernel.
struct Geom {
  int n0, n1, n2;
  long long P;  // n0*n1*n2
};

// Arguments of one fused stage (or RHS-only) launch.
struct StageArgs {
  Geom g;
  int zc;                  // planes per CTA along x2
  const void* q_in;        // stage input (stencil reads)
  const double* acc_in;    // accumulator in (binary64; on stage 0 the state itself)
  double* acc_out;         // accumulator out (binary64), may alias acc_in
  void* q_out;             // stage output, nullptr on the last stage
  double* r_out;           // RHS-only mode: R (binary64)
  double a_dt, b_dt;       // a_k dt, b_k dt
  double amb_dt;           // (a_k - b_k) dt
  float b_dt32, amb_dt32;  // the same rounded to binary32 on the host (binary32 stage updates)
  double* ke_partials;     // per-CTA (ke, enstrophy) partial sums, or nullptr
  // double-float accumulator (precision SBLI_FP32_DF): 5 hi fields then 5 lo
  // fields of binary32, P values each
  const float* dacc_in;
  float* dacc_out;
  int df_normalize;  // double-float accumulator: renormalise (hi, lo) in this stage (the last of a step)
};

// Launch configuration chosen for one grid (the autotuner's output).
struct FusedConfig {
  int ty;  // in-plane tile height (tile is 32 x ty)
  int zc;  // planes per CTA
  int zq;  // binary32 paths: 0 = x2-neighbour records from the shared-memory
           // ring, 1 = from a per-thread queue in tensor memory (TMEM)
  int px;  // binary32 paths: columns per thread (1, or 2 = columns x and x + 32
           // of a 64 x ty tile computed together)
};

// Host launchers (defined in fused_fp64.cu / fused_fp32.cu).
// in_fp64: stage input is binary64 (FP64 path, or FP32 path at stage 0).
// out_fp64: stage output is binary64.
cudaError_t launch_fused_fp64(const StageArgs& a, const Coef<double>& c, const FusedConfig& cfg, bool rhs_only,
                              cudaStream_t s);
cudaError_t launch_fused_fp32(const StageArgs& a, const Coef<float>& c, const FusedConfig& cfg, bool in_fp64,
                              bool rhs_only, cudaStream_t s);
// binary32 stage with a double-float accumulator (stage inputs are binary32)
cudaError_t launch_fused_fp32df(const StageArgs& a, const Coef<float>& c, const FusedConfig& cfg, bool rhs_only,
                                cudaStream_t s);
// binary64 storage, double-float arithmetic (fused_df64.cu): the stage input
// is a field of interleaved (hi, lo) binary32 pairs (in_pairs: every stage of
// a single grid) or the binary64 state (the residual alone); the stage output
// field is written as pairs.
cudaError_t launch_fused_df64(const StageArgs& a, const Coef<dfloat>& c, const FusedConfig& cfg, bool rhs_only,
                              bool in_pairs, cudaStream_t s);
// the two binary32 paths with two columns per thread (fused_fp32_pair.cu)
cudaError_t launch_fused_fp32_pair(const StageArgs& a, const Coef<float>& c, const FusedConfig& cfg, bool in_fp64,
                                   bool df, bool rhs_only, cudaStream_t s);
// the same two binary32 paths with the TMEM z queue (fused_fp32_tmem.cu)
cudaError_t launch_fused_fp32_tmem(const StageArgs& a, const Coef<float>& c, const FusedConfig& cfg, bool in_fp64,
                                   bool df, bool rhs_only, cudaStream_t s);
int fused_num_ctas(const Geom& g, const FusedConfig& cfg);

// Diagnostics and state conversion (diag.cu).
cudaError_t launch_init_tgv(const Geom& g, const sbli_params& p, double amplitude, double* q, cudaStream_t s);
cudaError_t launch_to_offset(const Geom& g, const RefState& r, const double* q_plain, double* q_off, cudaStream_t s);
cudaError_t launch_from_offset(const Geom& g, const RefState& r, const double* q_off, double* q_plain,
                               cudaStream_t s);
// dst[i] = (double)src[i], i < n
cudaError_t launch_widen(long long n, const float* src, double* dst, cudaStream_t s);
// dst[i] = the binary32 narrowing of src[i] that the binary32 stage kernels apply
cudaError_t launch_narrow(long long n, const double* src, float* dst, cudaStream_t s);
// double-float register (5 hi fields, then 5 lo fields, binary32) <-> binary64
// state (5 fields).  split: v = src - ref (fields 0 and 4), hi = (float)v,
// lo = (float)(v - hi); join: dst = ((double)hi + (double)lo) + ref.  Pass a
// zero RefState to stay in deviation form.
cudaError_t launch_df_split(long long P, const RefState& r, const double* src, float* dst, cudaStream_t s);
cudaError_t launch_df_join(long long P, const RefState& r, const float* src, double* dst, cudaStream_t s);
// dst[i] = (double)src[2i] + (double)src[2i+1], i < n (exact): a stage field of
// interleaved double-float pairs (binary64-register double-float grids) as binary64
cudaError_t launch_pair_join(long long n, const float* src, double* dst, cudaStream_t s);
// dst[2i], dst[2i+1] = the double-float split of src[i] (split_f64), i < n
cudaError_t launch_pair_split(long long n, const double* src, float* dst, cudaStream_t s);
// Gather the plain conserved variables of count points (q64: binary64 state,
// or qdf: double-float state) into out[5][count]; NaN for indices outside [0, P).
cudaError_t launch_sample_state(long long P, const RefState& r, const double* q64, const float* qdf,
                                const long long* idx, int count, double* out, cudaStream_t s);
// KE/enstrophy of a binary64 offset state: per-CTA partials into scratch,
// then a fixed-order final sum into out[0..1].
int ke_num_partials(const Geom& g);
cudaError_t launch_ke(const Geom& g, const Coef<double>& c, const RefState& r, const double* q_off,
                      double* partials, double* out, cudaStream_t s);
// Fixed-order sum of n (ke, ens) pairs, scaled by 1/P.
cudaError_t launch_finalize_ke(const double* partials, int n, double inv_p, double* out, cudaStream_t s);

// Store-all (BL) variant (storeall.cu).
size_t storeall_scratch_doubles(const Geom& g, int elem_bytes);
// element offset of the residual R inside the store-all scratch
long long storeall_r_offset(const Geom& g);
cudaError_t launch_storeall_rhs_fp64(const Geom& g, const Coef<double>& c, const double* q_off, double* scratch,
                                     double* r_out, cudaStream_t s);
cudaError_t launch_storeall_rhs_fp32(const Geom& g, const Coef<float>& c, const void* q_off, bool in_fp64,
                                     float* scratch, float* r_out, cudaStream_t s);
cudaError_t launch_rk_update(const Geom& g, const void* r, bool r_fp64, const double* acc_in, double* acc_out,
                             void* q_out, bool out_fp64, double a_dt, double b_dt, cudaStream_t s);
// One derivative of one binary64 array (Eq. 6 for order 1, Eq. 7 for order 2)
// along one axis into its own array, as the store-all variant computes them.
cudaError_t launch_derivative_fp64(const Geom& g, const Coef<double>& c, const double* f, double* df, int axis,
                                   int order, cudaStream_t s);

// The paper's other evaluation strategies, binary64 (algorithms.cu): alg is
// SBLI_RS, SBLI_SS, SBLI_RA, SBLI_SN or SBLI_SN2.  r_out != nullptr writes R
// instead of the stage update.
bool algorithm_stores_gradients(int alg);
size_t algorithm_scratch_doubles(const Geom& g, int alg);
cudaError_t launch_algorithm_stage(int alg, const Geom& g, const Coef<double>& c, const double* q_in,
                                   const double* acc_in, double* acc_out, double* q_out, double* r_out, double a_dt,
                                   double b_dt, double* scratch, cudaStream_t s);

// Record msg as this host thread's sbli_last_error() and return code.
int set_last_error(int code, const char* msg);

// Wrap i into [0, n) for |i| < 2^30.
__host__ __device__ inline int wrapi(int i, int n) {
  int r = i % n;
  return r < 0 ? r + n : r;
}

}  // namespace sbli
