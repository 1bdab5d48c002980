// fused_fp32.cu -- binary32 instantiations of the fused stage kernel.  Every
// stage reads binary32 fields (stage 0 the binary32 copy of the state that the
// previous step's last stage wrote); the accumulator is binary64 or, for the
// double-float mode, a hi/lo binary32 pair.  The residual alone (RHS only)
// may also read the binary64 state.  Tiles 32 x 8 (two CTAs per SM) and 32 x 16 (one
// CTA of 16 warps per SM); the TMEM-queue and two-column kernels are in
// their own files.
#include "fused_stage.cuh"

namespace sbli {

template <int TY>
static cudaError_t dispatch32(const StageArgs& a, const Coef<float>& c, bool in_fp64, bool rhs_only,
                              cudaStream_t s) {
  if (rhs_only) {
    if (in_fp64) return launch_fused_t<float, double, float, TY, true, false>(a, c, s);
    return launch_fused_t<float, float, float, TY, true, false>(a, c, s);
  }
  if (in_fp64) return cudaErrorInvalidValue;  // stages read the binary32 copy of the state
  if (a.ke_partials) return launch_fused_t<float, float, float, TY, false, true>(a, c, s);
  return launch_fused_t<float, float, float, TY, false, false>(a, c, s);
}

cudaError_t launch_fused_fp32(const StageArgs& a, const Coef<float>& c, const FusedConfig& cfg, bool in_fp64,
                              bool rhs_only, cudaStream_t s) {
  if (cfg.px == 2) return launch_fused_fp32_pair(a, c, cfg, in_fp64, false, rhs_only, s);
  if (cfg.zq) return launch_fused_fp32_tmem(a, c, cfg, in_fp64, false, rhs_only, s);
  switch (cfg.ty) {
    case 8: return dispatch32<8>(a, c, in_fp64, rhs_only, s);
    case 16: return dispatch32<16>(a, c, in_fp64, rhs_only, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int TY>
static cudaError_t dispatch32df(const StageArgs& a, const Coef<float>& c, bool rhs_only, cudaStream_t s) {
  if (rhs_only) return launch_fused_t<float, float, float, TY, true, false, false>(a, c, s);
  if (a.ke_partials) return launch_fused_t<float, float, float, TY, false, true, true>(a, c, s);
  return launch_fused_t<float, float, float, TY, false, false, true>(a, c, s);
}

cudaError_t launch_fused_fp32df(const StageArgs& a, const Coef<float>& c, const FusedConfig& cfg, bool rhs_only,
                                cudaStream_t s) {
  if (cfg.px == 2) return launch_fused_fp32_pair(a, c, cfg, false, true, rhs_only, s);
  if (cfg.zq) return launch_fused_fp32_tmem(a, c, cfg, false, true, rhs_only, s);
  switch (cfg.ty) {
    case 8: return dispatch32df<8>(a, c, rhs_only, s);
    case 16: return dispatch32df<16>(a, c, rhs_only, s);
    default: return cudaErrorInvalidValue;
  }
}

int fused_num_ctas(const Geom& g, const FusedConfig& cfg) {
  const long long w = TX * (cfg.px == 2 ? 2 : 1);
  const long long gx = (g.n0 + w - 1) / w, gy = (g.n1 + cfg.ty - 1) / cfg.ty, gz = (g.n2 + cfg.zc - 1) / cfg.zc;
  return (int)(gx * gy * gz);
}

}  // namespace sbli
