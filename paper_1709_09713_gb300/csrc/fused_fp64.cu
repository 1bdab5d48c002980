// fused_fp64.cu -- binary64 instantiations of the fused stage kernel
// (32 x 8 tiles: 80-byte records fill 194.5 KiB of shared memory per CTA with
// the five-plane ring, 124 KiB with the x2 queue in TMEM).
#include "fused_stage.cuh"

namespace sbli {

template <int TY, bool ZT>
static cudaError_t dispatch64(const StageArgs& a, const Coef<double>& c, bool rhs_only, cudaStream_t s) {
  if (rhs_only) return launch_fused_t<double, double, double, TY, true, false, false, ZT>(a, c, s);
  if (a.ke_partials) return launch_fused_t<double, double, double, TY, false, true, false, ZT>(a, c, s);
  return launch_fused_t<double, double, double, TY, false, false, false, ZT>(a, c, s);
}

cudaError_t launch_fused_fp64(const StageArgs& a, const Coef<double>& c, const FusedConfig& cfg, bool rhs_only,
                              cudaStream_t s) {
  switch (cfg.ty) {
    case 8: return cfg.zq ? dispatch64<8, true>(a, c, rhs_only, s) : dispatch64<8, false>(a, c, rhs_only, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace sbli
