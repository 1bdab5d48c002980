// fused_fp64.cu -- binary64 instantiations of the fused stage kernel
// (32 x 8 tiles: 80-byte records fill 194.5 KiB of shared memory per CTA).
#include "fused_stage.cuh"

namespace sbli {

template <int TY>
static cudaError_t dispatch64(const StageArgs& a, const Coef<double>& c, bool rhs_only, cudaStream_t s) {
  if (rhs_only) return launch_fused_t<double, double, double, TY, true, false>(a, c, s);
  if (a.ke_partials) return launch_fused_t<double, double, double, TY, false, true>(a, c, s);
  return launch_fused_t<double, double, double, TY, false, false>(a, c, s);
}

cudaError_t launch_fused_fp64(const StageArgs& a, const Coef<double>& c, const FusedConfig& cfg, bool rhs_only,
                              cudaStream_t s) {
  switch (cfg.ty) {
    case 8: return dispatch64<8>(a, c, rhs_only, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace sbli
