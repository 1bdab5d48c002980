// fused_fp32_tmem.cu -- binary32 stage kernels whose x2-neighbour records
// come from a per-thread queue in tensor memory instead of the shared-memory
// ring (both accumulator kinds): tiles 32 x 8 with three full-record planes
// in shared memory (three CTAs per SM) and 32 x 16 with four (two barriers
// per plane).
#include "fused_stage.cuh"

namespace sbli {

template <int TY>
static cudaError_t dispatch_tm(const StageArgs& a, const Coef<float>& c, bool in_fp64, bool df, bool rhs_only,
                               cudaStream_t s) {
  if (rhs_only) {
    if (in_fp64) return launch_fused_t<float, double, float, TY, true, false, false, true>(a, c, s);
    return launch_fused_t<float, float, float, TY, true, false, false, true>(a, c, s);
  }
  if (df) {
    if (a.ke_partials) return launch_fused_t<float, float, float, TY, false, true, true, true>(a, c, s);
    return launch_fused_t<float, float, float, TY, false, false, true, true>(a, c, s);
  }
  if (in_fp64) return cudaErrorInvalidValue;  // stages read the binary32 copy of the state
  if (a.ke_partials) return launch_fused_t<float, float, float, TY, false, true, false, true>(a, c, s);
  return launch_fused_t<float, float, float, TY, false, false, false, true>(a, c, s);
}

cudaError_t launch_fused_fp32_tmem(const StageArgs& a, const Coef<float>& c, const FusedConfig& cfg, bool in_fp64,
                                   bool df, bool rhs_only, cudaStream_t s) {
  switch (cfg.ty) {
    case 8: return dispatch_tm<8>(a, c, in_fp64, df, rhs_only, s);
    case 16: return dispatch_tm<16>(a, c, in_fp64, df, rhs_only, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace sbli
