// fused_df64.cu -- the fused stage kernel with binary64 storage and
// double-float arithmetic (dfloat.cuh): the state and accumulator are
// binary64, updated in place; every stage reads its stencil input as
// interleaved (hi, lo) binary32 pairs (the split a binary64 value gets, done
// once by the stage that writes the field: stages 0 and 1 write the next
// stage's field, stage 2 the pair copy of the new state, which the next step's
// stage 0 reads); every derivative and the residual run on the binary32 pipe,
// and the Runge-Kutta update of the binary64 accumulator is the binary64 FMA
// of the binary64 path.  The residual alone reads the binary64 state.
#include "fused_stage.cuh"

namespace sbli {

template <int TY, bool ZT>
static cudaError_t dispatch_df64(const StageArgs& a, const Coef<dfloat>& c, bool rhs_only, bool in_pairs,
                                 cudaStream_t s) {
  if (rhs_only) return launch_fused_t<dfloat, double, double, TY, true, false, false, ZT>(a, c, s);
  if (!in_pairs) return cudaErrorInvalidValue;  // single-grid stages read pair fields
  if (a.ke_partials) return launch_fused_t<dfloat, dfloat, dfloat, TY, false, true, false, ZT>(a, c, s);
  return launch_fused_t<dfloat, dfloat, dfloat, TY, false, false, false, ZT>(a, c, s);
}

cudaError_t launch_fused_df64(const StageArgs& a, const Coef<dfloat>& c, const FusedConfig& cfg, bool rhs_only,
                              bool in_pairs, cudaStream_t s) {
  switch (cfg.ty) {
    case 8:
      return cfg.zq ? dispatch_df64<8, true>(a, c, rhs_only, in_pairs, s)
                    : dispatch_df64<8, false>(a, c, rhs_only, in_pairs, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace sbli
