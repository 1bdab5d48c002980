// fused_fp32_pair.cu -- binary32 stage kernels in which each thread owns two
// columns of a 64 x 8 tile (x and x + 32), computed together in f32x2
// (both accumulator kinds).  Shared-memory records hold both columns'
// values side by side, so every record access moves two points.
#include "fused_stage.cuh"

namespace sbli {

cudaError_t launch_fused_fp32_pair(const StageArgs& a, const Coef<float>& cf, const FusedConfig& cfg, bool in_fp64,
                                   bool df, bool rhs_only, cudaStream_t s) {
  if (cfg.ty != 8) return cudaErrorInvalidValue;
  Coef<f32x2> c;
  for (int i = 0; i < 3; ++i) {
    c.c1[i] = f32x2(cf.c1[i], cf.c1[i]);
    c.c2[i] = f32x2(cf.c2[i], cf.c2[i]);
    c.e0[i] = f32x2(cf.e0[i], cf.e0[i]);
    c.e1[i] = f32x2(cf.e1[i], cf.e1[i]);
    c.e2[i] = f32x2(cf.e2[i], cf.e2[i]);
  }
  c.gm1 = f32x2(cf.gm1, cf.gm1);
  c.gM2 = f32x2(cf.gM2, cf.gM2);
  c.gm1x2 = f32x2(cf.gm1x2, cf.gm1x2);
  c.hgM2 = f32x2(cf.hgM2, cf.hgM2);
  c.inv_re = f32x2(cf.inv_re, cf.inv_re);
  c.kappa = f32x2(cf.kappa, cf.kappa);
  c.H0 = f32x2(cf.H0, cf.H0);
  if (rhs_only) {
    if (in_fp64) return launch_fused_t<f32x2, double, float, 8, true, false>(a, c, s);
    return launch_fused_t<f32x2, float, float, 8, true, false>(a, c, s);
  }
  if (df) {
    if (a.ke_partials) return launch_fused_t<f32x2, float, float, 8, false, true, true>(a, c, s);
    return launch_fused_t<f32x2, float, float, 8, false, false, true>(a, c, s);
  }
  if (in_fp64) return cudaErrorInvalidValue;  // stages read the binary32 copy of the state
  if (a.ke_partials) return launch_fused_t<f32x2, float, float, 8, false, true>(a, c, s);
  return launch_fused_t<f32x2, float, float, 8, false, false>(a, c, s);
}

}  // namespace sbli
