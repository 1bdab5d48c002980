// fused_fp32_zpair.cu -- launchers of the binary32 stage kernel with two x2
// planes per thread (fused_zpair.cuh), both accumulator kinds: 32 x 8 tiles,
// two CTAs per SM (83 KiB of shared memory, 256 TMEM columns each).
#include "fused_zpair.cuh"

namespace sbli {

template <bool DF, bool WITH_KE>
static cudaError_t launch_zp(const StageArgs& a, const Coef<f32x2>& c, cudaStream_t s) {
  auto k = fused_zpair_kernel<DF, WITH_KE>;
  const size_t smem = sizeof(zp::Smem);
  static std::atomic<unsigned long long> done{0};
  if (cudaError_t e = ensure_smem_limit(k, smem, done)) return e;
  k<<<fused_grid<zp::TY>(a.g, a.zc), zp::NT, smem, s>>>(a, c);
  return cudaGetLastError();
}

cudaError_t launch_fused_fp32_zpair(const StageArgs& a, const Coef<float>& cf, const FusedConfig& cfg, bool df,
                                    cudaStream_t s) {
  if (cfg.ty != zp::TY || a.r_out) return cudaErrorInvalidValue;  // stages only, 32 x 8 tiles
  const Coef<f32x2> c = zp::pair_coef(cf);
  if (df) return a.ke_partials ? launch_zp<true, true>(a, c, s) : launch_zp<true, false>(a, c, s);
  return a.ke_partials ? launch_zp<false, true>(a, c, s) : launch_zp<false, false>(a, c, s);
}

}  // namespace sbli
