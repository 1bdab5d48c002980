// batch_kernel.cuh -- the multi-member stage launch shared by ensembles
// (batch.cu) and the serving loop (server.cu).
#pragma once

#include "sbli_internal.cuh"

namespace sbli {

constexpr int BATCH_MAX_MEMBERS = 64;  // members per launch (parameter space bound)

template <typename T>
struct BatchParams {
  int count;                                  // members in this launch
  long long total_items;                      // sum of the members' items
  long long item_begin[BATCH_MAX_MEMBERS + 1];
  int tiles_x[BATCH_MAX_MEMBERS];
  int tiles_y[BATCH_MAX_MEMBERS];
  StageArgs a[BATCH_MAX_MEMBERS];             // geometry, zc, stage pointers, a_k dt, b_k dt
  Coef<T> c[BATCH_MAX_MEMBERS];
  double* ke_items;                           // per-item (ke, ens) partials, or nullptr
};

// One persistent launch of stage work for p.count members (grid = CTAs).
// in64: the members' stage inputs are binary64 (binary64-register kernels;
// binary32 stages always read binary32 fields, so it must be false for them);
// df: binary32 stages with the double-float accumulator (dacc pointers);
// zq: x2-neighbour records from a per-thread TMEM queue (1) or the
// shared-memory ring (0), as for single grids (bitwise the same results).
template <typename T>
cudaError_t launch_batch_t(const BatchParams<T>& p, bool in64, int grid, cudaStream_t s, bool df, int zq);

// The z-queue mode a batch of this precision starts with: binary32 members
// (either accumulator) the TMEM queue, binary64 and double-float arithmetic
// the shared-memory ring (their measured faster choices on single grids).
inline int batch_default_zq(int precision) { return precision == SBLI_FP32 || precision == SBLI_FP32_DF ? 1 : 0; }

// Resident CTAs per SM of the multi-member launch: binary32 members run the
// TMEM-queue kernel (59 KiB shared, 80 registers: 3 per SM) or the shared
// ring (113 KiB: 2 per SM); binary64 and double-float-arithmetic members
// the 194.5 KiB shared ring or the 124 KiB TMEM-queue kernel (1 per SM).
inline int batch_ctas_per_sm(int precision, int zq) {
  if (precision == SBLI_FP32 || precision == SBLI_FP32_DF) return zq ? 3 : 2;
  return 1;
}

// Work items (z chunk of zc planes x 32 x 8 tile) of one member; batch_zc is
// the planes per item a member starts with.
inline int batch_zc(int n2) { return n2 < 32 ? n2 : 32; }
inline long long member_items(const int n[3], int zc) {
  return (long long)((n[0] + 31) / 32) * ((n[1] + 7) / 8) * ((n[2] + zc - 1) / zc);
}
inline long long member_items(const int n[3]) { return member_items(n, batch_zc(n[2])); }

// Per member m: fixed-order sum of item partials [begin[m], begin[m+1]) times inv_p[m].
cudaError_t launch_batch_ke_finalize(const double* items, const long long* begin, const double* inv_p, double* out,
                                     int count, cudaStream_t s);

}  // namespace sbli
