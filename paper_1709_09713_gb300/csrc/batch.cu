// batch.cu -- ensembles of uneven grids advanced together: one persistent
// launch per Runge-Kutta stage over every member's work items, step loops
// captured as CUDA graphs, and the C ABI of sbli_batch_* (include/sbli.h).
//
// A member is one Taylor-Green problem (own n0 x n1 x n2, Re, M, Pr, gamma,
// L, amplitude).  Its work is split into items (z chunk, 32 x TY tile); items
// of all members are numbered consecutively, chunk-major inside a member so
// that CTAs running at the same time work on neighbouring tiles of the same
// planes.  The member table travels in the kernel's parameter space, so a
// captured graph needs no device-side table.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "batch_kernel.cuh"
#include "fused_stage.cuh"

namespace sbli {

// ZT: x2-neighbour records in a TMEM queue and the 3-slot shared ring (binary32),
// the CTA's TMEM columns held for all of its work items.  DF: binary32 stages
// with the double-float accumulator (SBLI_FP32_DF members).
template <typename T, typename TIN, typename TOUT, int TY, bool WITH_KE, bool ZT = false, bool DF = false>
__global__ void __launch_bounds__(TX* TY, fused_min_blocks<T, TY, ZT>())
    batch_stage_kernel(const __grid_constant__ BatchParams<T> p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  FusedSmem<T, TY, ZT>& sm = *reinterpret_cast<FusedSmem<T, TY, ZT>*>(smem_raw);
  constexpr int NCOL = tmem_columns<TY, T>();
  constexpr int NCOL2 = tmem_columns2<TY, T>();
  uint32_t tbase = 0, tbase2 = 0;
  if (ZT) tmem_acquire<NCOL, NCOL2>(sm.tmem_base, tbase, tbase2);
  for (long long item = blockIdx.x; item < p.total_items; item += gridDim.x) {
    // member owning this item (binary search over item_begin)
    int lo = 0, hi = p.count - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (p.item_begin[mid] <= item) lo = mid;
      else hi = mid - 1;
    }
    const StageArgs& a = p.a[lo];
    const long long local = item - p.item_begin[lo];
    const int ntile = p.tiles_x[lo] * p.tiles_y[lo];
    const int chunk = (int)(local / ntile);
    const int tile = (int)(local - (long long)chunk * ntile);
    const int bx = tile % p.tiles_x[lo], by = tile / p.tiles_x[lo];
    const int zbeg = chunk * a.zc;
    double ke = 0.0, ens = 0.0;
    fused_march<T, TIN, TOUT, TY, false, WITH_KE, DF, ZT>(a, p.c[lo], bx, by, zbeg, zbeg + a.zc, sm, ke, ens,
                                                            tbase, tbase2);
    if (WITH_KE) block_reduce_pair<TX * TY>(sm.red, ke, ens, p.ke_items + 2 * item);
  }
  if (ZT) tmem_release<NCOL, NCOL2>(tbase, tbase2);
}

// Per member: fixed-order sum of its items' partials, scaled by 1/P.
__global__ void __launch_bounds__(256) batch_ke_finalize(const double* __restrict__ items,
                                                         const long long* __restrict__ begin,
                                                         const double* __restrict__ inv_p, double* __restrict__ out) {
  const int m = blockIdx.x;
  double a = 0.0, b = 0.0;
  for (long long i = begin[m] + threadIdx.x; i < begin[m + 1]; i += 256) {
    a += items[2 * i];
    b += items[2 * i + 1];
  }
  __shared__ double red[2][32];
  block_reduce_pair<256>(red, a, b, out + 2 * m);
  if (threadIdx.x == 0) {
    out[2 * m] *= inv_p[m];
    out[2 * m + 1] *= inv_p[m];
  }
}

// ---- launchers (declared in batch_kernel.cuh)
// Launch one instantiation, setting its shared-memory limit on first use.
template <typename T, typename TIN, typename TOUT, bool WITH_KE, bool ZT, bool DF>
static cudaError_t launch_batch_k(const BatchParams<T>& p, int grid, cudaStream_t s) {
  auto k = batch_stage_kernel<T, TIN, TOUT, 8, WITH_KE, ZT, DF>;
  const size_t smem = sizeof(FusedSmem<T, 8, ZT>);
  static std::atomic<unsigned long long> done{0};
  if (cudaError_t e = ensure_smem_limit(k, smem, done)) return e;
  k<<<grid, TX * 8, smem, s>>>(p);
  return cudaGetLastError();
}

template <typename T, typename TIN, typename TOUT, bool DF>
static cudaError_t launch_batch_zq(const BatchParams<T>& p, int grid, cudaStream_t s, int zq) {
  if (zq)
    return p.ke_items ? launch_batch_k<T, TIN, TOUT, true, true, DF>(p, grid, s)
                      : launch_batch_k<T, TIN, TOUT, false, true, DF>(p, grid, s);
  return p.ke_items ? launch_batch_k<T, TIN, TOUT, true, false, DF>(p, grid, s)
                    : launch_batch_k<T, TIN, TOUT, false, false, DF>(p, grid, s);
}

// binary32 members (every stage input is binary32; the grid is sized by the
// caller with batch_ctas_per_sm for the z-queue mode)
template <>
cudaError_t launch_batch_t<float>(const BatchParams<float>& p, bool in64, int grid, cudaStream_t s, bool df, int zq) {
  if (in64) return cudaErrorInvalidValue;  // stages read the binary32 copy of the state
  if (df) return launch_batch_zq<float, float, float, true>(p, grid, s, zq);
  return launch_batch_zq<float, float, float, false>(p, grid, s, zq);
}

// double-float arithmetic members: every stage reads a field of (hi, lo)
// pairs and writes its stage field as pairs
template <>
cudaError_t launch_batch_t<dfloat>(const BatchParams<dfloat>& p, bool in64, int grid, cudaStream_t s, bool, int zq) {
  if (in64) return cudaErrorInvalidValue;
  return launch_batch_zq<dfloat, dfloat, dfloat, false>(p, grid, s, zq);
}

template <>
cudaError_t launch_batch_t<double>(const BatchParams<double>& p, bool, int grid, cudaStream_t s, bool, int zq) {
  return launch_batch_zq<double, double, double, false>(p, grid, s, zq);
}

cudaError_t launch_batch_ke_finalize(const double* items, const long long* begin, const double* inv_p, double* out,
                                     int count, cudaStream_t s) {
  batch_ke_finalize<<<count, 256, 0, s>>>(items, begin, inv_p, out);
  return cudaGetLastError();
}

}  // namespace sbli

using namespace sbli;

namespace {

int bfail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  return set_last_error(code, buf);
}

int bcuda(cudaError_t e, const char* what) {
  return bfail(SBLI_ECUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

#define SBLI_BTRY(expr, what)                         \
  do {                                                \
    cudaError_t e_ = (expr);                          \
    if (e_ != cudaSuccess) return bcuda(e_, what);    \
  } while (0)

constexpr size_t BALIGN = 256;
size_t balign(size_t v) { return (v + BALIGN - 1) / BALIGN * BALIGN; }

struct MemberLayout {
  int n[3];
  int zc;  // planes per work item (the schedule; batch_zc at creation)
  long long P;
  size_t off64, off32;  // byte offsets inside the binary64 / binary32 register regions
};

struct BatchLayout {
  std::vector<MemberLayout> m;
  size_t reg64, reg32;  // bytes of one register region
  int n64, n32;
  size_t items_bytes, misc_bytes, total;
  long long total_items;
};


// binary64 registers with the three-register rotation (binary64 and
// double-float arithmetic)
bool batch_f64_registers(int precision) { return precision == SBLI_FP64 || precision == SBLI_DF64; }

BatchLayout batch_layout(int count, const int* n, int precision) {
  BatchLayout L;
  L.m.resize(count);
  size_t o64 = 0, o32 = 0;
  L.total_items = 0;
  for (int i = 0; i < count; ++i) {
    MemberLayout& M = L.m[i];
    for (int a = 0; a < 3; ++a) M.n[a] = n[3 * i + a];
    M.P = (long long)M.n[0] * M.n[1] * M.n[2];
    M.zc = batch_zc(M.n[2]);
    M.off64 = o64;
    M.off32 = o32;
    o64 += balign((size_t)M.P * 5 * sizeof(double));
    o32 += balign((size_t)M.P * 5 * sizeof(float));
    L.total_items += member_items(M.n, std::min(4, M.n[2]));  // the most items any schedule gives
  }
  L.reg64 = o64;
  L.reg32 = batch_f64_registers(precision) ? 0 : o32;
  L.n64 = batch_f64_registers(precision) ? 3 : 2;
  L.n32 = batch_f64_registers(precision) ? 0 : 2;
  L.items_bytes = balign((size_t)(2 * L.total_items + 2) * sizeof(double));
  L.total_items = 0;
  for (const MemberLayout& M : L.m) L.total_items += member_items(M.n, M.zc);
  // per member: KE result pair, 1/P, item begin; plus the KE kernel partials
  L.misc_bytes = balign((size_t)count * 2 * sizeof(double)) + balign((size_t)count * sizeof(double)) +
                 balign((size_t)(count + 1) * sizeof(long long)) + balign(2 * 1024 * sizeof(double));
  L.total = L.reg64 * L.n64 + L.reg32 * L.n32 + L.items_bytes + L.misc_bytes;
  return L;
}

}  // namespace

struct sbli_batch {
  int count, precision;
  std::vector<sbli_params> params;
  BatchLayout L;
  cudaStream_t stream, cap_stream;
  char* reg64[3];
  char* reg32[2];
  double* ke_items;
  double* ke_out;     // count pairs
  double* inv_p;      // count
  long long* begin;   // count + 1 (device copy of item_begin)
  double* ke_scratch; // partials of the single-member KE kernel
  int state;
  long long steps_done;
  int zq;             // z-queue mode of the batch kernel (the schedule)
  int grid_ctas;      // persistent grid size
  // one graph of GRAPH_STEPS steps per starting rotation
  static constexpr int GRAPH_STEPS = 6;
  cudaGraphExec_t graph[3];
  double graph_dt[3];
};

namespace {

// Double-float members (SBLI_DF64) keep their binary64 state and accumulator
// in register 0, updated in place, and the (hi, lo) pair copy of the state in
// register `state` (1 or 2), as single grids do; every other precision keeps
// its state in register `state`.
int batch_initial_state(int precision) { return precision == SBLI_DF64 ? 1 : 0; }
int batch_next_state(const sbli_batch* b, int s) {
  if (b->precision == SBLI_DF64) return 3 - s;
  return batch_f64_registers(b->precision) ? (s + 1) % 3 : 1 - s;
}
int state_reg(const sbli_batch* b) { return b->precision == SBLI_DF64 ? 0 : b->state; }
int free_reg(const sbli_batch* b) { return b->precision == SBLI_DF64 ? 3 - b->state : (b->state + 1) % b->L.n64; }

Geom member_geom(const MemberLayout& M) { return Geom{M.n[0], M.n[1], M.n[2], M.P}; }

// StageArgs of member m for stage k in rotation `state` (same scheme as a single grid).
StageArgs member_stage(const sbli_batch* b, int m, int k, int state, double dt, bool* in64) {
  const MemberLayout& M = b->L.m[m];
  StageArgs a{};
  a.g = member_geom(M);
  a.zc = M.zc;
  a.a_dt = RK_A[k] * dt;
  a.b_dt = RK_B[k] * dt;
  a.amb_dt = (RK_A[k] - RK_B[k]) * dt;
  a.b_dt32 = (float)a.b_dt;
  a.amb_dt32 = (float)a.amb_dt;
  a.df_normalize = (k == 2);
  auto r64 = [&](int r) { return reinterpret_cast<double*>(b->reg64[r] + M.off64); };
  auto r32 = [&](int r) { return reinterpret_cast<float*>(b->reg32[r] + M.off32); };
  if (b->precision == SBLI_DF64) {
    // accumulator in place in register 0; stage fields of (hi, lo) pairs
    // alternate between registers `state` (the pair copy of Q^n) and 3 - state
    double* S = r64(0);
    double* Pa = r64(state);
    double* Pb = r64(3 - state);
    *in64 = false;
    a.acc_in = S;
    a.acc_out = S;
    if (k == 0) { a.q_in = Pa; a.q_out = Pb; }
    else if (k == 1) { a.q_in = Pb; a.q_out = Pa; }
    else { a.q_in = Pa; a.q_out = Pb; }  // a_3 = b_3: the pair copy of Q^{n+1}
  } else if (batch_f64_registers(b->precision)) {
    double* S = r64(state);
    double* A = r64((state + 1) % 3);
    double* B = r64((state + 2) % 3);
    *in64 = true;
    if (k == 0) { a.q_in = S; a.acc_in = S; a.acc_out = A; a.q_out = B; }
    else if (k == 1) { a.q_in = B; a.acc_in = A; a.acc_out = A; a.q_out = S; }
    else { a.q_in = S; a.acc_in = A; a.acc_out = A; a.q_out = nullptr; }
  } else if (b->precision == SBLI_FP32_DF) {
    // state and accumulator as double-float pairs (hi fields, then lo fields)
    float* S = reinterpret_cast<float*>(r64(state));
    float* A = reinterpret_cast<float*>(r64(1 - state));
    *in64 = false;
    if (k == 0) { a.q_in = S; a.dacc_in = S; a.dacc_out = A; a.q_out = r32(0); }
    else if (k == 1) { a.q_in = r32(0); a.dacc_in = A; a.dacc_out = A; a.q_out = r32(1); }
    else { a.q_in = r32(1); a.dacc_in = A; a.dacc_out = A; a.q_out = nullptr; }
  } else {
    // binary64 state and accumulator; binary32 register `state` holds the
    // binary32 copy of the state (as for single grids)
    double* S = r64(state);
    double* A = r64(1 - state);
    float* Cs = r32(state);
    float* Ds = r32(1 - state);
    *in64 = false;
    if (k == 0) { a.q_in = Cs; a.acc_in = S; a.acc_out = A; a.q_out = Ds; }
    else if (k == 1) { a.q_in = Ds; a.acc_in = A; a.acc_out = A; a.q_out = Cs; }
    else { a.q_in = Cs; a.acc_in = A; a.acc_out = A; a.q_out = Ds; }
  }
  return a;
}

template <typename T>
cudaError_t enqueue_batch_stage_t(sbli_batch* b, int k, int state, double dt, double* ke_items, cudaStream_t s) {
  BatchParams<T> p;
  memset(&p, 0, sizeof p);
  p.count = b->count;
  p.ke_items = ke_items;
  long long acc = 0;
  bool in64 = true;
  for (int m = 0; m < b->count; ++m) {
    const MemberLayout& M = b->L.m[m];
    p.item_begin[m] = acc;
    p.tiles_x[m] = (M.n[0] + TX - 1) / TX;
    p.tiles_y[m] = (M.n[1] + 7) / 8;
    acc += member_items(M.n, M.zc);
    p.a[m] = member_stage(b, m, k, state, dt, &in64);
    p.c[m] = make_coef<T>(M.n, b->params[m]);
  }
  p.item_begin[b->count] = acc;
  p.total_items = acc;
  return launch_batch_t<T>(p, in64, b->grid_ctas, s, b->precision == SBLI_FP32_DF, b->zq);
}

cudaError_t enqueue_batch_stage(sbli_batch* b, int k, int state, double dt, double* ke_items, cudaStream_t s) {
  if (b->precision == SBLI_FP64) return enqueue_batch_stage_t<double>(b, k, state, dt, ke_items, s);
  if (b->precision == SBLI_DF64) return enqueue_batch_stage_t<dfloat>(b, k, state, dt, ke_items, s);
  return enqueue_batch_stage_t<float>(b, k, state, dt, ke_items, s);
}

void batch_drop_graphs(sbli_batch* b) {
  for (int r = 0; r < 3; ++r) {
    if (b->graph[r]) cudaGraphExecDestroy(b->graph[r]);
    b->graph[r] = nullptr;
  }
}

int batch_build_graph(sbli_batch* b, int state, double dt) {
  if (b->graph[state] && b->graph_dt[state] == dt) return SBLI_OK;
  if (b->graph[state]) {
    cudaGraphExecDestroy(b->graph[state]);
    b->graph[state] = nullptr;
  }
  SBLI_BTRY(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
  int st = state;
  cudaError_t err = cudaSuccess;
  for (int s = 0; s < sbli_batch::GRAPH_STEPS && err == cudaSuccess; ++s) {
    for (int k = 0; k < 3 && err == cudaSuccess; ++k) err = enqueue_batch_stage(b, k, st, dt, nullptr, b->cap_stream);
    st = batch_next_state(b, st);
  }
  cudaGraph_t graph = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(b->cap_stream, &graph);
  if (err != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return bcuda(err, "batch launch during capture");
  }
  if (e2 != cudaSuccess) return bcuda(e2, "cudaStreamEndCapture");
  cudaGraphExec_t exec = nullptr;
  cudaError_t e3 = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e3 != cudaSuccess) return bcuda(e3, "cudaGraphInstantiate");
  b->graph[state] = exec;
  b->graph_dt[state] = dt;
  return SBLI_OK;
}

// Item ranges of the members under the current schedule, for the KE
// finalisation (device copy, written on the batch's stream).
cudaError_t upload_item_begin(sbli_batch* b) {
  std::vector<long long> beg(b->count + 1);
  long long acc = 0;
  for (int m = 0; m < b->count; ++m) {
    beg[m] = acc;
    acc += member_items(b->L.m[m].n, b->L.m[m].zc);
  }
  beg[b->count] = acc;
  b->L.total_items = acc;
  cudaError_t e = cudaMemcpyAsync(b->begin, beg.data(), (b->count + 1) * sizeof(long long), cudaMemcpyHostToDevice,
                                  b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);  // beg is a host temporary
  return e;
}

// Apply a schedule (z-queue mode, planes per item of each member); the
// captured step graphs are rebuilt on the next step.
cudaError_t apply_schedule(sbli_batch* b, int zq, const std::vector<int>& zc) {
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  b->zq = zq;
  b->grid_ctas = sms * batch_ctas_per_sm(b->precision, zq);
  for (int m = 0; m < b->count; ++m) b->L.m[m].zc = zc[m];
  batch_drop_graphs(b);
  return upload_item_begin(b);
}

int check_batch(const sbli_batch* b, int member) {
  if (!b) return bfail(SBLI_EINVAL, "null batch handle");
  if (member < 0 || member >= b->count) return bfail(SBLI_EINVAL, "member %d not in 0..%d", member, b->count - 1);
  return SBLI_OK;
}

}  // namespace

extern "C" {

int sbli_batch_workspace_bytes(int count, const int* n, int precision, size_t* bytes) {
  if (!bytes || !n) return bfail(SBLI_EINVAL, "null argument");
  if (count < 1 || count > BATCH_MAX_MEMBERS) return bfail(SBLI_EINVAL, "count %d not in 1..%d", count, BATCH_MAX_MEMBERS);
  if (precision < SBLI_FP64 || precision > SBLI_DF64) return bfail(SBLI_EINVAL, "unknown precision %d", precision);
  for (int i = 0; i < count; ++i) {
    const int* m = n + 3 * i;
    if (m[0] < 5 || m[1] < 5 || m[2] < 5 || (long long)m[0] * m[1] >= (1LL << 31) ||
        (long long)m[0] * m[1] * m[2] >= (1LL << 32))
      return bfail(SBLI_EINVAL, "member %d grid %d x %d x %d invalid", i, m[0], m[1], m[2]);
  }
  *bytes = batch_layout(count, n, precision).total;
  return SBLI_OK;
}

int sbli_batch_create(sbli_batch** out, int count, const int* n, const sbli_params* params, int precision,
                      void* workspace, size_t workspace_bytes, void* stream) {
  if (!out) return bfail(SBLI_EINVAL, "out is null");
  *out = nullptr;
  size_t need = 0;
  if (int rc = sbli_batch_workspace_bytes(count, n, precision, &need)) return rc;
  if (!params) return bfail(SBLI_EINVAL, "params is null");
  for (int i = 0; i < count; ++i) {
    const sbli_params& p = params[i];
    if (!(p.Re > 0) || !(p.Mach > 0) || !(p.Pr > 0) || !(p.gamma > 1) || !(p.L > 0) || isnan(p.Re) ||
        !isfinite(p.Mach) || !isfinite(p.Pr) || !isfinite(p.gamma) || !isfinite(p.L))
      return bfail(SBLI_EINVAL, "member %d: invalid physical parameters", i);
  }
  if (!workspace || ((uintptr_t)workspace) % BALIGN) return bfail(SBLI_EINVAL, "workspace must be 256-byte aligned device memory");
  if (workspace_bytes < need) return bfail(SBLI_ENOMEM, "workspace has %zu bytes, batch needs %zu", workspace_bytes, need);
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, workspace) != cudaSuccess || attr.type != cudaMemoryTypeDevice) {
    cudaGetLastError();
    return bfail(SBLI_EINVAL, "workspace is not device memory");
  }
  sbli_batch* b = new sbli_batch();
  b->count = count;
  b->precision = precision;
  b->params.assign(params, params + count);
  b->L = batch_layout(count, n, precision);
  b->stream = static_cast<cudaStream_t>(stream);
  memset(b->graph, 0, sizeof b->graph);
  char* w = static_cast<char*>(workspace);
  for (int r = 0; r < b->L.n64; ++r, w += b->L.reg64) b->reg64[r] = w;
  for (int r = 0; r < b->L.n32; ++r, w += b->L.reg32) b->reg32[r] = w;
  b->ke_items = reinterpret_cast<double*>(w);
  w += b->L.items_bytes;
  b->ke_out = reinterpret_cast<double*>(w);
  w += balign((size_t)count * 2 * sizeof(double));
  b->inv_p = reinterpret_cast<double*>(w);
  w += balign((size_t)count * sizeof(double));
  b->begin = reinterpret_cast<long long*>(w);
  w += balign((size_t)(count + 1) * sizeof(long long));
  b->ke_scratch = reinterpret_cast<double*>(w);
  b->state = batch_initial_state(b->precision);
  b->steps_done = 0;
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  b->zq = batch_default_zq(precision);
  b->grid_ctas = sms * batch_ctas_per_sm(precision, b->zq);
  // per-member constants for the KE finalisation
  std::vector<double> inv(count);
  for (int m = 0; m < count; ++m) inv[m] = 1.0 / (double)b->L.m[m].P;
  cudaError_t e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->inv_p, inv.data(), count * sizeof(double), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = upload_item_begin(b);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) {
    delete b;
    return bcuda(e, "batch set-up");
  }
  *out = b;
  return SBLI_OK;
}

int sbli_batch_destroy(sbli_batch* b) {
  if (!b) return SBLI_OK;
  cudaStreamSynchronize(b->stream);
  batch_drop_graphs(b);
  cudaStreamDestroy(b->cap_stream);
  delete b;
  return SBLI_OK;
}

int sbli_batch_count(const sbli_batch* b, int* count) {
  if (!b || !count) return bfail(SBLI_EINVAL, "null argument");
  *count = b->count;
  return SBLI_OK;
}

int sbli_batch_init_tgv(sbli_batch* b, const double* amplitudes) {
  if (int rc = check_batch(b, 0)) return rc;
  if (!amplitudes) return bfail(SBLI_EINVAL, "amplitudes is null");
  b->state = batch_initial_state(b->precision);
  b->steps_done = 0;
  for (int m = 0; m < b->count; ++m) {
    if (!isfinite(amplitudes[m])) return bfail(SBLI_EINVAL, "amplitude %d not finite", m);
    const MemberLayout& M = b->L.m[m];
    if (b->precision == SBLI_FP32_DF) {
      // binary64 deviation field into the free register, then split into hi/lo
      double* tmp = reinterpret_cast<double*>(b->reg64[1] + M.off64);
      SBLI_BTRY(launch_init_tgv(member_geom(M), b->params[m], amplitudes[m], tmp, b->stream), "init_tgv");
      SBLI_BTRY(launch_df_split(M.P, RefState{0.0, 0.0}, tmp, reinterpret_cast<float*>(b->reg64[0] + M.off64),
                                b->stream),
                "df_split");
      continue;
    }
    SBLI_BTRY(launch_init_tgv(member_geom(M), b->params[m], amplitudes[m],
                              reinterpret_cast<double*>(b->reg64[0] + M.off64), b->stream),
              "init_tgv");
    if (b->precision == SBLI_DF64)
      SBLI_BTRY(launch_pair_split(5 * M.P, reinterpret_cast<double*>(b->reg64[0] + M.off64),
                                  reinterpret_cast<float*>(b->reg64[b->state] + M.off64), b->stream),
                "pair_split");
    if (b->precision == SBLI_FP32)
      SBLI_BTRY(launch_narrow(5 * M.P, reinterpret_cast<double*>(b->reg64[0] + M.off64),
                              reinterpret_cast<float*>(b->reg32[0] + M.off32), b->stream),
                "narrow");
  }
  return SBLI_OK;
}

int sbli_batch_set_state(sbli_batch* b, int member, const double* q, int q_is_host) {
  if (int rc = check_batch(b, member)) return rc;
  if (!q) return bfail(SBLI_EINVAL, "q is null");
  const MemberLayout& M = b->L.m[member];
  double* dst = reinterpret_cast<double*>(b->reg64[state_reg(b)] + M.off64);
  double* tmp = reinterpret_cast<double*>(b->reg64[free_reg(b)] + M.off64);
  SBLI_BTRY(cudaMemcpyAsync(tmp, q, 5 * M.P * sizeof(double), q_is_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                            b->stream),
            "cudaMemcpyAsync");
  if (b->precision == SBLI_FP32_DF) {
    SBLI_BTRY(launch_df_split(M.P, make_ref(b->params[member]), tmp, reinterpret_cast<float*>(dst), b->stream),
              "df_split");
  } else {
    SBLI_BTRY(launch_to_offset(member_geom(M), make_ref(b->params[member]), tmp, dst, b->stream), "to_offset");
    if (b->precision == SBLI_DF64)
      SBLI_BTRY(launch_pair_split(5 * M.P, dst, reinterpret_cast<float*>(b->reg64[b->state] + M.off64), b->stream),
                "pair_split");
    if (b->precision == SBLI_FP32)
      SBLI_BTRY(launch_narrow(5 * M.P, dst, reinterpret_cast<float*>(b->reg32[b->state] + M.off32), b->stream),
                "narrow");
  }
  if (q_is_host) SBLI_BTRY(cudaStreamSynchronize(b->stream), "cudaStreamSynchronize");
  return SBLI_OK;
}

int sbli_batch_get_state(sbli_batch* b, int member, double* q, int q_is_host) {
  if (int rc = check_batch(b, member)) return rc;
  if (!q) return bfail(SBLI_EINVAL, "q is null");
  const MemberLayout& M = b->L.m[member];
  const double* src = reinterpret_cast<double*>(b->reg64[state_reg(b)] + M.off64);
  double* tmp = reinterpret_cast<double*>(b->reg64[free_reg(b)] + M.off64);
  if (b->precision == SBLI_FP32_DF) {
    SBLI_BTRY(launch_df_join(M.P, make_ref(b->params[member]), reinterpret_cast<const float*>(src), tmp, b->stream),
              "df_join");
  } else {
    SBLI_BTRY(launch_from_offset(member_geom(M), make_ref(b->params[member]), src, tmp, b->stream), "from_offset");
  }
  SBLI_BTRY(cudaMemcpyAsync(q, tmp, 5 * M.P * sizeof(double), q_is_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                            b->stream),
            "cudaMemcpyAsync");
  if (q_is_host) SBLI_BTRY(cudaStreamSynchronize(b->stream), "cudaStreamSynchronize");
  return SBLI_OK;
}

int sbli_batch_step_n(sbli_batch* b, int nsteps, double dt) {
  if (int rc = check_batch(b, 0)) return rc;
  if (nsteps < 0) return bfail(SBLI_EINVAL, "nsteps < 0");
  if (!(dt > 0) || !isfinite(dt)) return bfail(SBLI_EINVAL, "dt must be finite and > 0");
  int left = nsteps;
  while (left >= sbli_batch::GRAPH_STEPS) {
    if (int rc = batch_build_graph(b, b->state, dt)) return rc;
    SBLI_BTRY(cudaGraphLaunch(b->graph[b->state], b->stream), "cudaGraphLaunch");
    left -= sbli_batch::GRAPH_STEPS;  // a multiple of both rotation periods
    b->steps_done += sbli_batch::GRAPH_STEPS;
  }
  for (; left > 0; --left) {
    for (int k = 0; k < 3; ++k) SBLI_BTRY(enqueue_batch_stage(b, k, b->state, dt, nullptr, b->stream), "batch stage");
    b->state = batch_next_state(b, b->state);
    b->steps_done++;
  }
  return SBLI_OK;
}

int sbli_batch_step_n_history(sbli_batch* b, int nsteps, double dt, double* ke_hist_dev) {
  if (int rc = check_batch(b, 0)) return rc;
  if (nsteps < 0) return bfail(SBLI_EINVAL, "nsteps < 0");
  if (!ke_hist_dev && nsteps > 0) return bfail(SBLI_EINVAL, "ke_hist_dev is null");
  if (!(dt > 0) || !isfinite(dt)) return bfail(SBLI_EINVAL, "dt must be finite and > 0");
  for (int s = 0; s < nsteps; ++s) {
    SBLI_BTRY(enqueue_batch_stage(b, 0, b->state, dt, b->ke_items, b->stream), "batch stage");
    SBLI_BTRY(launch_batch_ke_finalize(b->ke_items, b->begin, b->inv_p, ke_hist_dev + (size_t)2 * b->count * s,
                                       b->count, b->stream),
              "ke finalize");
    for (int k = 1; k < 3; ++k) SBLI_BTRY(enqueue_batch_stage(b, k, b->state, dt, nullptr, b->stream), "batch stage");
    b->state = batch_next_state(b, b->state);
    b->steps_done++;
  }
  return SBLI_OK;
}

int sbli_batch_kinetic_energy(sbli_batch* b, double* ke, double* enstrophy) {
  if (int rc = check_batch(b, 0)) return rc;
  if (!ke || !enstrophy) return bfail(SBLI_EINVAL, "null output");
  for (int m = 0; m < b->count; ++m) {
    const MemberLayout& M = b->L.m[m];
    const double* q = reinterpret_cast<double*>(b->reg64[state_reg(b)] + M.off64);
    if (b->precision == SBLI_FP32_DF) {  // join into the register free at a step boundary
      double* tmp = reinterpret_cast<double*>(b->reg64[1 - b->state] + M.off64);
      SBLI_BTRY(launch_df_join(M.P, RefState{0.0, 0.0}, reinterpret_cast<const float*>(q), tmp, b->stream),
                "df_join");
      q = tmp;
    }
    SBLI_BTRY(launch_ke(member_geom(M), make_coef<double>(M.n, b->params[m]), make_ref(b->params[m]), q,
                        b->ke_scratch, b->ke_out + 2 * m, b->stream),
              "ke");
  }
  std::vector<double> h(2 * b->count);
  SBLI_BTRY(cudaMemcpyAsync(h.data(), b->ke_out, h.size() * sizeof(double), cudaMemcpyDeviceToHost, b->stream), "D2H");
  SBLI_BTRY(cudaStreamSynchronize(b->stream), "cudaStreamSynchronize");
  for (int m = 0; m < b->count; ++m) {
    ke[m] = h[2 * m];
    enstrophy[m] = h[2 * m + 1];
  }
  return SBLI_OK;
}

int sbli_batch_work_items(const sbli_batch* b, long long* items) {
  if (!b || !items) return bfail(SBLI_EINVAL, "null argument");
  *items = b->L.total_items;
  return SBLI_OK;
}

int sbli_batch_get_schedule(const sbli_batch* b, int* z_queue, int* planes_per_item) {
  if (!b || !z_queue) return bfail(SBLI_EINVAL, "null argument");
  *z_queue = b->zq;
  if (planes_per_item)
    for (int m = 0; m < b->count; ++m) planes_per_item[m] = b->L.m[m].zc;
  return SBLI_OK;
}

int sbli_batch_set_schedule(sbli_batch* b, int z_queue, const int* planes_per_item) {
  if (int rc = check_batch(b, 0)) return rc;
  if (z_queue < 0 || z_queue > 1) return bfail(SBLI_EINVAL, "z_queue %d not 0 or 1", z_queue);
  std::vector<int> zc(b->count);
  for (int m = 0; m < b->count; ++m) {
    zc[m] = planes_per_item ? planes_per_item[m] : b->L.m[m].zc;
    if (zc[m] < 4) return bfail(SBLI_EINVAL, "member %d: planes per item %d < 4", m, zc[m]);
    zc[m] = std::min(zc[m], b->L.m[m].n[2]);
  }
  SBLI_BTRY(apply_schedule(b, z_queue, zc), "schedule");
  return SBLI_OK;
}

int sbli_batch_autotune(sbli_batch* b, int reps, int* z_queue, float* best_stage_ms) {
  if (int rc = check_batch(b, 0)) return rc;
  if (reps < 1) return bfail(SBLI_EINVAL, "reps must be >= 1");
  cudaEvent_t e0, e1;
  SBLI_BTRY(cudaEventCreate(&e0), "cudaEventCreate");
  if (cudaError_t ce = cudaEventCreate(&e1)) {
    cudaEventDestroy(e0);
    return bcuda(ce, "cudaEventCreate");
  }
  // time one schedule: one untimed and `reps` timed stage-0 launches with
  // dt = 0, which write an accumulator equal to the state (acc + 0 * R; the
  // double-float members update theirs in place) and a stage field into a
  // free register
  cudaError_t err = cudaSuccess;
  auto time_schedule = [&](int zq, const std::vector<int>& zc) -> float {
    if (err == cudaSuccess) err = apply_schedule(b, zq, zc);
    if (err == cudaSuccess) err = enqueue_batch_stage(b, 0, b->state, 0.0, nullptr, b->stream);
    if (err == cudaSuccess) err = cudaEventRecord(e0, b->stream);
    for (int r = 0; r < reps && err == cudaSuccess; ++r) err = enqueue_batch_stage(b, 0, b->state, 0.0, nullptr, b->stream);
    if (err == cudaSuccess) err = cudaEventRecord(e1, b->stream);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float ms = 1e30f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    return err == cudaSuccess ? ms / (float)reps : 1e30f;
  };
  auto uniform = [&](int Z) {
    std::vector<int> zc(b->count);
    for (int m = 0; m < b->count; ++m) zc[m] = std::max(4, std::min(Z, b->L.m[m].n[2]));
    return zc;
  };
  const int Zs[6] = {8, 16, 32, 64, 128, 1 << 24};
  // 1. one z-queue mode and one planes-per-item value for every member
  int best_zq = b->zq;
  std::vector<int> best_zc(b->count);
  for (int m = 0; m < b->count; ++m) best_zc[m] = b->L.m[m].zc;
  const int start_zq = best_zq;
  const std::vector<int> start_zc = best_zc;  // restored if a trial launch fails
  float best = time_schedule(best_zq, best_zc);
  for (int zq = 0; zq <= 1; ++zq)
    for (int Z : Zs) {
      const std::vector<int> zc = uniform(Z);
      const float ms = time_schedule(zq, zc);
      if (ms < best) {
        best = ms;
        best_zq = zq;
        best_zc = zc;
      }
    }
  // 2. each size class (members with the same x2 extent) refined in turn
  std::vector<int> classes;
  for (int m = 0; m < b->count; ++m)
    if (std::find(classes.begin(), classes.end(), b->L.m[m].n[2]) == classes.end()) classes.push_back(b->L.m[m].n[2]);
  for (int n2 : classes) {
    for (int Z : Zs) {
      std::vector<int> zc = best_zc;
      for (int m = 0; m < b->count; ++m)
        if (b->L.m[m].n[2] == n2) zc[m] = std::max(4, std::min(Z, n2));
      if (zc == best_zc) continue;
      const float ms = time_schedule(best_zq, zc);
      if (ms < best) {
        best = ms;
        best_zc = zc;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) {
    apply_schedule(b, start_zq, start_zc);
    return bcuda(err, "autotune launch");
  }
  SBLI_BTRY(apply_schedule(b, best_zq, best_zc), "schedule");
  if (z_queue) *z_queue = best_zq;
  if (best_stage_ms) *best_stage_ms = best;
  return SBLI_OK;
}

}  // extern "C"
