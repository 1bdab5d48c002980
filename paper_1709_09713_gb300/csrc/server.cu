// server.cu -- continuous-batching request loop for Taylor-Green solves.
//
// Requests (grid size, physical parameters, precision, step count, dt) wait
// in a FIFO and are admitted when a slot and a block of the caller's device
// arena are free (first-fit allocation with coalescing of freed blocks).  An
// admitted request's state stays resident in its block for its whole life.
// The requests run in two independent lanes: the binary64-register
// precisions (binary64, double-float arithmetic) on one stream, the binary32
// ones (either accumulator) on another, so their work overlaps on the device
// and neither waits for the other.  A lane advances its requests in batches
// of K time steps (each stage of each precision one persistent multi-member
// launch, batch_kernel.cuh), K chosen so that a batch takes about
// LANE_BATCH_MS of device time (measured with events on the lane's stream)
// and no request of the batch overshoots its step count.  A tick looks at
// each lane: if its batch has completed, the lane's finished requests are
// retired (binary64 kinetic energy and enstrophy, optional copy of the final
// state to a caller buffer, release of their memory) and the next batch is
// launched; a lane still running is left alone.  Waiting requests are
// admitted at the start of every tick and join their lane's next batch.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <deque>
#include <map>
#include <thread>
#include <vector>

#include "batch_kernel.cuh"

using namespace sbli;

namespace {

int sfail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  return set_last_error(code, buf);
}

int scuda(cudaError_t e, const char* what) {
  return sfail(SBLI_ECUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

#define SBLI_STRY(expr, what)                        \
  do {                                               \
    cudaError_t e_ = (expr);                         \
    if (e_ != cudaSuccess) return scuda(e_, what);   \
  } while (0)

constexpr size_t SALIGN = 256;
size_t salign(size_t v) { return (v + SALIGN - 1) / SALIGN * SALIGN; }

// First-fit allocator over [0, cap) with coalescing of freed blocks.
class ArenaAllocator {
 public:
  explicit ArenaAllocator(size_t cap) : cap_(cap) { free_[0] = cap; }
  bool alloc(size_t bytes, size_t* off) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes;
        const size_t noff = it->first + bytes;
        free_.erase(it);
        if (rest) free_[noff] = rest;
        used_ += bytes;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto next = std::next(it);
    if (next != free_.end() && it->first + it->second == next->first) {
      it->second += next->second;
      free_.erase(next);
    }
    if (it != free_.begin()) {
      auto prev = std::prev(it);
      if (prev->first + prev->second == it->first) {
        prev->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t free_bytes() const { return cap_ - used_; }
  size_t largest_free() const {
    size_t m = 0;
    for (auto& kv : free_) m = std::max(m, kv.second);
    return m;
  }

 private:
  size_t cap_, used_ = 0;
  std::map<size_t, size_t> free_;  // offset -> length
};

struct Req {
  long long id;
  sbli_request r;
  double t_submit = 0, t_admit = 0, t_done = 0;
  int state = 0;
  int remaining = 0;
  size_t off = 0, bytes = 0;
  long long P = 0;
  size_t reg64 = 0, reg32 = 0;  // register sizes inside the block
  double ke = 0, ens = 0;
};

// binary64 registers with the three-register rotation (binary64 and
// double-float arithmetic)
bool req_f64_registers(int precision) { return precision == SBLI_FP64 || precision == SBLI_DF64; }

size_t request_bytes(const sbli_request& r, size_t* reg64, size_t* reg32) {
  const long long P = (long long)r.n0 * r.n1 * r.n2;
  *reg64 = salign((size_t)P * 5 * sizeof(double));
  *reg32 = salign((size_t)P * 5 * sizeof(float));
  return req_f64_registers(r.precision) ? 3 * *reg64 : 2 * *reg64 + 2 * *reg32;
}

}  // namespace

// Device time one lane batch aims at: long enough to amortise the host's
// launch work over several steps, short enough that a request arriving
// meanwhile waits only a few milliseconds to join.
constexpr double LANE_BATCH_MS = 4.0;
constexpr int LANE_MAX_STEPS = 256;

struct Lane {
  cudaStream_t st = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;  // start and end of the batch in flight
  bool busy = false;
  int steps = 0;            // time steps of the batch in flight
  double ms_per_step = 0;   // running estimate (0: none yet)
};

struct sbli_server {
  char* arena;
  size_t arena_bytes;
  ArenaAllocator* alloc;
  int max_slots;
  int backfill;
  cudaStream_t s64, s32;
  double* ke_dev;      // 2 doubles for retirement reductions
  double* ke_scratch;  // partials of the KE kernel
  std::deque<Req> pending;
  std::vector<Req> active;
  std::deque<Req> done;
  long long next_id = 0;
  long long ticks = 0;
  int grid64, grid32;
  Lane lane[2];  // 0: binary64-register precisions on s64; 1: binary32 precisions on s32
  std::chrono::steady_clock::time_point t0;
  double now() const { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); }
};

namespace {

double* r64(const sbli_server* s, const Req& q, int r) {
  return reinterpret_cast<double*>(s->arena + q.off + (size_t)r * q.reg64);
}
float* r32(const sbli_server* s, const Req& q, int r) {
  return reinterpret_cast<float*>(s->arena + q.off + 2 * q.reg64 + (size_t)r * q.reg32);
}

StageArgs req_stage(const sbli_server* s, const Req& q, int k, bool* in64) {
  StageArgs a{};
  a.g = Geom{q.r.n0, q.r.n1, q.r.n2, q.P};
  a.zc = batch_zc(q.r.n2);
  a.a_dt = RK_A[k] * q.r.dt;
  a.b_dt = RK_B[k] * q.r.dt;
  a.amb_dt = (RK_A[k] - RK_B[k]) * q.r.dt;
  a.b_dt32 = (float)a.b_dt;
  a.amb_dt32 = (float)a.amb_dt;
  a.df_normalize = (k == 2);
  const int st = q.state;
  if (q.r.precision == SBLI_DF64) {
    // accumulator in place in register 0; stage fields of (hi, lo) pairs
    // alternate between registers st (the pair copy of Q^n) and 3 - st
    double* S = r64(s, q, 0);
    double* Pa = r64(s, q, st);
    double* Pb = r64(s, q, 3 - st);
    *in64 = false;
    a.acc_in = S;
    a.acc_out = S;
    if (k == 0) { a.q_in = Pa; a.q_out = Pb; }
    else if (k == 1) { a.q_in = Pb; a.q_out = Pa; }
    else { a.q_in = Pa; a.q_out = Pb; }  // a_3 = b_3: the pair copy of Q^{n+1}
  } else if (req_f64_registers(q.r.precision)) {
    double* S = r64(s, q, st);
    double* A = r64(s, q, (st + 1) % 3);
    double* B = r64(s, q, (st + 2) % 3);
    *in64 = true;
    if (k == 0) { a.q_in = S; a.acc_in = S; a.acc_out = A; a.q_out = B; }
    else if (k == 1) { a.q_in = B; a.acc_in = A; a.acc_out = A; a.q_out = S; }
    else { a.q_in = S; a.acc_in = A; a.acc_out = A; a.q_out = nullptr; }
  } else if (q.r.precision == SBLI_FP32_DF) {
    // state and accumulator as double-float pairs (hi fields, then lo fields)
    float* S = reinterpret_cast<float*>(r64(s, q, st));
    float* A = reinterpret_cast<float*>(r64(s, q, 1 - st));
    *in64 = false;
    if (k == 0) { a.q_in = S; a.dacc_in = S; a.dacc_out = A; a.q_out = r32(s, q, 0); }
    else if (k == 1) { a.q_in = r32(s, q, 0); a.dacc_in = A; a.dacc_out = A; a.q_out = r32(s, q, 1); }
    else { a.q_in = r32(s, q, 1); a.dacc_in = A; a.dacc_out = A; a.q_out = nullptr; }
  } else {
    // binary64 state and accumulator; binary32 register `st` holds the binary32
    // copy of the state (as for single grids)
    double* S = r64(s, q, st);
    double* A = r64(s, q, 1 - st);
    float* Cs = r32(s, q, st);
    float* Ds = r32(s, q, 1 - st);
    *in64 = false;
    if (k == 0) { a.q_in = Cs; a.acc_in = S; a.acc_out = A; a.q_out = Ds; }
    else if (k == 1) { a.q_in = Ds; a.acc_in = A; a.acc_out = A; a.q_out = Cs; }
    else { a.q_in = Cs; a.acc_in = A; a.acc_out = A; a.q_out = Ds; }
  }
  return a;
}

// Stage k of the requests of `run` that have the given precision, in
// launches of at most BATCH_MAX_MEMBERS members.
template <typename T>
cudaError_t launch_group(sbli_server* s, int k, int precision, const std::vector<Req*>& run, cudaStream_t st,
                         int grid) {
  std::vector<const Req*> mem;
  for (const Req* q : run)
    if (q->r.precision == precision) mem.push_back(q);
  for (size_t base = 0; base < mem.size(); base += BATCH_MAX_MEMBERS) {
    const int cnt = (int)std::min<size_t>(BATCH_MAX_MEMBERS, mem.size() - base);
    BatchParams<T> p;
    memset(&p, 0, sizeof p);
    p.count = cnt;
    long long acc = 0;
    bool in64 = true;
    for (int m = 0; m < cnt; ++m) {
      const Req& q = *mem[base + m];
      const int n[3] = {q.r.n0, q.r.n1, q.r.n2};
      p.item_begin[m] = acc;
      p.tiles_x[m] = (n[0] + 31) / 32;
      p.tiles_y[m] = (n[1] + 7) / 8;
      acc += member_items(n);
      p.a[m] = req_stage(s, q, k, &in64);
      p.c[m] = make_coef<T>(n, q.r.params);
    }
    p.item_begin[cnt] = acc;
    p.total_items = acc;
    cudaError_t e = launch_batch_t<T>(p, in64, grid, st, precision == SBLI_FP32_DF, batch_default_zq(precision));
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int valid_request(const sbli_request* r) {
  if (!r) return sfail(SBLI_EINVAL, "request is null");
  if (r->n0 < 5 || r->n1 < 5 || r->n2 < 5 || (long long)r->n0 * r->n1 >= (1LL << 31) ||
      (long long)r->n0 * r->n1 * r->n2 >= (1LL << 32))
    return sfail(SBLI_EINVAL, "request grid %d x %d x %d invalid", r->n0, r->n1, r->n2);
  if (r->precision < SBLI_FP64 || r->precision > SBLI_DF64) return sfail(SBLI_EINVAL, "unknown precision %d", r->precision);
  if (r->steps < 0) return sfail(SBLI_EINVAL, "steps < 0");
  if (!(r->dt > 0) || !isfinite(r->dt)) return sfail(SBLI_EINVAL, "dt must be finite and > 0");
  const sbli_params& p = r->params;
  if (!(p.Re > 0) || !(p.Mach > 0) || !(p.Pr > 0) || !(p.gamma > 1) || !(p.L > 0) || isnan(p.Re) ||
      !isfinite(p.Mach) || !isfinite(p.Pr) || !isfinite(p.gamma) || !isfinite(p.L) || !isfinite(r->amplitude))
    return sfail(SBLI_EINVAL, "request physical parameters invalid");
  return SBLI_OK;
}

int lane_of(int precision) { return req_f64_registers(precision) ? 0 : 1; }

// Register rotation of a request (as for single grids): double-float requests
// keep the binary64 state in register 0 and the pair copy of the state in
// register `state` (1 or 2); the others keep the state in register `state`.
int req_initial_state(int precision) { return precision == SBLI_DF64 ? 1 : 0; }
int req_next_state(int precision, int st) {
  if (precision == SBLI_DF64) return 3 - st;
  return req_f64_registers(precision) ? (st + 1) % 3 : 1 - st;
}
int req_state_reg(const Req& q) { return q.r.precision == SBLI_DF64 ? 0 : q.state; }
int req_free_reg(const Req& q) { return q.r.precision == SBLI_DF64 ? 3 - q.state : (q.state + 1) % 2; }

// Taylor-Green initial field of a newly admitted request in its registers,
// on its lane's stream.
int init_request(sbli_server* s, const Req& q) {
  cudaStream_t st = s->lane[lane_of(q.r.precision)].st;
  const Geom qg{q.r.n0, q.r.n1, q.r.n2, q.P};
  if (q.r.precision == SBLI_FP32_DF) {  // binary64 deviation field, then split into hi/lo
    SBLI_STRY(launch_init_tgv(qg, q.r.params, q.r.amplitude, r64(s, q, 1), st), "init_tgv");
    SBLI_STRY(launch_df_split(q.P, RefState{0.0, 0.0}, r64(s, q, 1), reinterpret_cast<float*>(r64(s, q, 0)), st),
              "df_split");
  } else {
    SBLI_STRY(launch_init_tgv(qg, q.r.params, q.r.amplitude, r64(s, q, 0), st), "init_tgv");
    if (q.r.precision == SBLI_FP32) SBLI_STRY(launch_narrow(5 * q.P, r64(s, q, 0), r32(s, q, 0), st), "narrow");
    if (q.r.precision == SBLI_DF64)
      SBLI_STRY(launch_pair_split(5 * q.P, r64(s, q, 0), reinterpret_cast<float*>(r64(s, q, q.state)), st),
                "pair_split");
  }
  return SBLI_OK;
}

// Final diagnostics and copy-out of a finished request; frees its block.
int retire(sbli_server* s, Req& q) {
  cudaStream_t st = s->lane[lane_of(q.r.precision)].st;
  const Geom g{q.r.n0, q.r.n1, q.r.n2, q.P};
  const int n[3] = {q.r.n0, q.r.n1, q.r.n2};
  const double* state = r64(s, q, req_state_reg(q));
  if (q.r.precision == SBLI_FP32_DF) {
    // join the double-float state (deviation form) into the other register
    double* joined = r64(s, q, 1 - q.state);
    SBLI_STRY(launch_df_join(q.P, RefState{0.0, 0.0}, reinterpret_cast<const float*>(state), joined, st), "df_join");
    state = joined;
  }
  SBLI_STRY(launch_ke(g, make_coef<double>(n, q.r.params), make_ref(q.r.params), state, s->ke_scratch, s->ke_dev, st),
            "ke");
  double h[2];
  SBLI_STRY(cudaMemcpyAsync(h, s->ke_dev, sizeof h, cudaMemcpyDeviceToHost, st), "D2H");
  if (q.r.result) {
    double* tmp = r64(s, q, req_free_reg(q));  // a register the finished state does not occupy
    if (q.r.precision == SBLI_FP32_DF) {
      SBLI_STRY(launch_df_join(q.P, make_ref(q.r.params), reinterpret_cast<const float*>(r64(s, q, q.state)), tmp, st),
                "df_join");
    } else {
      SBLI_STRY(launch_from_offset(g, make_ref(q.r.params), state, tmp, st), "from_offset");
    }
    SBLI_STRY(cudaMemcpyAsync(q.r.result, tmp, 5 * (size_t)q.P * sizeof(double),
                              q.r.result_is_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st),
              "copy result");
  }
  SBLI_STRY(cudaStreamSynchronize(st), "cudaStreamSynchronize");
  q.ke = h[0];
  q.ens = h[1];
  q.t_done = s->now();
  s->alloc->release(q.off, q.bytes);
  return SBLI_OK;
}

}  // namespace

extern "C" {

int sbli_server_create(sbli_server** out, void* arena, size_t arena_bytes, int max_slots, int backfill,
                       void* stream_fp64, void* stream_fp32) {
  if (!out) return sfail(SBLI_EINVAL, "out is null");
  *out = nullptr;
  if (!arena || ((uintptr_t)arena) % SALIGN) return sfail(SBLI_EINVAL, "arena must be 256-byte aligned device memory");
  const size_t reserve = salign(2 * sizeof(double)) + salign(2 * 1024 * sizeof(double));
  if (arena_bytes <= reserve) return sfail(SBLI_ENOMEM, "arena of %zu bytes is too small", arena_bytes);
  if (max_slots < 1) return sfail(SBLI_EINVAL, "max_slots must be >= 1");
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, arena) != cudaSuccess || attr.type != cudaMemoryTypeDevice) {
    cudaGetLastError();
    return sfail(SBLI_EINVAL, "arena is not device memory");
  }
  sbli_server* s = new sbli_server();
  s->ke_dev = reinterpret_cast<double*>(arena);
  s->ke_scratch = reinterpret_cast<double*>(static_cast<char*>(arena) + salign(2 * sizeof(double)));
  s->arena = static_cast<char*>(arena) + reserve;
  s->arena_bytes = (arena_bytes - reserve) / SALIGN * SALIGN;
  s->alloc = new ArenaAllocator(s->arena_bytes);
  s->max_slots = max_slots;
  s->backfill = backfill;
  s->s64 = static_cast<cudaStream_t>(stream_fp64);
  s->s32 = static_cast<cudaStream_t>(stream_fp32);
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  s->grid64 = sms * batch_ctas_per_sm(SBLI_FP64, batch_default_zq(SBLI_FP64));
  s->grid32 = sms * batch_ctas_per_sm(SBLI_FP32, batch_default_zq(SBLI_FP32));
  s->lane[0].st = s->s64;
  s->lane[1].st = s->s32;
  for (Lane& l : s->lane) {
    if (cudaEventCreate(&l.ev0) != cudaSuccess || cudaEventCreate(&l.ev1) != cudaSuccess) {
      cudaGetLastError();
      for (Lane& m : s->lane) {
        if (m.ev0) cudaEventDestroy(m.ev0);
        if (m.ev1) cudaEventDestroy(m.ev1);
      }
      delete s->alloc;
      delete s;
      return sfail(SBLI_ECUDA, "cudaEventCreate failed");
    }
  }
  s->t0 = std::chrono::steady_clock::now();
  *out = s;
  return SBLI_OK;
}

int sbli_server_destroy(sbli_server* s) {
  if (!s) return SBLI_OK;
  cudaStreamSynchronize(s->s64);
  cudaStreamSynchronize(s->s32);
  for (Lane& l : s->lane) {
    cudaEventDestroy(l.ev0);
    cudaEventDestroy(l.ev1);
  }
  delete s->alloc;
  delete s;
  return SBLI_OK;
}

int sbli_server_request_bytes(const sbli_request* r, size_t* bytes) {
  if (int rc = valid_request(r)) return rc;
  if (!bytes) return sfail(SBLI_EINVAL, "bytes is null");
  size_t a, b;
  *bytes = request_bytes(*r, &a, &b);
  return SBLI_OK;
}

int sbli_server_submit(sbli_server* s, const sbli_request* r, long long* id) {
  if (!s) return sfail(SBLI_EINVAL, "null server");
  if (int rc = valid_request(r)) return rc;
  Req q;
  q.id = s->next_id++;
  q.r = *r;
  q.t_submit = s->now();
  q.P = (long long)r->n0 * r->n1 * r->n2;
  q.bytes = request_bytes(*r, &q.reg64, &q.reg32);
  if (q.bytes > s->arena_bytes) return sfail(SBLI_ENOMEM, "request needs %zu bytes, arena has %zu", q.bytes, s->arena_bytes);
  s->pending.push_back(q);
  if (id) *id = q.id;
  return SBLI_OK;
}

int sbli_server_tick(sbli_server* s, int* completed) {
  if (!s) return sfail(SBLI_EINVAL, "null server");
  // admit in arrival order while a slot and memory are free; with backfill,
  // later requests that fit may pass a head request that does not
  for (auto it = s->pending.begin(); it != s->pending.end() && (int)s->active.size() < s->max_slots;) {
    size_t off = 0;
    if (!s->alloc->alloc(it->bytes, &off)) {
      if (!s->backfill) break;
      ++it;
      continue;
    }
    Req q = *it;
    it = s->pending.erase(it);
    q.off = off;
    q.t_admit = s->now();
    q.state = req_initial_state(q.r.precision);
    q.remaining = q.r.steps;
    if (int rc = init_request(s, q)) {  // back to the head of the queue, its block free again
      s->alloc->release(q.off, q.bytes);
      s->pending.push_front(q);
      return rc;
    }
    s->active.push_back(q);
  }
  int n = 0;
  // a tick that finds both lanes busy waits (bounded) for the first to finish
  const auto wait_start = std::chrono::steady_clock::now();
  for (;;) {
    bool progressed = false;
    for (int li = 0; li < 2; ++li) {
      Lane& L = s->lane[li];
      if (L.busy) {
        const cudaError_t q = cudaEventQuery(L.ev1);
        if (q == cudaErrorNotReady) continue;
        SBLI_STRY(q, "cudaEventQuery");
        float ms = 0.f;
        SBLI_STRY(cudaEventElapsedTime(&ms, L.ev0, L.ev1), "cudaEventElapsedTime");
        const double per = (double)ms / L.steps;
        L.ms_per_step = L.ms_per_step > 0 ? 0.5 * (L.ms_per_step + per) : per;
        L.busy = false;
        progressed = true;
      }
      // retire this lane's finished requests (its stream holds no step work now)
      for (auto it = s->active.begin(); it != s->active.end();) {
        if (lane_of(it->r.precision) == li && it->remaining == 0) {
          if (int rc = retire(s, *it)) return rc;
          s->done.push_back(*it);
          it = s->active.erase(it);
          ++n;
          progressed = true;
        } else {
          ++it;
        }
      }
      // next batch: every request of the lane with steps left, K steps
      std::vector<Req*> run;
      int kmin = LANE_MAX_STEPS;
      bool has[4] = {false, false, false, false};
      for (Req& q : s->active) {
        if (lane_of(q.r.precision) != li || q.remaining == 0) continue;
        run.push_back(&q);
        kmin = std::min(kmin, q.remaining);
        has[q.r.precision] = true;
      }
      if (run.empty()) continue;
      int K = 1;
      if (L.ms_per_step > 0) K = (int)std::max(1.0, std::floor(LANE_BATCH_MS / L.ms_per_step));
      K = std::min(K, kmin);
      SBLI_STRY(cudaEventRecord(L.ev0, L.st), "cudaEventRecord");
      for (int step = 0; step < K; ++step) {
        for (int k = 0; k < 3; ++k) {
          if (has[SBLI_FP64]) SBLI_STRY(launch_group<double>(s, k, SBLI_FP64, run, L.st, s->grid64), "fp64 stage");
          if (has[SBLI_DF64])
            SBLI_STRY(launch_group<dfloat>(s, k, SBLI_DF64, run, L.st, s->grid64), "double-float stage");
          if (has[SBLI_FP32]) SBLI_STRY(launch_group<float>(s, k, SBLI_FP32, run, L.st, s->grid32), "fp32 stage");
          if (has[SBLI_FP32_DF])
            SBLI_STRY(launch_group<float>(s, k, SBLI_FP32_DF, run, L.st, s->grid32), "fp32 double-float stage");
        }
        for (Req* q : run) q->state = req_next_state(q->r.precision, q->state);
      }
      SBLI_STRY(cudaEventRecord(L.ev1, L.st), "cudaEventRecord");
      for (Req* q : run) q->remaining -= K;
      L.busy = true;
      L.steps = K;
      progressed = true;
    }
    if (progressed || (!s->lane[0].busy && !s->lane[1].busy)) break;
    // nothing to do until a lane finishes: poll its event, at most ~2 ms
    const double waited = std::chrono::duration<double>(std::chrono::steady_clock::now() - wait_start).count();
    if (waited > 0.002) break;
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
  s->ticks++;
  if (completed) *completed = n;
  return SBLI_OK;
}

int sbli_server_poll(sbli_server* s, sbli_result* out, int max, int* n) {
  if (!s || !n || (max > 0 && !out)) return sfail(SBLI_EINVAL, "null argument");
  int k = 0;
  while (k < max && !s->done.empty()) {
    const Req& q = s->done.front();
    sbli_result& r = out[k++];
    r.id = q.id;
    r.ke = q.ke;
    r.enstrophy = q.ens;
    r.t_submit = q.t_submit;
    r.t_admit = q.t_admit;
    r.t_done = q.t_done;
    r.steps = q.r.steps;
    r.points = q.P;
    r.precision = q.r.precision;
    s->done.pop_front();
  }
  *n = k;
  return SBLI_OK;
}

int sbli_server_stats(const sbli_server* s, sbli_server_status* st) {
  if (!s || !st) return sfail(SBLI_EINVAL, "null argument");
  st->pending = (int)s->pending.size();
  st->active = (int)s->active.size();
  st->completed_unpolled = (int)s->done.size();
  st->free_bytes = s->alloc->free_bytes();
  st->largest_free_block = s->alloc->largest_free();
  st->arena_bytes = s->arena_bytes;
  st->ticks = s->ticks;
  st->now = s->now();
  return SBLI_OK;
}

}  // extern "C"
