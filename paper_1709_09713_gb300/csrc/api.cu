// api.cu -- the C ABI of include/sbli.h: grid handles over caller-owned
// device memory, stage sequencing of the low-storage scheme (§2.2, Fig. 1),
// CUDA-graph step loops and the binary64 diagnostics.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>

#include "sbli_internal.cuh"

using namespace sbli;

namespace {

thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(SBLI_ECUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

#define SBLI_TRY(expr, what)                       \
  do {                                             \
    cudaError_t e_ = (expr);                       \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

constexpr size_t ALIGN = 256;
size_t align_up(size_t v) { return (v + ALIGN - 1) / ALIGN * ALIGN; }

struct Layout {
  size_t reg64;      // bytes of one binary64 state register (5P doubles)
  size_t reg32;      // bytes of one binary32 stage register (5P floats)
  int n64, n32;      // registers of each kind
  size_t partials;   // bytes of the reduction scratch
  size_t storeall;   // bytes of the store-all scratch
  size_t total;
};

bool valid_sizes(int n0, int n1, int n2) {
  if (n0 < 5 || n1 < 5 || n2 < 5) return false;
  // in-plane offsets are 32-bit in the kernels; grid index fits 2^31 planes
  if ((long long)n0 * n1 >= (1LL << 31)) return false;
  // the fused kernels address a point within one field with a 32-bit unsigned offset
  if ((long long)n0 * n1 * n2 >= (1LL << 32)) return false;
  if (n0 > (1 << 24) || n1 > (1 << 24) || n2 > (1 << 24)) return false;
  return true;
}

FusedConfig default_config(const Geom& g, int precision);

// binary64 state, accumulator and stage registers (three-register rotation)
bool f64_registers(int precision) { return precision == SBLI_FP64 || precision == SBLI_DF64; }

Layout layout_for(int n0, int n1, int n2, int precision, int variant) {
  Geom g{n0, n1, n2, (long long)n0 * n1 * n2};
  Layout L{};
  L.reg64 = align_up((size_t)g.P * 5 * sizeof(double));
  L.reg32 = align_up((size_t)g.P * 5 * sizeof(float));
  L.n64 = f64_registers(precision) ? 3 : 2;
  L.n32 = f64_registers(precision) ? 0 : 2;
  // partial sums: the fused kernel's CTAs for any configuration the grid may
  // use (the smallest zc gives the most CTAs), or the KE kernel's blocks
  const long long tiles = (long long)((n0 + 31) / 32) * ((n1 + 3) / 4);
  const long long max_ctas = tiles * ((n2 + 3) / 4);
  const long long np = std::max<long long>(max_ctas, ke_num_partials(g));
  L.partials = align_up((size_t)(2 * np + 2) * sizeof(double));
  L.storeall = variant == SBLI_STORE_ALL
                   ? align_up(storeall_scratch_doubles(g, precision == SBLI_FP64 ? 8 : 4) * sizeof(double))
                   : align_up(algorithm_scratch_doubles(g, variant) * sizeof(double));
  L.total = L.reg64 * L.n64 + L.reg32 * L.n32 + L.partials + L.storeall;
  return L;
}

}  // namespace

int sbli::set_last_error(int code, const char* msg) {
  g_last_error = msg;
  return code;
}

struct sbli_grid {
  int n[3];
  int precision, variant;
  sbli_params params;
  Geom geom;
  cudaStream_t stream;      // caller's stream (work and graph launches)
  cudaStream_t cap_stream;  // private stream used only to record graphs
  Layout layout;
  double* reg64[3];
  float* reg32[2];
  double* partials;  // reduction scratch; last two doubles hold a (ke, ens) result
  double* ke_out;
  void* storeall;
  int state;       // index of the binary64 register holding Q^n (deviation form)
  int next_stage;  // 0, 1, 2
  long long stages_done;
  FusedConfig cfg;
  Coef<double> cd;
  Coef<float> cf;
  Coef<dfloat> cw;
  RefState ref;
  // graph of GRAPH_STEPS steps per starting register rotation
  static constexpr int GRAPH_STEPS = 6;
  cudaGraphExec_t graph[3];
  double graph_dt[3];
};

namespace {

// Where a grid keeps its binary64 state between steps.  Double-float grids
// (SBLI_DF64) keep the state and accumulator in reg64[0], updated in place
// by every stage, and the (hi, lo) pair copy of the state in reg64[state]
// (1 or 2): the stages read only pair fields as stencil input, so the
// accumulator is read pointwise and may be overwritten in place.  Every other
// precision keeps the state in reg64[state].
double* state64(const sbli_grid* g) { return g->precision == SBLI_DF64 ? g->reg64[0] : g->reg64[g->state]; }
int initial_state(int precision) { return precision == SBLI_DF64 ? 1 : 0; }
// a binary64 register that holds nothing live at a step boundary
double* free64(const sbli_grid* g) {
  if (g->precision == SBLI_DF64) return g->reg64[3 - g->state];
  return g->reg64[(g->state + 1) % g->layout.n64];
}

// CTAs per SM a tile height allows (shared memory bound).
int ctas_per_sm(int precision, int ty, int px = 1, int zq = 0) {
  if (f64_registers(precision) || ty >= 16 || px == 2) return 1;
  return zq ? 3 : 2;  // the TMEM z queue keeps 3 full-record planes in shared memory
}

// Planes per CTA ranked by a wave-balance model: cost = waves * (zc + 1.5),
// the 4 warm-up planes of a z segment costing about 1.5 full planes.
void rank_zc(const Geom& g, int precision, int ty, int* best, int nbest, int px = 1, int zq = 0) {
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long slots = (long long)sms * ctas_per_sm(precision, ty, px, zq);
  const int w = 32 * px;
  const long long tiles = (long long)((g.n0 + w - 1) / w) * ((g.n1 + ty - 1) / ty);
  double cost[8];
  for (int i = 0; i < nbest; ++i) {
    best[i] = 0;
    cost[i] = 1e300;
  }
  for (int zc = 4; zc <= g.n2; ++zc) {
    const long long gz = (g.n2 + zc - 1) / zc;
    if (zc > 4 && (gz - 1) * zc >= g.n2) continue;  // same CTA count as a smaller zc
    const long long waves = (tiles * gz + slots - 1) / slots;
    const double c = (double)waves * (zc + 1.5);
    for (int i = 0; i < nbest; ++i) {
      if (c < cost[i] - 1e-9) {
        for (int j = nbest - 1; j > i; --j) {
          cost[j] = cost[j - 1];
          best[j] = best[j - 1];
        }
        cost[i] = c;
        best[i] = zc;
        break;
      }
    }
  }
  for (int i = 0; i < nbest; ++i)
    if (best[i] == 0) best[i] = best[0] ? best[0] : std::min(4, g.n2);
}

FusedConfig default_config(const Geom& g, int precision) {
  FusedConfig cfg;
  cfg.ty = 8;
  cfg.zq = 0;
  cfg.px = 1;
  int zc[1];
  rank_zc(g, precision, cfg.ty, zc, 1);
  cfg.zc = std::max(4, std::min(zc[0], g.n2));
  return cfg;
}

bool valid_config(int precision, int ty, int zc, int zq = 0, int px = 1) {
  if (zc < 4 || zq < 0 || zq > 1 || px < 1 || px > 2) return false;
  if (f64_registers(precision)) return ty == 8 && px == 1;  // shared-memory ring or TMEM queue
  if (px == 2) return ty == 8 && zq == 0;  // 64 x 8 two-column tiles, shared-memory ring
  return ty == 8 || ty == 16;  // binary32 stage fields (either accumulator)
}

// Pointers of stage k for the current rotation.
struct StagePtrs {
  const void* q_in;
  bool in64;
  const double* acc_in;
  double* acc_out;
  void* q_out;
  bool out64;
  const float* dacc_in;  // double-float accumulator (SBLI_FP32_DF)
  float* dacc_out;
};

StagePtrs stage_ptrs(const sbli_grid* g, int k, int state) {
  StagePtrs p{};
  if (g->precision == SBLI_DF64) {
    // double-float arithmetic: accumulator S updated in place; the stage
    // fields alternate between the two pair registers, Pa holding the pair
    // copy of Q^n at the step boundary (written by the previous stage 2)
    double* S = g->reg64[0];
    double* Pa = g->reg64[state];
    double* Pb = g->reg64[3 - state];
    p.in64 = p.out64 = false;
    p.acc_in = S;
    p.acc_out = S;
    if (k == 0) {
      p.q_in = Pa; p.q_out = Pb;
    } else if (k == 1) {
      p.q_in = Pb; p.q_out = Pa;
    } else {
      p.q_in = Pa; p.q_out = Pb;  // a_3 = b_3: the pair copy of Q^{n+1}
    }
  } else if (f64_registers(g->precision)) {
    double* S = g->reg64[state];
    double* A = g->reg64[(state + 1) % 3];
    double* B = g->reg64[(state + 2) % 3];
    p.in64 = p.out64 = true;
    if (k == 0) {
      p.q_in = S; p.acc_in = S; p.acc_out = A; p.q_out = B;
    } else if (k == 1) {
      p.q_in = B; p.acc_in = A; p.acc_out = A; p.q_out = S;
    } else {
      p.q_in = S; p.acc_in = A; p.acc_out = A; p.q_out = nullptr;
    }
  } else if (g->precision == SBLI_FP32_DF) {
    // double-float registers: the hi fields are the binary32 stage input
    float* S = reinterpret_cast<float*>(g->reg64[state]);
    float* A = reinterpret_cast<float*>(g->reg64[1 - state]);
    p.out64 = false;
    p.in64 = false;
    if (k == 0) {
      p.q_in = S; p.dacc_in = S; p.dacc_out = A; p.q_out = g->reg32[0];
    } else if (k == 1) {
      p.q_in = g->reg32[0]; p.dacc_in = A; p.dacc_out = A; p.q_out = g->reg32[1];
    } else {
      p.q_in = g->reg32[1]; p.dacc_in = A; p.dacc_out = A; p.q_out = nullptr;
    }
  } else {
    // binary64 state S and accumulator A; the binary32 register `state` holds
    // the binary32 copy of S (written by the previous step's last stage, whose
    // stage output a_3 = b_3 makes exactly the narrowed new state, or by the
    // calls that set the state), so every stage reads binary32 fields
    double* S = g->reg64[state];
    double* A = g->reg64[1 - state];
    float* C = g->reg32[state];
    float* D = g->reg32[1 - state];
    p.out64 = false;
    p.in64 = false;
    if (k == 0) {
      p.q_in = C; p.acc_in = S; p.acc_out = A; p.q_out = D;
    } else if (k == 1) {
      p.q_in = D; p.acc_in = A; p.acc_out = A; p.q_out = C;
    } else {
      p.q_in = C; p.acc_in = A; p.acc_out = A; p.q_out = D;  // D: the next state's binary32 copy
    }
  }
  return p;
}

int next_state(const sbli_grid* g, int state) {
  if (g->precision == SBLI_DF64) return 3 - state;
  return f64_registers(g->precision) ? (state + 1) % 3 : 1 - state;
}

// Enqueue stage k on stream s for the given rotation; ke_partials != nullptr
// (stage 0 only) also accumulates the diagnostics of the stage input.
cudaError_t enqueue_stage(sbli_grid* g, int k, int state, double dt, double* ke_partials, cudaStream_t s) {
  const StagePtrs p = stage_ptrs(g, k, state);
  const double a_dt = RK_A[k] * dt, b_dt = RK_B[k] * dt;
  if (g->variant == SBLI_FUSED) {
    StageArgs a{};
    a.g = g->geom;
    a.zc = g->cfg.zc;
    a.q_in = p.q_in;
    a.acc_in = p.acc_in;
    a.acc_out = p.acc_out;
    a.q_out = p.q_out;
    a.a_dt = a_dt;
    a.b_dt = b_dt;
    a.amb_dt = (RK_A[k] - RK_B[k]) * dt;
    a.b_dt32 = (float)a.b_dt;
    a.amb_dt32 = (float)a.amb_dt;
    a.ke_partials = ke_partials;
    a.dacc_in = p.dacc_in;
    a.dacc_out = p.dacc_out;
    a.df_normalize = (k == 2);
    if (g->precision == SBLI_FP64) return launch_fused_fp64(a, g->cd, g->cfg, false, s);
    if (g->precision == SBLI_DF64) return launch_fused_df64(a, g->cw, g->cfg, false, !p.in64, s);
    if (g->precision == SBLI_FP32_DF) return launch_fused_fp32df(a, g->cf, g->cfg, false, s);
    return launch_fused_fp32(a, g->cf, g->cfg, p.in64, false, s);
  }
  if (g->variant > SBLI_STORE_ALL)
    return launch_algorithm_stage(g->variant, g->geom, g->cd, static_cast<const double*>(p.q_in), p.acc_in,
                                  p.acc_out, static_cast<double*>(p.q_out), nullptr, a_dt, b_dt,
                                  static_cast<double*>(g->storeall), s);
  // store-all: residual into scratch, then the update kernel
  cudaError_t e;
  if (g->precision == SBLI_FP64) {
    double* scr = static_cast<double*>(g->storeall);
    e = launch_storeall_rhs_fp64(g->geom, g->cd, static_cast<const double*>(p.q_in), scr, nullptr, s);
    if (e != cudaSuccess) return e;
    const double* r = scr + storeall_r_offset(g->geom);
    return launch_rk_update(g->geom, r, true, p.acc_in, p.acc_out, p.q_out, true, a_dt, b_dt, s);
  }
  float* scr = static_cast<float*>(g->storeall);
  e = launch_storeall_rhs_fp32(g->geom, g->cf, p.q_in, p.in64, scr, nullptr, s);
  if (e != cudaSuccess) return e;
  const float* r = scr + storeall_r_offset(g->geom);
  return launch_rk_update(g->geom, r, false, p.acc_in, p.acc_out, p.q_out, false, a_dt, b_dt, s);
}

int check_grid(const sbli_grid* g) {
  if (!g) return fail(SBLI_EINVAL, "null grid handle");
  return SBLI_OK;
}

void drop_graphs(sbli_grid* g) {
  for (int r = 0; r < 3; ++r) {
    if (g->graph[r]) cudaGraphExecDestroy(g->graph[r]);
    g->graph[r] = nullptr;
    g->graph_dt[r] = 0.0;
  }
}

// Record GRAPH_STEPS steps starting from rotation `state` into an executable graph.
int build_graph(sbli_grid* g, int state, double dt) {
  if (g->graph[state] && g->graph_dt[state] == dt) return SBLI_OK;
  if (g->graph[state]) {
    cudaGraphExecDestroy(g->graph[state]);
    g->graph[state] = nullptr;
  }
  SBLI_TRY(cudaStreamBeginCapture(g->cap_stream, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
  int st = state;
  cudaError_t err = cudaSuccess;
  for (int s = 0; s < sbli_grid::GRAPH_STEPS && err == cudaSuccess; ++s) {
    for (int k = 0; k < 3 && err == cudaSuccess; ++k) err = enqueue_stage(g, k, st, dt, nullptr, g->cap_stream);
    st = next_state(g, st);
  }
  cudaGraph_t graph = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(g->cap_stream, &graph);
  if (err != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return cuda_fail(err, "kernel launch during graph capture");
  }
  if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
  cudaGraphExec_t exec = nullptr;
  cudaError_t e3 = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e3 != cudaSuccess) return cuda_fail(e3, "cudaGraphInstantiate");
  g->graph[state] = exec;
  g->graph_dt[state] = dt;
  return SBLI_OK;
}

}  // namespace

extern "C" {

int sbli_abi_version(void) { return SBLI_ABI_VERSION; }

const char* sbli_last_error(void) { return g_last_error.c_str(); }

int sbli_workspace_bytes(int n0, int n1, int n2, int precision, int variant, size_t* bytes) {
  if (!bytes) return fail(SBLI_EINVAL, "bytes is null");
  if (!valid_sizes(n0, n1, n2)) return fail(SBLI_EINVAL, "grid %d x %d x %d: each edge must be >= 5, n0*n1 < 2^31 and n0*n1*n2 < 2^32", n0, n1, n2);
  if (precision < SBLI_FP64 || precision > SBLI_DF64) return fail(SBLI_EINVAL, "unknown precision %d", precision);
  if (variant < SBLI_FUSED || variant > SBLI_SN2) return fail(SBLI_EINVAL, "unknown variant %d", variant);
  if ((precision == SBLI_FP32_DF || precision == SBLI_DF64) && variant != SBLI_FUSED)
    return fail(SBLI_EUNSUPPORTED, "the double-float modes are provided for the fused variant only");
  if (variant > SBLI_STORE_ALL && precision != SBLI_FP64)
    return fail(SBLI_EUNSUPPORTED, "the RS/SS/RA/SN/SN2 comparison variants are binary64 only");
  *bytes = layout_for(n0, n1, n2, precision, variant).total;
  return SBLI_OK;
}

int sbli_create_grid(sbli_grid** out, int n0, int n1, int n2, int precision, int variant, const sbli_params* params,
                     void* workspace, size_t workspace_bytes, void* stream) {
  if (!out) return fail(SBLI_EINVAL, "out is null");
  *out = nullptr;
  size_t need = 0;
  int rc = sbli_workspace_bytes(n0, n1, n2, precision, variant, &need);
  if (rc != SBLI_OK) return rc;
  if (!params) return fail(SBLI_EINVAL, "params is null");
  const sbli_params& p = *params;
  if (!(p.Re > 0) || !(p.Mach > 0) || !(p.Pr > 0) || !(p.gamma > 1) || !(p.L > 0) || isnan(p.Re) ||
      !isfinite(p.Mach) || !isfinite(p.Pr) || !isfinite(p.gamma) || !isfinite(p.L))
    return fail(SBLI_EINVAL, "invalid physical parameters (Re=%g M=%g Pr=%g gamma=%g L=%g)", p.Re, p.Mach, p.Pr,
                p.gamma, p.L);
  if (!workspace) return fail(SBLI_EINVAL, "workspace is null");
  if (((uintptr_t)workspace) % ALIGN) return fail(SBLI_EINVAL, "workspace must be 256-byte aligned");
  if (workspace_bytes < need)
    return fail(SBLI_ENOMEM, "workspace has %zu bytes, grid needs %zu", workspace_bytes, need);
  cudaPointerAttributes attr;
  cudaError_t pe = cudaPointerGetAttributes(&attr, workspace);
  if (pe != cudaSuccess || attr.type != cudaMemoryTypeDevice) {
    cudaGetLastError();
    return fail(SBLI_EINVAL, "workspace is not device memory");
  }

  sbli_grid* g = new sbli_grid();
  memset(g->graph, 0, sizeof g->graph);
  g->n[0] = n0; g->n[1] = n1; g->n[2] = n2;
  g->precision = precision;
  g->variant = variant;
  g->params = p;
  g->geom = Geom{n0, n1, n2, (long long)n0 * n1 * n2};
  g->stream = static_cast<cudaStream_t>(stream);
  g->layout = layout_for(n0, n1, n2, precision, variant);
  char* w = static_cast<char*>(workspace);
  for (int r = 0; r < g->layout.n64; ++r, w += g->layout.reg64) g->reg64[r] = reinterpret_cast<double*>(w);
  for (int r = 0; r < g->layout.n32; ++r, w += g->layout.reg32) g->reg32[r] = reinterpret_cast<float*>(w);
  g->partials = reinterpret_cast<double*>(w);
  g->ke_out = g->partials + (g->layout.partials / sizeof(double) - 2);
  w += g->layout.partials;
  g->storeall = g->layout.storeall ? static_cast<void*>(w) : nullptr;
  g->state = initial_state(precision);
  g->next_stage = 0;
  g->stages_done = 0;
  g->cfg = default_config(g->geom, precision);
  g->cd = make_coef<double>(g->n, p);
  g->cf = make_coef<float>(g->n, p);
  g->cw = make_coef<dfloat>(g->n, p);
  g->ref = make_ref(p);
  cudaError_t e = cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete g;
    return cuda_fail(e, "cudaStreamCreateWithFlags");
  }
  *out = g;
  return SBLI_OK;
}

int sbli_destroy_grid(sbli_grid* g) {
  if (!g) return SBLI_OK;
  cudaStreamSynchronize(g->stream);
  drop_graphs(g);
  cudaStreamDestroy(g->cap_stream);
  delete g;
  return SBLI_OK;
}

int sbli_init_tgv(sbli_grid* g, double amplitude) {
  if (int rc = check_grid(g)) return rc;
  if (!isfinite(amplitude)) return fail(SBLI_EINVAL, "amplitude must be finite");
  g->state = initial_state(g->precision);
  g->next_stage = 0;
  g->stages_done = 0;
  if (g->precision == SBLI_FP32_DF) {
    // binary64 deviation field into the free register, then split into hi/lo
    SBLI_TRY(launch_init_tgv(g->geom, g->params, amplitude, g->reg64[1], g->stream), "init_tgv launch");
    const RefState zero{0.0, 0.0};
    SBLI_TRY(launch_df_split(g->geom.P, zero, g->reg64[1], reinterpret_cast<float*>(g->reg64[0]), g->stream),
             "df_split");
    return SBLI_OK;
  }
  SBLI_TRY(launch_init_tgv(g->geom, g->params, amplitude, g->reg64[0], g->stream), "init_tgv launch");
  if (g->precision == SBLI_FP32)
    SBLI_TRY(launch_narrow(5 * g->geom.P, g->reg64[0], g->reg32[0], g->stream), "narrow launch");
  if (g->precision == SBLI_DF64)
    SBLI_TRY(launch_pair_split(5 * g->geom.P, g->reg64[0], reinterpret_cast<float*>(g->reg64[g->state]), g->stream),
             "pair_split launch");
  return SBLI_OK;
}

int sbli_set_state(sbli_grid* g, const double* q, int q_is_host) {
  if (int rc = check_grid(g)) return rc;
  if (!q) return fail(SBLI_EINVAL, "q is null");
  if (g->next_stage != 0) return fail(SBLI_EINVAL, "set_state between stages of a step (next stage %d)", g->next_stage);
  const size_t bytes = 5 * (size_t)g->geom.P * sizeof(double);
  // stage through a free register, then convert to deviation form
  const int dst = g->state;
  double* tmp = free64(g);
  if (q_is_host) {
    SBLI_TRY(cudaMemcpyAsync(tmp, q, bytes, cudaMemcpyHostToDevice, g->stream), "cudaMemcpyAsync H2D");
  } else {
    SBLI_TRY(cudaMemcpyAsync(tmp, q, bytes, cudaMemcpyDeviceToDevice, g->stream), "cudaMemcpyAsync D2D");
  }
  if (g->precision == SBLI_FP32_DF) {
    SBLI_TRY(launch_df_split(g->geom.P, g->ref, tmp, reinterpret_cast<float*>(g->reg64[dst]), g->stream), "df_split");
  } else {
    SBLI_TRY(launch_to_offset(g->geom, g->ref, tmp, state64(g), g->stream), "to_offset launch");
    if (g->precision == SBLI_FP32)
      SBLI_TRY(launch_narrow(5 * g->geom.P, g->reg64[dst], g->reg32[dst], g->stream), "narrow launch");
    if (g->precision == SBLI_DF64)
      SBLI_TRY(launch_pair_split(5 * g->geom.P, state64(g), reinterpret_cast<float*>(g->reg64[dst]), g->stream),
               "pair_split launch");
  }
  if (q_is_host) SBLI_TRY(cudaStreamSynchronize(g->stream), "cudaStreamSynchronize");
  g->stages_done = 0;
  return SBLI_OK;
}

int sbli_get_state(sbli_grid* g, double* q, int q_is_host) {
  if (int rc = check_grid(g)) return rc;
  if (!q) return fail(SBLI_EINVAL, "q is null");
  if (g->next_stage != 0) return fail(SBLI_EINVAL, "get_state between stages of a step (next stage %d)", g->next_stage);
  const size_t bytes = 5 * (size_t)g->geom.P * sizeof(double);
  double* tmp = free64(g);
  if (g->precision == SBLI_FP32_DF) {
    SBLI_TRY(launch_df_join(g->geom.P, g->ref, reinterpret_cast<const float*>(g->reg64[g->state]), tmp, g->stream),
             "df_join");
  } else {
    SBLI_TRY(launch_from_offset(g->geom, g->ref, state64(g), tmp, g->stream), "from_offset launch");
  }
  if (q_is_host) {
    SBLI_TRY(cudaMemcpyAsync(q, tmp, bytes, cudaMemcpyDeviceToHost, g->stream), "cudaMemcpyAsync D2H");
    SBLI_TRY(cudaStreamSynchronize(g->stream), "cudaStreamSynchronize");
  } else {
    SBLI_TRY(cudaMemcpyAsync(q, tmp, bytes, cudaMemcpyDeviceToDevice, g->stream), "cudaMemcpyAsync D2D");
  }
  return SBLI_OK;
}

int sbli_sample_state(sbli_grid* g, const long long* idx_dev, int count, double* out_dev) {
  if (int rc = check_grid(g)) return rc;
  if (count < 0) return fail(SBLI_EINVAL, "count %d < 0", count);
  if (count == 0) return SBLI_OK;
  if (!idx_dev || !out_dev) return fail(SBLI_EINVAL, "idx_dev or out_dev is null");
  if (g->next_stage != 0) return fail(SBLI_EINVAL, "sample_state between stages of a step (next stage %d)", g->next_stage);
  const bool df = g->precision == SBLI_FP32_DF;
  const double* q64 = df ? nullptr : state64(g);
  const float* qdf = df ? reinterpret_cast<const float*>(g->reg64[g->state]) : nullptr;
  SBLI_TRY(launch_sample_state(g->geom.P, g->ref, q64, qdf, idx_dev, count, out_dev, g->stream), "sample_state launch");
  return SBLI_OK;
}

int sbli_get_stage(sbli_grid* g, double* q_stage, double* q_acc, int q_is_host) {
  if (int rc = check_grid(g)) return rc;
  if (g->next_stage == 0) return fail(SBLI_EINVAL, "get_stage outside a step (no stage in progress)");
  const size_t n = 5 * (size_t)g->geom.P;
  const StagePtrs p = stage_ptrs(g, g->next_stage, g->state);
  // convert through the binary64 register this stage does not read
  auto copy_out = [&](const void* src, bool src64, double* dst) -> int {
    double* tmp = nullptr;
    if (f64_registers(g->precision)) {
      // the register not used by this stage holds nothing live
      for (int r = 0; r < 3; ++r)
        if (g->reg64[r] != p.q_in && g->reg64[r] != p.acc_in) tmp = g->reg64[r];
    } else if (g->precision == SBLI_FP32_DF) {
      tmp = g->reg64[g->state];  // Q^n (double-float) is not needed after stage 0
    } else {
      tmp = g->reg64[g->state];  // Q^n is not needed after stage 0
    }
    if (!tmp) return fail(SBLI_EINVAL, "no free register");
    if (src64) {
      SBLI_TRY(launch_from_offset(g->geom, g->ref, static_cast<const double*>(src), tmp, g->stream), "from_offset");
    } else if (g->precision == SBLI_DF64) {  // interleaved double-float pairs
      SBLI_TRY(launch_pair_join(5 * g->geom.P, static_cast<const float*>(src), tmp, g->stream), "pair_join");
      SBLI_TRY(launch_from_offset(g->geom, g->ref, tmp, tmp, g->stream), "from_offset");
    } else {
      SBLI_TRY(launch_widen(5 * g->geom.P, static_cast<const float*>(src), tmp, g->stream), "widen");
      SBLI_TRY(launch_from_offset(g->geom, g->ref, tmp, tmp, g->stream), "from_offset");
    }
    SBLI_TRY(cudaMemcpyAsync(dst, tmp, n * sizeof(double), q_is_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                             g->stream),
             "cudaMemcpyAsync");
    if (q_is_host) SBLI_TRY(cudaStreamSynchronize(g->stream), "cudaStreamSynchronize");
    return SBLI_OK;
  };
  if (q_stage)
    if (int rc = copy_out(p.q_in, p.in64, q_stage)) return rc;
  if (q_acc) {
    if (g->precision == SBLI_FP32_DF) {
      double* tmp = g->reg64[g->state];  // Q^n is not needed after stage 0
      SBLI_TRY(launch_df_join(g->geom.P, g->ref, p.dacc_in, tmp, g->stream), "df_join");
      SBLI_TRY(cudaMemcpyAsync(q_acc, tmp, n * sizeof(double),
                               q_is_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, g->stream),
               "cudaMemcpyAsync");
      if (q_is_host) SBLI_TRY(cudaStreamSynchronize(g->stream), "cudaStreamSynchronize");
    } else if (int rc = copy_out(p.acc_in, true, q_acc)) {
      return rc;
    }
  }
  return SBLI_OK;
}

int sbli_rhs(sbli_grid* g, double* r_dev) {
  if (int rc = check_grid(g)) return rc;
  if (!r_dev) return fail(SBLI_EINVAL, "r_dev is null");
  if (g->next_stage != 0) return fail(SBLI_EINVAL, "rhs between stages of a step");
  const double* q = state64(g);
  if (g->variant == SBLI_FUSED) {
    StageArgs a{};
    a.g = g->geom;
    a.zc = g->cfg.zc;
    a.q_in = q;
    a.r_out = r_dev;
    cudaError_t e = g->precision == SBLI_FP64      ? launch_fused_fp64(a, g->cd, g->cfg, true, g->stream)
                    : g->precision == SBLI_DF64    ? launch_fused_df64(a, g->cw, g->cfg, true, false, g->stream)
                    : g->precision == SBLI_FP32_DF ? launch_fused_fp32df(a, g->cf, g->cfg, true, g->stream)
                                                   : launch_fused_fp32(a, g->cf, g->cfg, true, true, g->stream);
    SBLI_TRY(e, "fused rhs launch");
    return SBLI_OK;
  }
  if (g->variant > SBLI_STORE_ALL) {
    SBLI_TRY(launch_algorithm_stage(g->variant, g->geom, g->cd, q, nullptr, nullptr, nullptr, r_dev, 0.0, 0.0,
                                    static_cast<double*>(g->storeall), g->stream),
             "rhs launch");
    return SBLI_OK;
  }
  if (g->precision == SBLI_FP64) {
    SBLI_TRY(launch_storeall_rhs_fp64(g->geom, g->cd, q, static_cast<double*>(g->storeall), r_dev, g->stream),
             "store-all rhs");
    return SBLI_OK;
  }
  // binary32 residual, widened to binary64
  float* scr = static_cast<float*>(g->storeall);
  SBLI_TRY(launch_storeall_rhs_fp32(g->geom, g->cf, q, true, scr, nullptr, g->stream), "store-all rhs");
  SBLI_TRY(launch_widen(5 * g->geom.P, scr + storeall_r_offset(g->geom), r_dev, g->stream), "widen residual");
  return SBLI_OK;
}

int sbli_rk_stage(sbli_grid* g, int stage, double dt) {
  if (int rc = check_grid(g)) return rc;
  if (stage < 0 || stage > 2) return fail(SBLI_EINVAL, "stage %d not in 0..2", stage);
  if (stage != g->next_stage) return fail(SBLI_EINVAL, "stage %d called, stage %d expected", stage, g->next_stage);
  if (!(dt > 0) || !isfinite(dt)) return fail(SBLI_EINVAL, "dt must be finite and > 0");
  SBLI_TRY(enqueue_stage(g, stage, g->state, dt, nullptr, g->stream), "stage launch");
  g->next_stage = (stage + 1) % 3;
  if (stage == 2) g->state = next_state(g, g->state);
  g->stages_done++;
  return SBLI_OK;
}

int sbli_step_n(sbli_grid* g, int nsteps, double dt) {
  if (int rc = check_grid(g)) return rc;
  if (nsteps < 0) return fail(SBLI_EINVAL, "nsteps < 0");
  if (!(dt > 0) || !isfinite(dt)) return fail(SBLI_EINVAL, "dt must be finite and > 0");
  if (g->next_stage != 0) return fail(SBLI_EINVAL, "step_n must start at a step boundary");
  int left = nsteps;
  while (left >= sbli_grid::GRAPH_STEPS) {
    if (int rc = build_graph(g, g->state, dt)) return rc;
    SBLI_TRY(cudaGraphLaunch(g->graph[g->state], g->stream), "cudaGraphLaunch");
    // GRAPH_STEPS is a multiple of the rotation period (3 and 2)
    left -= sbli_grid::GRAPH_STEPS;
    g->stages_done += 3 * sbli_grid::GRAPH_STEPS;
  }
  for (; left > 0; --left) {
    for (int k = 0; k < 3; ++k) SBLI_TRY(enqueue_stage(g, k, g->state, dt, nullptr, g->stream), "stage launch");
    g->state = next_state(g, g->state);
    g->stages_done += 3;
  }
  return SBLI_OK;
}

int sbli_step_n_history(sbli_grid* g, int nsteps, double dt, double* ke_hist_dev) {
  if (int rc = check_grid(g)) return rc;
  if (nsteps < 0) return fail(SBLI_EINVAL, "nsteps < 0");
  if (!ke_hist_dev && nsteps > 0) return fail(SBLI_EINVAL, "ke_hist_dev is null");
  if (!(dt > 0) || !isfinite(dt)) return fail(SBLI_EINVAL, "dt must be finite and > 0");
  if (g->next_stage != 0) return fail(SBLI_EINVAL, "step_n_history must start at a step boundary");
  if (g->variant != SBLI_FUSED) return fail(SBLI_EUNSUPPORTED, "history needs the fused variant");
  const int nctas = fused_num_ctas(g->geom, g->cfg);
  for (int s = 0; s < nsteps; ++s) {
    SBLI_TRY(enqueue_stage(g, 0, g->state, dt, g->partials, g->stream), "stage launch");
    SBLI_TRY(launch_finalize_ke(g->partials, nctas, 1.0 / (double)g->geom.P, ke_hist_dev + 2 * s, g->stream),
             "finalize launch");
    for (int k = 1; k < 3; ++k) SBLI_TRY(enqueue_stage(g, k, g->state, dt, nullptr, g->stream), "stage launch");
    g->state = next_state(g, g->state);
    g->stages_done += 3;
  }
  return SBLI_OK;
}

int sbli_kinetic_energy_async(sbli_grid* g, double* out_dev) {
  if (int rc = check_grid(g)) return rc;
  if (!out_dev) return fail(SBLI_EINVAL, "out_dev is null");
  if (g->next_stage != 0) return fail(SBLI_EINVAL, "kinetic_energy between stages of a step");
  const double* q = state64(g);
  if (g->precision == SBLI_FP32_DF) {
    double* tmp = g->reg64[1 - g->state];  // free at a step boundary
    const RefState zero{0.0, 0.0};
    SBLI_TRY(launch_df_join(g->geom.P, zero, reinterpret_cast<const float*>(g->reg64[g->state]), tmp, g->stream),
             "df_join");
    q = tmp;
  }
  SBLI_TRY(launch_ke(g->geom, g->cd, g->ref, q, g->partials, out_dev, g->stream), "ke launch");
  return SBLI_OK;
}

int sbli_kinetic_energy(sbli_grid* g, double* ke, double* enstrophy) {
  if (int rc = check_grid(g)) return rc;
  if (!ke || !enstrophy) return fail(SBLI_EINVAL, "null output pointer");
  if (int rc = sbli_kinetic_energy_async(g, g->ke_out)) return rc;
  double h[2];
  SBLI_TRY(cudaMemcpyAsync(h, g->ke_out, sizeof h, cudaMemcpyDeviceToHost, g->stream), "cudaMemcpyAsync D2H");
  SBLI_TRY(cudaStreamSynchronize(g->stream), "cudaStreamSynchronize");
  *ke = h[0];
  *enstrophy = h[1];
  return SBLI_OK;
}

int sbli_get_config(const sbli_grid* g, int* tile_y, int* planes_per_cta, int* z_queue, int* columns_per_thread) {
  if (!g || !tile_y || !planes_per_cta) return fail(SBLI_EINVAL, "null argument");
  *tile_y = g->cfg.ty;
  *planes_per_cta = g->cfg.zc;
  if (z_queue) *z_queue = g->cfg.zq;
  if (columns_per_thread) *columns_per_thread = g->cfg.px;
  return SBLI_OK;
}

int sbli_set_config(sbli_grid* g, int tile_y, int planes_per_cta, int z_queue, int columns_per_thread) {
  if (int rc = check_grid(g)) return rc;
  if (g->next_stage != 0) return fail(SBLI_EINVAL, "set_config between stages of a step");
  if (!valid_config(g->precision, tile_y, planes_per_cta, z_queue, columns_per_thread) ||
      ((z_queue || columns_per_thread != 1) && g->variant != SBLI_FUSED))
    return fail(SBLI_EINVAL,
                "config tile_y=%d planes_per_cta=%d z_queue=%d columns_per_thread=%d not available for this grid",
                tile_y, planes_per_cta, z_queue, columns_per_thread);
  FusedConfig cfg;
  cfg.ty = tile_y;
  cfg.zc = std::min(planes_per_cta, g->geom.n2);
  cfg.zq = z_queue;
  cfg.px = columns_per_thread;
  if (cfg.ty != g->cfg.ty || cfg.zc != g->cfg.zc || cfg.zq != g->cfg.zq || cfg.px != g->cfg.px) {
    g->cfg = cfg;
    drop_graphs(g);
  }
  return SBLI_OK;
}

int sbli_autotune(sbli_grid* g, int reps, int* tile_y, int* planes_per_cta, int* z_queue, int* columns_per_thread,
                  float* best_stage_ms) {
  if (int rc = check_grid(g)) return rc;
  if (g->next_stage != 0) return fail(SBLI_EINVAL, "autotune between stages of a step");
  if (g->variant != SBLI_FUSED) return fail(SBLI_EUNSUPPORTED, "autotune needs the fused variant");
  if (reps < 1) return fail(SBLI_EINVAL, "reps must be >= 1");
  constexpr int ZC_CANDIDATES = 6;  // planes-per-CTA values per kernel shape, best first by the wave model
  FusedConfig cand[8 * ZC_CANDIDATES];
  int nc = 0;
  const int tys[2] = {8, 16};
  for (int px = 1; px <= 2; ++px)
    for (int zq = 0; zq < 2; ++zq)
      for (int t = 0; t < 2; ++t) {
        if (!valid_config(g->precision, tys[t], 4, zq, px)) continue;
        int zc[ZC_CANDIDATES];
        rank_zc(g->geom, g->precision, tys[t], zc, ZC_CANDIDATES, px, zq);
        for (int i = 0; i < ZC_CANDIDATES; ++i) {
          bool dup = false;
          const int z = std::max(4, std::min(zc[i], g->geom.n2));
          for (int j = 0; j < nc; ++j)
            dup |= (cand[j].ty == tys[t] && cand[j].zc == z && cand[j].zq == zq && cand[j].px == px);
          if (!dup && nc < 8 * ZC_CANDIDATES) cand[nc++] = FusedConfig{tys[t], z, zq, px};
        }
      }
  cudaEvent_t e0, e1;
  SBLI_TRY(cudaEventCreate(&e0), "cudaEventCreate");
  cudaError_t ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_fail(ce, "cudaEventCreate");
  }
  const FusedConfig saved = g->cfg;
  int best = -1;
  float best_ms = 1e30f;
  cudaError_t err = cudaSuccess;
  for (int i = 0; i < nc && err == cudaSuccess; ++i) {
    g->cfg = cand[i];
    // stage 0 with dt = 0: the accumulator it writes equals the state it
    // reads (acc + 0 * R), so a double-float grid's state, updated in place,
    // keeps its value; the stage field goes to a free register
    err = enqueue_stage(g, 0, g->state, 0.0, nullptr, g->stream);
    if (err == cudaSuccess) err = cudaEventRecord(e0, g->stream);
    for (int r = 0; r < reps && err == cudaSuccess; ++r) err = enqueue_stage(g, 0, g->state, 0.0, nullptr, g->stream);
    if (err == cudaSuccess) err = cudaEventRecord(e1, g->stream);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    ms /= (float)reps;
    if (err == cudaSuccess && ms < best_ms) {
      best_ms = ms;
      best = i;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) {
    g->cfg = saved;
    return cuda_fail(err, "autotune launch");
  }
  g->cfg = cand[best];
  if (g->cfg.ty != saved.ty || g->cfg.zc != saved.zc || g->cfg.zq != saved.zq || g->cfg.px != saved.px)
    drop_graphs(g);
  if (tile_y) *tile_y = g->cfg.ty;
  if (planes_per_cta) *planes_per_cta = g->cfg.zc;
  if (z_queue) *z_queue = g->cfg.zq;
  if (columns_per_thread) *columns_per_thread = g->cfg.px;
  if (best_stage_ms) *best_stage_ms = best_ms;
  return SBLI_OK;
}

int sbli_stage_count(const sbli_grid* g, long long* stages) {
  if (!g || !stages) return fail(SBLI_EINVAL, "null argument");
  *stages = g->stages_done;
  return SBLI_OK;
}

}  // extern "C"
