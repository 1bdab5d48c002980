/*
 * sbli.h -- C ABI of the GB300 (sm_103a) fused Navier-Stokes RHS + RK3 stage.
 *
 * The operation is the residual R(Q) of the non-dimensional compressible
 * Navier-Stokes equations (Jammy, Jacobs, Lusher & Sandham, arXiv:1709.09713,
 * §2, Eqs. 1-5) discretised by the fourth-order central stencils of Eqs. 6-7
 * on a periodic grid, advanced by the three-stage low-storage Runge-Kutta
 * scheme of §2.2 (Eq. 8, Fig. 1), on the Taylor-Green vortex of §4.
 *
 * Conventions for every call:
 *  - Every function returns an int status (enum sbli_status).  Nothing aborts
 *    the process; on failure sbli_last_error() returns a message (per host
 *    thread) and the grid is left as it was before the call.
 *  - Grids are n0 x n1 x n2 points on [0, 2*pi*L)^3, x_i = i*h_i,
 *    h_i = 2*pi*L/n_i, periodic in every direction; each n_i >= 5 (the
 *    5-point stencils of Eqs. 6-7).  Fields are stored x0-fastest
 *    (index i + n0*(j + n1*k)), five consecutive fields per state in the
 *    order (rho, rho*u0, rho*u1, rho*u2, rho*E).
 *  - Device memory is owned by the caller (e.g. PyTorch): the library never
 *    allocates or frees device memory.  It carves the caller's workspace.
 *  - Work is enqueued on the CUDA stream given at creation; the library does
 *    not synchronise except in calls that return host scalars or copy to or
 *    from host memory (stated per call).
 *  - Precision SBLI_FP64: every value stored and computed in IEEE binary64.
 *    Precision SBLI_FP32: stage fields stored and the residual computed in
 *    binary32; the Runge-Kutta accumulator (the n+1 level of Fig. 1) and
 *    the state between steps are binary64; kinetic-energy and enstrophy sums
 *    are binary64.  Precision SBLI_FP32_DF: as SBLI_FP32, but the accumulator
 *    and the state between steps are double-float pairs (hi + lo, two
 *    binary32, about 48 significant bits) updated with error-free binary32
 *    additions, so no binary64 arithmetic runs in the stages (fused variant;
 *    single grids, batches and requests).  Precision SBLI_DF64: binary64 state and
 *    accumulator as SBLI_FP64, but the stage arithmetic (primitives,
 *    derivatives, residual) in double-float: each value a hi + lo pair of
 *    binary32 (about 48 significant bits) evaluated on the binary32 pipe with
 *    error-free transformations; the RK update is the binary64 FMA.  The
 *    stage fields, and on single grids a copy of the state, are stored as
 *    those (hi, lo) pairs, split once by the stage that writes them (fused
 *    variant; single grids, batches and requests).  All store the state as deviations from the uniform
 *    reference state (rho = 1, u = 0, p = 1/(gamma M^2)); the
 *    get/set calls convert to and from the plain conserved variables.
 *  - Variant SBLI_FUSED evaluates every derivative on the fly and writes the
 *    stage update in the same kernel (the minimal-storage class of §2.5, with
 *    the RK update of Fig. 1 fused in): the product path.  Variant
 *    SBLI_STORE_ALL stores each derivative in its own array first (the BL
 *    algorithm of §2.3.1).  Variants SBLI_RS and SBLI_SS store the 9 velocity
 *    gradients to arrays and evaluate the other derivatives on the fly,
 *    recomputed at each occurrence (RS) or once into thread-local variables
 *    (SS); SBLI_RA, SBLI_SN and SBLI_SN2 store nothing and recompute every
 *    derivative at each occurrence (RA), or evaluate each once into
 *    thread-local variables in listed order (SN) or grouped by velocity
 *    component (SN2): the paper's intermediate- and minimal-storage classes
 *    (§2.4, §2.5), one thread per point, binary64 only, for comparison.
 */
#ifndef SBLI_H
#define SBLI_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SBLI_ABI_VERSION 1

#if defined(__GNUC__)
#define SBLI_API __attribute__((visibility("default")))
#else
#define SBLI_API
#endif

enum sbli_status {
  SBLI_OK = 0,
  SBLI_EINVAL = 1,       /* bad argument: size, pointer, alignment, stage order */
  SBLI_ENOMEM = 2,       /* the caller's workspace is smaller than required */
  SBLI_ECUDA = 3,        /* a CUDA runtime call or kernel launch failed */
  SBLI_ETIMEOUT = 4,     /* a bounded device-side wait gave up */
  SBLI_EUNSUPPORTED = 5  /* precision/variant combination not provided */
};

enum sbli_precision { SBLI_FP64 = 0, SBLI_FP32 = 1, SBLI_FP32_DF = 2, SBLI_DF64 = 3 };
enum sbli_variant {
  SBLI_FUSED = 0,
  SBLI_STORE_ALL = 1,
  SBLI_RS = 2,
  SBLI_SS = 3,
  SBLI_RA = 4,
  SBLI_SN = 5,
  SBLI_SN2 = 6
};

/* Physical parameters (§2 Eqs. 1-5, §4): Re may be +INFINITY, which removes
 * the viscous and heat-flux terms. */
typedef struct {
  double Re;    /* Reynolds number, > 0 */
  double Mach;  /* reference Mach number M, > 0 */
  double Pr;    /* Prandtl number, > 0 */
  double gamma; /* ratio of specific heats, > 1 */
  double L;     /* domain edge is 2*pi*L, > 0 */
} sbli_params;

typedef struct sbli_grid sbli_grid;

/* ABI version the library was built with (SBLI_ABI_VERSION). */
SBLI_API int sbli_abi_version(void);

/* Bytes of device workspace a grid needs (state registers, stage fields and
 * scratch).  Returns SBLI_EINVAL for n_i < 5, n0*n1 >= 2^31, n0*n1*n2 >= 2^32
 * (the stage kernels address a point of one field with a 32-bit unsigned
 * offset) or unknown precision/variant. */
SBLI_API int sbli_workspace_bytes(int n0, int n1, int n2, int precision, int variant, size_t* bytes);

/* Create a grid over a caller-owned device workspace of at least
 * sbli_workspace_bytes() bytes, 256-byte aligned.  stream is a cudaStream_t
 * (NULL = legacy default stream).  The workspace must stay allocated until
 * sbli_destroy_grid.  The state is undefined until sbli_init_tgv or
 * sbli_set_state. */
SBLI_API int sbli_create_grid(sbli_grid** out, int n0, int n1, int n2, int precision, int variant,
                     const sbli_params* params, void* workspace, size_t workspace_bytes, void* stream);

/* Release the handle (not the workspace).  Waits for the grid's stream. */
SBLI_API int sbli_destroy_grid(sbli_grid* g);

/* Taylor-Green initial field of §4 (Eqs. 9-12), velocity amplitude A
 * (A = 1 is the paper's), density from T = 1 (rho = gamma M^2 p, Eq. 5) and
 * rho*E from Eq. 4.  Asynchronous. */
SBLI_API int sbli_init_tgv(sbli_grid* g, double amplitude);

/* Copy the state in or out as 5*n0*n1*n2 binary64 plain conserved variables.
 * q_is_host != 0: q is host memory (ideally pinned); the call copies through
 * the grid's stream and returns after the copy completed.  q_is_host == 0: q
 * is device memory, asynchronous.  Fails with SBLI_EINVAL between the stages
 * of a time step. */
SBLI_API int sbli_set_state(sbli_grid* g, const double* q, int q_is_host);
SBLI_API int sbli_get_state(sbli_grid* g, double* q, int q_is_host);

/* Read a few points of the state without a full copy (grids too large for a
 * second state-sized buffer).  idx_dev: count linear point indices
 * i0 + n0*(i1 + n1*i2) in device memory (int64); out_dev: device memory for
 * 5*count binary64, written field-major (out_dev[f*count + m] is field f of
 * point idx_dev[m]) with the plain conserved variables, bit-identical to the
 * same entries of sbli_get_state.  An index outside [0, n0*n1*n2) yields NaN
 * in its five entries (no fault).  count == 0 is a no-op.  Asynchronous on
 * the grid's stream; SBLI_EINVAL between the stages of a step. */
SBLI_API int sbli_sample_state(sbli_grid* g, const long long* idx_dev, int count, double* out_dev);

/* Between the stages of a step (after stage 0 or 1): copy out the next
 * stage's input field Q_k and the accumulator Q_acc as 5*n0*n1*n2 binary64
 * plain conserved variables (binary32 stage fields are widened, double-float
 * pair fields joined exactly).  For
 * verifying single stages.  Either pointer may be NULL.  q_is_host as in
 * sbli_get_state (host copies synchronise). */
SBLI_API int sbli_get_stage(sbli_grid* g, double* q_stage, double* q_acc, int q_is_host);

/* R(Q) of the current state (Eqs. 1-3 with Eqs. 4-7) into r_dev, a device
 * array of 5*n0*n1*n2 binary64, same field order as the state.  For SBLI_FP32
 * grids the residual is computed in binary32 and widened.  Asynchronous. */
SBLI_API int sbli_rhs(sbli_grid* g, double* r_dev);

/* One Runge-Kutta stage k = 0, 1, 2 of the current step (§2.2, Fig. 1), in
 * two-register form with stage coefficients a = (2/3, 5/12, 3/5) and
 * accumulator coefficients b = (1/4, 3/20, 3/5):
 *     R = R(Q_k);  Q_{k+1} = Q_acc + a_k dt R;  Q_acc = Q_acc + b_k dt R,
 * Q_acc = Q^n before stage 0 and Q^{n+1} = Q_acc after stage 2.  Stages
 * must be called in order 0, 1, 2 (else SBLI_EINVAL); dt > 0.  Asynchronous. */
SBLI_API int sbli_rk_stage(sbli_grid* g, int stage, double dt);

/* nsteps complete time steps (3*nsteps stages), launched as a captured CUDA
 * graph.  Must start at a step boundary.  Asynchronous. */
SBLI_API int sbli_step_n(sbli_grid* g, int nsteps, double dt);

/* As sbli_step_n, and writes the volume-averaged kinetic energy and enstrophy
 * of Q^n before each step s into ke_hist_dev[2*s], ke_hist_dev[2*s+1]
 * (device memory, 2*nsteps binary64).  Fused variant only. Asynchronous. */
SBLI_API int sbli_step_n_history(sbli_grid* g, int nsteps, double dt, double* ke_hist_dev);

/* Volume averages of the current state, accumulated in binary64:
 *   ke = <rho |u|^2 / 2>,  enstrophy = <rho |omega|^2 / 2>,  omega = curl u
 * with Eq. 6 derivatives.  Synchronises the grid's stream. */
SBLI_API int sbli_kinetic_energy(sbli_grid* g, double* ke, double* enstrophy);

/* Same quantities written to device memory out_dev[0..1]; asynchronous. */
SBLI_API int sbli_kinetic_energy_async(sbli_grid* g, double* out_dev);

/* Kinetic energy and enstrophy, as sbli_kinetic_energy computes them, of a
 * state the caller owns, without any device allocation by the caller or the
 * library.  The paper has no counterpart: this entry point exists for callers
 * that cannot allocate device memory (an application that reserves the whole
 * device up front, code handed only a state pointer, loops that must not
 * allocate once running) and therefore cannot provide a grid workspace.
 *   q_dev   device array of 5*n0*n1*n2 binary64 plain conserved variables,
 *           layout as sbli_get_state writes it (read only);
 *   L       domain edge / (2 pi) (h_i = 2 pi L / n_i);
 *   out_dev device array of 2 binary64: (ke, enstrophy) volume averages;
 *   stream  cudaStream_t the kernels run on (NULL = legacy default stream).
 * The partial sums live in one static device array of the library, 8192
 * pairs (128 KiB per GPU, held until the process exits); grids of more than
 * 8192 * 16384 = 134,217,728 points (512^3) are rejected with SBLI_EINVAL.
 * A call made while its stream is not being captured looks up that array's
 * device address (again, so a device reset between calls is harmless); a call
 * during stream capture reuses the address found by an earlier call on the
 * device, so make the first call on each device before any stream capture
 * (else SBLI_EINVAL).  q_dev and out_dev must be device or managed memory of
 * the current device (else SBLI_EINVAL, nothing launched).  Every call
 * overwrites the array (each partial sum is written before it is read, so
 * nothing needs clearing); calls that overlap on the GPU, on any streams, race
 * on it and must be ordered by the caller.  Asynchronous. */
SBLI_API int sbli_kinetic_energy_noalloc(const double* q_dev, int n0, int n1, int n2, double L, double* out_dev,
                                         void* stream);

/* Launch configuration of the fused kernel: in-plane tile height (the tile
 * is 32 x tile_y points per column a thread owns; binary64-register grids
 * (SBLI_FP64, SBLI_DF64) use 8, binary32 grids 8 or 16), planes per CTA
 * along x2 (>= 4), where each thread keeps its column's records of the five
 * x2 planes (z_queue = 0: the shared-memory ring; 1: a per-thread queue in
 * Blackwell tensor memory, with only three full-record planes in shared
 * memory -- four for binary32 tile_y 16, which saves one barrier per plane)
 * and, for binary32 grids, how many columns each thread owns
 * (columns_per_thread = 1, or 2: columns x and x + 32 of a 64 x 8 tile
 * computed together in packed two-lane FP32 instructions; shared-memory
 * ring only).  Tile height, planes
 * per CTA and z_queue give bitwise the same state; two columns per thread
 * fuse multiply-adds differently (bitwise equal among themselves, within the
 * binary32 tolerance of one column).  set_config validates and applies it
 * (cached step graphs are rebuilt); must be called at a step boundary.
 * z_queue and columns_per_thread may be NULL in get_config. */
SBLI_API int sbli_get_config(const sbli_grid* g, int* tile_y, int* planes_per_cta, int* z_queue,
                             int* columns_per_thread);
SBLI_API int sbli_set_config(sbli_grid* g, int tile_y, int planes_per_cta, int z_queue, int columns_per_thread);

/* Autotuner: times candidate configurations (each allowed tile height, z
 * queue and columns per thread with the six planes-per-CTA values a
 * wave-balance model ranks best) on this grid with `reps` timed stage-0 launches each,
 * at dt = 0 (the accumulator they write equals the state they read, so a
 * double-float grid's state, updated in place, keeps its value; the stage
 * field goes to a free register), keeps the
 * fastest and returns it.  The state is not changed.  Synchronises the grid's
 * stream.  Fused variant only. */
SBLI_API int sbli_autotune(sbli_grid* g, int reps, int* tile_y, int* planes_per_cta, int* z_queue,
                           int* columns_per_thread, float* best_stage_ms);

/* ---------------------------------------------------------------------
 * Batched ensembles: up to 64 members (each its own grid size, Re, M, Pr,
 * gamma, L) advanced together.  Every Runge-Kutta stage of all members is one
 * persistent kernel launch that walks the members' work items (z chunk x
 * 32 x 8 tile, the z chunk per member set by the schedule below); step loops
 * are captured as CUDA graphs.  Any precision of
 * sbli_precision, as for single grids (others: SBLI_EINVAL).  Members'
 * results are bitwise those of the same member run alone as a single grid
 * with tile height 8.
 * n: 3*count edge lengths (n0, n1, n2 per member); params: count entries.
 * --------------------------------------------------------------------- */
typedef struct sbli_batch sbli_batch;

SBLI_API int sbli_batch_workspace_bytes(int count, const int* n, int precision, size_t* bytes);
SBLI_API int sbli_batch_create(sbli_batch** out, int count, const int* n, const sbli_params* params, int precision,
                               void* workspace, size_t workspace_bytes, void* stream);
SBLI_API int sbli_batch_destroy(sbli_batch* b);
SBLI_API int sbli_batch_count(const sbli_batch* b, int* count);
/* Total work items of one stage (for scheduling diagnostics). */
SBLI_API int sbli_batch_work_items(const sbli_batch* b, long long* items);
/* The batch's schedule: z_queue (0 = x2-neighbour records from the
 * shared-memory ring, 1 = from the per-thread TMEM queue, as for single grids)
 * and each member's planes per work item (planes_per_item[count]: the z chunk
 * a CTA marches through; >= 4, clamped to the member's n2).  A batch starts
 * with the TMEM queue for binary32 precisions and the ring otherwise, and
 * min(n2, 32) planes per item.  Every schedule gives bitwise the same
 * results.  set_schedule (between steps; SBLI_EINVAL for z_queue outside 0..1
 * or fewer than 4 planes) drops the captured step graphs; planes_per_item may
 * be NULL in both calls (keep, or do not return, the per-member values). */
SBLI_API int sbli_batch_get_schedule(const sbli_batch* b, int* z_queue, int* planes_per_item);
SBLI_API int sbli_batch_set_schedule(sbli_batch* b, int z_queue, const int* planes_per_item);
/* Autotuner of the schedule: times stage-0 launches with dt = 0 (reps each;
 * the accumulator they write equals the state they read, so a state updated
 * in place keeps its value, and the stage field goes to a free register) of
 * every z_queue mode with one planes-per-item value for all
 * members (8, 16, 32, 64, 128, whole member), then refines the planes per
 * item of each size class (members with the same n2) in turn, and keeps the
 * fastest schedule (if a trial launch fails, the schedule in place before
 * the call is restored and SBLI_ECUDA returned).  The state is not
 * changed.  Synchronises the batch's
 * stream.  *z_queue and *best_stage_ms (may be NULL) return the choice and
 * its stage time; sbli_batch_get_schedule returns the planes per item. */
SBLI_API int sbli_batch_autotune(sbli_batch* b, int reps, int* z_queue, float* best_stage_ms);
/* Taylor-Green initial field per member with amplitudes[count]. */
SBLI_API int sbli_batch_init_tgv(sbli_batch* b, const double* amplitudes);
/* Member state in/out as plain binary64 conserved variables (as sbli_set_state). */
SBLI_API int sbli_batch_set_state(sbli_batch* b, int member, const double* q, int q_is_host);
SBLI_API int sbli_batch_get_state(sbli_batch* b, int member, double* q, int q_is_host);
/* nsteps time steps of every member with time step dt.  Asynchronous. */
SBLI_API int sbli_batch_step_n(sbli_batch* b, int nsteps, double dt);
/* As sbli_batch_step_n, writing (ke, enstrophy) of every member before each
 * step s at ke_hist_dev[2*(count*s + m)] (device, 2*count*nsteps binary64). */
SBLI_API int sbli_batch_step_n_history(sbli_batch* b, int nsteps, double dt, double* ke_hist_dev);
/* Per-member volume averages (binary64) into host arrays ke[count],
 * enstrophy[count].  Synchronises the batch's stream. */
SBLI_API int sbli_batch_kinetic_energy(sbli_batch* b, double* ke, double* enstrophy);

/* ---------------------------------------------------------------------
 * Serving: a continuous-batching request loop.  Requests wait in arrival
 * order and are admitted when one of max_slots slots and a block of the
 * caller's device arena are free (first fit; with backfill != 0 a later
 * request that fits may pass one that does not).  Admitted requests keep
 * their state resident and run in two independent lanes: binary64-register
 * precisions on the first stream, binary32 ones on the second, which overlap
 * on the device and never wait for each other.  A lane advances all its
 * requests together in batches of K time steps (the requests of each
 * precision as one persistent multi-member launch per stage), K sized for a
 * few milliseconds of device time and never past the smallest remaining step
 * count of the batch.  When a lane's batch has completed, its finished
 * requests are retired (binary64 kinetic energy and enstrophy of the final
 * state, optional copy of the state to `result`, release of the block) and
 * its next batch starts.  A request's result equals the same problem run
 * alone as a single grid with tile height 8, bitwise.
 * --------------------------------------------------------------------- */
typedef struct sbli_server sbli_server;

typedef struct {
  int n0, n1, n2;      /* grid */
  int precision;       /* any sbli_precision */
  int steps;           /* time steps to run (>= 0) */
  double dt;           /* time step (> 0) */
  sbli_params params;  /* Re, M, Pr, gamma, L */
  double amplitude;    /* Taylor-Green velocity amplitude of the initial field */
  double* result;      /* final plain state (5*P binary64) is copied here, or NULL */
  int result_is_host;  /* result is host memory */
} sbli_request;

typedef struct {
  long long id;        /* as returned by sbli_server_submit */
  double ke, enstrophy;  /* volume averages of the final state (binary64) */
  double t_submit, t_admit, t_done;  /* seconds since server creation */
  int steps, precision;
  long long points;
} sbli_result;

typedef struct {
  int pending, active, completed_unpolled;
  size_t free_bytes, largest_free_block, arena_bytes;
  long long ticks;
  double now;          /* seconds since server creation */
} sbli_server_status;

/* arena: caller-owned device memory (256-byte aligned) the server carves into
 * per-request blocks; it stays owned by the caller. */
SBLI_API int sbli_server_create(sbli_server** out, void* arena, size_t arena_bytes, int max_slots, int backfill,
                                void* stream_fp64, void* stream_fp32);
SBLI_API int sbli_server_destroy(sbli_server* s);
/* Device bytes a request occupies while active. */
SBLI_API int sbli_server_request_bytes(const sbli_request* r, size_t* bytes);
/* Queue a request (copied); SBLI_ENOMEM if it can never fit the arena. */
SBLI_API int sbli_server_submit(sbli_server* s, const sbli_request* r, long long* id);
/* Admit waiting requests, then for each lane whose batch has completed:
 * retire its finished requests and launch its next batch (a lane still
 * running is left alone).  If neither lane could make progress, waits up to
 * about 2 ms for one to finish.  Returns without synchronising a running
 * lane; *completed = requests retired by this tick.  SBLI_ECUDA if a launch
 * or copy fails: a request whose initial field could not be launched goes
 * back to the head of the queue with its block released; a request whose
 * retirement failed stays active and is retried by the next tick. */
SBLI_API int sbli_server_tick(sbli_server* s, int* completed);
/* Move up to max retired requests' results into out; *n = how many. */
SBLI_API int sbli_server_poll(sbli_server* s, sbli_result* out, int max, int* n);
SBLI_API int sbli_server_stats(const sbli_server* s, sbli_server_status* status);

/* Number of stages completed since creation or the last set_state/init. */
SBLI_API int sbli_stage_count(const sbli_grid* g, long long* stages);

/* Message describing the last failure on this host thread ("" if none). */
SBLI_API const char* sbli_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SBLI_H */
