// fused_stage.cuh -- fused residual + low-storage RK stage kernel (sm_103a).
//
// One kernel evaluates R(Q) of Eqs. 1-3 (arXiv:1709.09713, §2) with every
// derivative of Eqs. 6-7 computed on the fly (no derivative arrays: the
// "store none" class of §2.5, ordered by velocity component as in SN2) and
// writes the Runge-Kutta stage of §2.2 / Fig. 1 in the same pass.
//
// Work decomposition (2.5D streaming):
//   * a CTA owns a 32 x TY tile of (x0, x1) columns and marches along x2
//     over zc planes; one thread per column, a warp is one x0 row, so every
//     global access is a coalesced row segment;
//   * a ring of 5 shared-memory slots holds the primitives of planes
//     z-2..z+2 on the tile plus a 2-point halo in x0 and x1 (corners
//     included), one 10-value record per point (array of structures, read
//     with 8- or 16-byte vector loads at bank-conflict-free strides).  A
//     plane's primitives are computed once, when it enters the ring, from the
//     conserved variables loaded from HBM (periodic wrap in the index
//     arithmetic replaces the boundary pass of Fig. 1);
//   * the loads of the next entering plane are issued as soon as the current
//     plane is stored, and the centre plane's accumulator values as its
//     derivative terms start, so HBM latency overlaps the arithmetic;
//   * x0/x1 derivatives read the centre slot, x2 derivatives read the ring;
//     each axis streams its four neighbour records through the accumulators
//     one at a time (axis_terms_stream; the double-float type keeps the
//     difference-first form, axis_terms);
//   * ZT (the z queue): each thread keeps its own column's records of the
//     five ring planes, and their in-plane gradients, in tensor memory
//     (TMEM), so the x2 derivatives read TMEM and shared memory keeps full
//     records only for the entering, middle and centre planes: binary32 59 KiB
//     per 32 x 8 CTA, three CTAs per SM (binary64 and double-float records
//     take two TMEM columns per value and keep u_2 of the five planes for
//     D1_z u_2 on the halo: 124 KiB, one CTA).  32 x 16 binary32 tiles (one
//     CTA per SM) keep a fourth full-record plane (the one that was the
//     centre one plane earlier): the next entering plane then overwrites a
//     slot nobody reads any more, so the barrier that ends each plane is not
//     needed;
//   * the arithmetic type T is double, float, dfloat (double-float, binary64
//     storage) or f32x2 (two columns per thread in packed FP32x2 instructions);
//   * the mixed second derivatives of the stress divergence (the D1_a o D1_b
//     reading of the mixed term), for each i sum_{j != i} d2 u_j/dx_i dx_j:
//     - binary64 and double-float, by linearity of D1_i,
//         = D1_i( s_i ),  s_i = sum_{j != i} D1_j u_j,
//       so only the three diagonal gradients D1_j u_j are needed around a
//       point: D1_x u0 and D1_y u1 are kept per plane, D1_z u2 is formed on
//       the centre plane's tile and halo (a third barrier per plane);
//     - binary32, with every x2 derivative applied last (D1_a and D1_b
//       commute on the periodic grid):
//         i = 0:  D1_x(D1_y u1) + D1_z(D1_x u2)
//         i = 1:  D1_y(D1_x u0) + D1_z(D1_y u2)
//         i = 2:  D1_z(D1_x u0 + D1_y u1)
//       so the halo helpers D1_y u1 and D1_x u0 are in-plane, formed as a
//       plane enters (three planes of helper buffers), and the x2 parts come
//       from the thread's own column (D1_x u2, D1_y u2 kept per plane in a
//       second TMEM window): no u_2 on the halo and two barriers per plane.
//
// Variables are stored as deviations from the reference state
// (rho' = rho - 1, rho u_i, (rho E)' = rho E - p_ref/(gamma-1)), which keeps
// binary32 storage free of the low-Mach cancellation in rho E; the residual
// is the same algebraic expression (the constant parts of rho E and p enter
// only through the reference enthalpy term -H0 div u).
#pragma once

#include <atomic>
#include <type_traits>

#include "dfloat.cuh"
#include "f32x2.cuh"
#include "fpconv.cuh"
#include "sbli_internal.cuh"

namespace sbli {

constexpr int TX = 32;  // tile width along x0 (one warp)
constexpr int HALO = 2;
constexpr int SX = TX + 2 * HALO;
constexpr int NSLOT = 5;

// primitive values of one point record in a ring slot; V_P holds 2 p' (the
// pressure enters Eqs. 2-3 only as 2 D_i p and 2 D_j(p u_j) in the combined
// skew form, so the factor 2 is applied once per point instead of once per
// stencil neighbour; scaling by 2 is exact)
enum { V_RHO, V_M0, V_M1, V_M2, V_E, V_U0, V_U1, V_U2, V_P, V_T, NV };
static_assert(V_U2 == V_U1 + 1 && V_U1 % 2 == 0, "u1, u2 form one 8-byte pair of a binary32 record");

// ZT (binary32 with the TMEM z queue): the x2 neighbours of a thread's own
// column come from tensor memory, so shared memory keeps full records only
// for the planes that are still to become the centre (entering, middle,
// centre: 3 slots), u_2 alone on the five ring planes (for D1_z u_2 on the
// halo), and no D1_x u0 / D1_y u1 ring.
template <int TY, bool ZT>
constexpr int full_slots() {
  return ZT ? (TY >= 16 ? 4 : 3) : NSLOT;
}
// Binary32 arithmetic types group the mixed second derivatives so that the
// x2 derivative is applied last (see fused_march): their helpers are
// in-plane and formed as each plane enters.
template <typename T>
constexpr bool mixz() {
  return std::is_same<T, float>::value || std::is_same<T, f32x2>::value;
}
template <typename T, int TY, bool ZT = false>
struct FusedSmem {
  static constexpr int SY = TY + 2 * HALO;
  static constexpr int NFULL = full_slots<TY, ZT>();
  static constexpr bool MIXZ = mixz<T>();
  static constexpr bool U2 = ZT && !MIXZ;      // u_2 ring (binary64 / double-float TMEM queue)
  static constexpr int NDV = MIXZ ? 4 : 2;     // per-plane gradients in the shared ring
  static constexpr int NSB = MIXZ ? 3 : 1;     // planes of helper buffers
  T ring[NFULL][SY][SX][NV];  // rho', m_i, E', u_i, p', T' per haloed point
  T u2ring[U2 ? NSLOT : 1][U2 ? SY : 1][U2 ? SX : 1];  // u_2 per haloed point of the five ring planes
  // without the TMEM queue: D1_x u0, D1_y u1 (and, binary32, D1_x u2, D1_y u2)
  // per plane (tile only)
  T dring[ZT ? 1 : NSLOT][ZT ? 1 : NDV][ZT ? 1 : TY][ZT ? 1 : TX];
  // binary64 / double-float: s_0 = D1_y u1 + D1_z u2 and s_1 = D1_x u0 + D1_z u2
  // on the centre plane; binary32: D1_y u1 and D1_x u0 of the last three
  // planes to enter (x0-haloed rows, x1-haloed columns)
  T s0buf[NSB][TY][SX];
  T s1buf[NSB][SY][TX];
  double red[2][32];          // block reduction of (ke, enstrophy)
  uint32_t tmem_base[2];      // TMEM allocations (z queue variant)
};

// 1/rho for the primitives (Eqs. 4-5): a Newton-refined approximation in
// binary64, a double-word reciprocal in double-float; binary32 takes the
// hardware approximation (rcp.approx, within one unit in the last place),
// far inside the binary32 tolerance and one instruction instead of the
// rounding-correction sequence.
__device__ __forceinline__ float rcp_approx_f32(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
template <typename T>
__device__ __forceinline__ T recip(T x);
// binary64: the hardware approximation (rcp.approx.ftz.f64) refined by two
// Newton-Raphson steps y <- y + y (1 - x y), each a pair of fused
// multiply-adds that squares the relative error (within one unit in the
// last place of 1/x; tests/test_gpu_recip.py compares it with CUDA's
// correctly rounded reciprocal)
template <>
__device__ __forceinline__ double recip<double>(double x) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  double e = fma(-x, y, 1.0);
  y = fma(y, e, y);
  e = fma(-x, y, 1.0);
  return fma(y, e, y);
}
template <>
__device__ __forceinline__ float recip<float>(float x) { return rcp_approx_f32(x); }
template <>
__device__ __forceinline__ dfloat recip<dfloat>(dfloat x) { return dw_reciprocal(x); }
template <>
__device__ __forceinline__ f32x2 recip<f32x2>(f32x2 x) { return f32x2(rcp_approx_f32(x.x), rcp_approx_f32(x.y)); }

// Record load/store with 8-byte (binary32: 40-byte records) or 16-byte
// (binary64: 80-byte records) vector accesses; both strides are bank-conflict
// free for the vector width used.
__device__ __forceinline__ void load_rec(const float* p, float (&r)[NV]) {
  const float2* q = reinterpret_cast<const float2*>(p);
#pragma unroll
  for (int i = 0; i < NV / 2; ++i) {
    const float2 t = q[i];
    r[2 * i] = t.x;
    r[2 * i + 1] = t.y;
  }
}
__device__ __forceinline__ void load_rec(const double* p, double (&r)[NV]) {
  const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
  for (int i = 0; i < NV / 2; ++i) {
    const double2 t = q[i];
    r[2 * i] = t.x;
    r[2 * i + 1] = t.y;
  }
}
__device__ __forceinline__ void store_rec(float* p, const float (&r)[NV]) {
  float2* q = reinterpret_cast<float2*>(p);
#pragma unroll
  for (int i = 0; i < NV / 2; ++i) q[i] = make_float2(r[2 * i], r[2 * i + 1]);
}
__device__ __forceinline__ void store_rec(double* p, const double (&r)[NV]) {
  double2* q = reinterpret_cast<double2*>(p);
#pragma unroll
  for (int i = 0; i < NV / 2; ++i) q[i] = make_double2(r[2 * i], r[2 * i + 1]);
}
// two-column binary32 records: 80 bytes, two values of both columns per 16-byte access
__device__ __forceinline__ void load_rec(const f32x2* p, f32x2 (&r)[NV]) {
  const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
  for (int i = 0; i < NV / 2; ++i) {
    const float4 v = q[i];
    r[2 * i] = f32x2(v.x, v.y);
    r[2 * i + 1] = f32x2(v.z, v.w);
  }
}
__device__ __forceinline__ void store_rec(f32x2* p, const f32x2 (&r)[NV]) {
  float4* q = reinterpret_cast<float4*>(p);
#pragma unroll
  for (int i = 0; i < NV / 2; ++i) q[i] = make_float4(r[2 * i].x, r[2 * i].y, r[2 * i + 1].x, r[2 * i + 1].y);
}
// double-float records: 80 bytes, two values per 16-byte access
__device__ __forceinline__ void load_rec(const dfloat* p, dfloat (&r)[NV]) {
  const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
  for (int i = 0; i < NV / 2; ++i) {
    const float4 v = q[i];
    r[2 * i] = dfloat(v.x, v.y);
    r[2 * i + 1] = dfloat(v.z, v.w);
  }
}
__device__ __forceinline__ void store_rec(dfloat* p, const dfloat (&r)[NV]) {
  float4* q = reinterpret_cast<float4*>(p);
#pragma unroll
  for (int i = 0; i < NV / 2; ++i) q[i] = make_float4(r[2 * i].hi, r[2 * i].lo, r[2 * i + 1].hi, r[2 * i + 1].lo);
}

// ---- tensor memory (TMEM) as a per-thread queue of x2-neighbour records.
// Each warp of the CTA owns the 32 TMEM lanes of its quarter (warp % 4) and a
// column window (warp / 4); a thread keeps its own column's records of the
// five ring planes there.  A value takes W 32-bit columns (binary32: 1;
// binary64 and double-float: 2): fields 0-7 of slot s in columns 8W s ..
// 8W s + 8W - 1, fields 8-9 from column 40W + 2W s, and the pair
// (D1_x u0, D1_y u1) from column 50W + 2W s, so every access is aligned to
// its own width; windows are 64 W columns.  32x32b shapes: each thread of
// the warp reads or writes its own lane.
template <typename T>
struct TmLayout {
  static constexpr int W = sizeof(T) / 4;      // 32-bit columns per value
  static constexpr int HEAD = 8 * W;           // columns of fields 0-7 of one slot
  static constexpr int TAIL = HEAD * NSLOT;    // fields 8-9 of slot s: columns TAIL + 2W s ...
  static constexpr int DIAG = TAIL + 2 * W * NSLOT;  // D1_x u0, D1_y u1 of slot s: DIAG + 2W s ...
  static constexpr int COLS = 64 * W;          // window width
  static_assert(NV == 10 && DIAG + 2 * W * NSLOT <= COLS, "z queue must fit the warp's TMEM window");
};

// columns a CTA of NW warps allocates: a power of two, at least 32
template <int NW, typename T = float>
constexpr int tmem_columns() {
  constexpr int need = TmLayout<T>::COLS * ((NW + 3) / 4);
  int c = 32;
  while (c < need) c *= 2;
  return c;
}
// The binary32 queue's second window (a separate allocation): the pair
// (D1_x u2, D1_y u2) of slot s in columns 2s, 2s + 1 of a 16-column window.
constexpr int TM_XCOLS = 16;
template <int NW, typename T = float>
constexpr int tmem_columns2() {
  if (!mixz<T>()) return 0;
  constexpr int need = TM_XCOLS * ((NW + 3) / 4);
  int c = 32;
  while (c < need) c *= 2;
  return c;
}

// win: this thread's window address (lane and window column), slot: ring slot
__device__ __forceinline__ void tmem_store_rec(uint32_t win, int slot, const float (&r)[NV]) {
  using L = TmLayout<float>;
  const uint32_t taddr = win + (uint32_t)(L::HEAD * slot), ttail = win + (uint32_t)(L::TAIL + 2 * slot);
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};\n\t"
      "tcgen05.st.sync.aligned.32x32b.x2.b32 [%9], {%10, %11};\n\t"
      "tcgen05.wait::st.sync.aligned;" ::"r"(taddr),
      "r"(__float_as_uint(r[0])), "r"(__float_as_uint(r[1])), "r"(__float_as_uint(r[2])), "r"(__float_as_uint(r[3])),
      "r"(__float_as_uint(r[4])), "r"(__float_as_uint(r[5])), "r"(__float_as_uint(r[6])), "r"(__float_as_uint(r[7])),
      "r"(ttail), "r"(__float_as_uint(r[8])), "r"(__float_as_uint(r[9]))
      : "memory");
}

__device__ __forceinline__ void tmem_load_rec(uint32_t win, int slot, float (&r)[NV]) {
  using L = TmLayout<float>;
  const uint32_t taddr = win + (uint32_t)(L::HEAD * slot), ttail = win + (uint32_t)(L::TAIL + 2 * slot);
  uint32_t v[NV];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%10];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%8, %9}, [%11];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9])
      : "r"(taddr), "r"(ttail)
      : "memory");
#pragma unroll
  for (int i = 0; i < NV; ++i) r[i] = __uint_as_float(v[i]);
}
// the pair (D1_x u0, D1_y u1) of this thread's column in slot `slot`
__device__ __forceinline__ void tmem_store_diag(uint32_t win, int slot, float d00, float d11) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1, %2};\n\t"
      "tcgen05.wait::st.sync.aligned;" ::"r"(win + (uint32_t)(TmLayout<float>::DIAG + 2 * slot)),
      "r"(__float_as_uint(d00)), "r"(__float_as_uint(d11))
      : "memory");
}
__device__ __forceinline__ void tmem_load_diag(uint32_t win, int slot, float& d00, float& d11) {
  uint32_t a, b;
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%2];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(a), "=r"(b)
      : "r"(win + (uint32_t)(TmLayout<float>::DIAG + 2 * slot))
      : "memory");
  d00 = __uint_as_float(a);
  d11 = __uint_as_float(b);
}

// 8-byte values as two 32-bit words: binary64 (low, high word), double-float (hi, lo)
__device__ __forceinline__ void to_words(double x, uint32_t& a, uint32_t& b) {
  a = (uint32_t)__double2loint(x);
  b = (uint32_t)__double2hiint(x);
}
__device__ __forceinline__ void from_words(uint32_t a, uint32_t b, double& x) {
  x = __hiloint2double((int)b, (int)a);
}
__device__ __forceinline__ void to_words(dfloat x, uint32_t& a, uint32_t& b) {
  a = __float_as_uint(x.hi);
  b = __float_as_uint(x.lo);
}
__device__ __forceinline__ void from_words(uint32_t a, uint32_t b, dfloat& x) {
  x.hi = __uint_as_float(a);
  x.lo = __uint_as_float(b);
}

template <typename T>
__device__ __forceinline__ void tmem_store_rec8(uint32_t win, int slot, const T (&r)[NV]) {
  using L = TmLayout<T>;
  const uint32_t taddr = win + (uint32_t)(L::HEAD * slot), ttail = win + (uint32_t)(L::TAIL + 4 * slot);
  uint32_t w[2 * NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) to_words(r[i], w[2 * i], w[2 * i + 1]);
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16};\n\t"
      "tcgen05.st.sync.aligned.32x32b.x4.b32 [%17], {%18, %19, %20, %21};\n\t"
      "tcgen05.wait::st.sync.aligned;" ::"r"(taddr),
      "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3]), "r"(w[4]), "r"(w[5]), "r"(w[6]), "r"(w[7]), "r"(w[8]), "r"(w[9]),
      "r"(w[10]), "r"(w[11]), "r"(w[12]), "r"(w[13]), "r"(w[14]), "r"(w[15]), "r"(ttail), "r"(w[16]), "r"(w[17]),
      "r"(w[18]), "r"(w[19])
      : "memory");
}
template <typename T>
__device__ __forceinline__ void tmem_load_rec8(uint32_t win, int slot, T (&r)[NV]) {
  using L = TmLayout<T>;
  const uint32_t taddr = win + (uint32_t)(L::HEAD * slot), ttail = win + (uint32_t)(L::TAIL + 4 * slot);
  uint32_t w[2 * NV];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%20];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%16, %17, %18, %19}, [%21];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]), "=r"(w[7]), "=r"(w[8]),
        "=r"(w[9]), "=r"(w[10]), "=r"(w[11]), "=r"(w[12]), "=r"(w[13]), "=r"(w[14]), "=r"(w[15]), "=r"(w[16]),
        "=r"(w[17]), "=r"(w[18]), "=r"(w[19])
      : "r"(taddr), "r"(ttail)
      : "memory");
#pragma unroll
  for (int i = 0; i < NV; ++i) from_words(w[2 * i], w[2 * i + 1], r[i]);
}
template <typename T>
__device__ __forceinline__ void tmem_store_diag8(uint32_t win, int slot, T d00, T d11) {
  uint32_t w[4];
  to_words(d00, w[0], w[1]);
  to_words(d11, w[2], w[3]);
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};\n\t"
      "tcgen05.wait::st.sync.aligned;" ::"r"(win + (uint32_t)(TmLayout<T>::DIAG + 4 * slot)),
      "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3])
      : "memory");
}
template <typename T>
__device__ __forceinline__ void tmem_load_diag8(uint32_t win, int slot, T& d00, T& d11) {
  uint32_t w[4];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3])
      : "r"(win + (uint32_t)(TmLayout<T>::DIAG + 4 * slot))
      : "memory");
  from_words(w[0], w[1], d00);
  from_words(w[2], w[3], d11);
}
__device__ __forceinline__ void tmem_store_rec(uint32_t win, int slot, const double (&r)[NV]) {
  tmem_store_rec8(win, slot, r);
}
__device__ __forceinline__ void tmem_load_rec(uint32_t win, int slot, double (&r)[NV]) { tmem_load_rec8(win, slot, r); }
__device__ __forceinline__ void tmem_store_rec(uint32_t win, int slot, const dfloat (&r)[NV]) {
  tmem_store_rec8(win, slot, r);
}
__device__ __forceinline__ void tmem_load_rec(uint32_t win, int slot, dfloat (&r)[NV]) { tmem_load_rec8(win, slot, r); }
__device__ __forceinline__ void tmem_store_diag(uint32_t win, int slot, double d00, double d11) {
  tmem_store_diag8(win, slot, d00, d11);
}
__device__ __forceinline__ void tmem_load_diag(uint32_t win, int slot, double& d00, double& d11) {
  tmem_load_diag8(win, slot, d00, d11);
}
__device__ __forceinline__ void tmem_store_diag(uint32_t win, int slot, dfloat d00, dfloat d11) {
  tmem_store_diag8(win, slot, d00, d11);
}
__device__ __forceinline__ void tmem_load_diag(uint32_t win, int slot, dfloat& d00, dfloat& d11) {
  tmem_load_diag8(win, slot, d00, d11);
}
// two columns per thread keep the shared-memory ring (no TMEM queue)
__device__ __forceinline__ void tmem_store_diag(uint32_t, int, f32x2, f32x2) {}
__device__ __forceinline__ void tmem_load_diag(uint32_t, int, f32x2&, f32x2&) {}
__device__ __forceinline__ void tmem_load_rec(uint32_t, int, f32x2 (&)[NV]) {}
__device__ __forceinline__ void tmem_store_rec(uint32_t, int, const f32x2 (&)[NV]) {}

// Allocate / release the CTA's TMEM columns (warp 0): NCOL for the queue
// and, binary32, NCOL2 for its second window, publishing the base addresses
// through shared memory.  The CTAs that shared memory lets share an SM never
// ask for more than the 512 columns available (binary32 32 x 8: 3 x (128 +
// 32); 32 x 16: 256 + 64; binary64 and double-float 32 x 8: 256, one CTA),
// so the allocation never waits.
template <int NCOL, int NCOL2 = 0>
__device__ __forceinline__ void tmem_acquire(uint32_t (&smem_slot)[2], uint32_t& base, uint32_t& base2) {
  if ((threadIdx.x >> 5) == 0) {
    const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&smem_slot[0]);
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst), "r"(NCOL) : "memory");
    if (NCOL2 > 0) {
      const uint32_t dst2 = (uint32_t)__cvta_generic_to_shared(&smem_slot[1]);
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst2), "r"(NCOL2)
                   : "memory");
    }
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  base = *(volatile uint32_t*)&smem_slot[0];
  base2 = NCOL2 > 0 ? *(volatile uint32_t*)&smem_slot[1] : 0u;
}

template <int NCOL, int NCOL2 = 0>
__device__ __forceinline__ void tmem_release(uint32_t base, uint32_t base2) {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if ((threadIdx.x >> 5) == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(base), "r"(NCOL) : "memory");
    if (NCOL2 > 0)
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(base2), "r"(NCOL2) : "memory");
  }
}

// This thread's TMEM window: lane quarter of its warp, column window warp / 4.
template <typename T>
__device__ __forceinline__ uint32_t tmem_window(uint32_t base) {
  const uint32_t w = threadIdx.x >> 5;
  return base + (((w & 3u) * 32u) << 16) + (w >> 2) * (uint32_t)TmLayout<T>::COLS;
}
__device__ __forceinline__ uint32_t tmem_window2(uint32_t base2) {
  const uint32_t w = threadIdx.x >> 5;
  return base2 + (((w & 3u) * 32u) << 16) + (w >> 2) * (uint32_t)TM_XCOLS;
}
// the pair (D1_x u2, D1_y u2) of this thread's column in slot `slot` of the
// second window
__device__ __forceinline__ void tmem_store_xdiag(uint32_t win2, int slot, float d02, float d12) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1, %2};\n\t"
      "tcgen05.wait::st.sync.aligned;" ::"r"(win2 + (uint32_t)(2 * slot)),
      "r"(__float_as_uint(d02)), "r"(__float_as_uint(d12))
      : "memory");
}
__device__ __forceinline__ void tmem_load_xdiag(uint32_t win2, int slot, float& d02, float& d12) {
  uint32_t a, b;
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%2];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(a), "=r"(b)
      : "r"(win2 + (uint32_t)(2 * slot))
      : "memory");
  d02 = __uint_as_float(a);
  d12 = __uint_as_float(b);
}

// Stage input value in the arithmetic type (binary64 inputs to a binary32
// stage are narrowed with integer re-packing, see fpconv.cuh).
template <typename T, typename TIN>
__device__ __forceinline__ T to_compute(TIN v) {
  return T(v);
}
template <>
__device__ __forceinline__ float to_compute<float, double>(double v) {
  return narrow_f64_fast(v);
}
// binary64 -> double-float: hi = RN32(v), lo = RN32(v - hi); the narrowings
// and the widening of hi are integer re-packings, the remainder one DADD
// (exact: v - hi has at most 29 significant bits)
template <>
__device__ __forceinline__ dfloat to_compute<dfloat, double>(double v) {
  float hi, lo;
  split_f64(v, hi, lo);
  return dfloat(hi, lo);
}

// A binary64 stage output in the stored type: itself, or (double-float
// stage fields) the same hi + lo split a binary64 input gets when it is
// loaded, so the consumer reads the pair it would have formed.
template <typename TOUT>
__device__ __forceinline__ TOUT to_output(double v) {
  return TOUT(v);
}
template <>
__device__ __forceinline__ dfloat to_output<dfloat>(double v) {
  return to_compute<dfloat, double>(v);
}

// a * b + c: left to the compiler's contraction for scalar types, an explicit
// packed FMA for f32x2 (whose operators are not contracted)
template <typename T>
__device__ __forceinline__ T mad(T a, T b, T c) {
  return a * b + c;
}
__device__ __forceinline__ f32x2 mad(f32x2 a, f32x2 b, f32x2 c) { return fma(a, b, c); }

// A stage value built from the stage input of each column a thread owns.
template <typename T, typename TIN>
__device__ __forceinline__ T from_lanes(const TIN (&v)[1]) {
  return to_compute<T, TIN>(v[0]);
}
template <typename T, typename TIN>
__device__ __forceinline__ T from_lanes(const TIN (&v)[2]) {
  return T(to_compute<float, TIN>(v[0]), to_compute<float, TIN>(v[1]));
}

// binary64-class arithmetic types (binary64 Runge-Kutta update in place)
template <typename T>
constexpr bool is_f64_class() {
  return std::is_same<T, double>::value || std::is_same<T, dfloat>::value;
}

// A stage value in binary64 for the Runge-Kutta update.
__device__ __forceinline__ double as_double(double x) { return x; }
__device__ __forceinline__ double as_double(float x) { return widen_f32_fast(x); }
__device__ __forceinline__ double as_double(dfloat x) { return widen_f32_fast(x.hi) + widen_f32_fast(x.lo); }

// Accumulated terms of the residual at one point.  By linearity of D1 and
// because the centre values u_j^c are constants over a stencil, the
// convective and skew terms of Eqs. 1-3 combine into single derivatives:
//   D_j(m_i u_j) + u_j^c D_j m_i       = D_j( m_i (u_j + u_j^c) )
//   D_j m_j + u_j^c D_j rho'            = D_j( m_j + u_j^c rho' )
//   D_j(E' u_j) + u_j^c D_j E'          = D_j( E' (u_j + u_j^c) )
template <typename T>
struct Terms {
  T g[3][3];   // g[i][j] = D1_j u_i
  T rrho;      // sum_j D_j(m_j + u_j^c rho')                     (Eq. 1 without rho div u)
  T rM[3];     // sum_j D_j(m_i (u_j + u_j^c)) + 2 D_i p'          (Eq. 2 without m_i div u)
  T rE;        // sum_j D_j(E' (u_j + u_j^c)) + 2 D_j(p' u_j)      (Eq. 3 without E' div u)
  T lap[3];    // sum_j D2_j u_i, off-centre part
  T lapT;      // sum_j D2_j T', off-centre part
  T G[3];      // sum_j d2 u_j / dx_i dx_j (Eq. 7 on j = i, D1 o D1 otherwise)
};

// All derivatives along axis A at one point.  ldrec(k, r) loads the record of
// the neighbour k = 0..3 (offsets -2, -1, +1, +2 along A); uc are the centre
// velocities; sfun(k, record) gives the mixed-term helper s_A at neighbour k.
template <int A, typename T, typename LD, typename SF>
__device__ __forceinline__ void axis_terms(const LD& ldrec, const SF& sfun, const Coef<T>& c, const T (&uc)[3],
                                           Terms<T>& t) {
  const T c1 = c.c1[A], c2 = c.c2[A], e0 = c.e0[A], e1 = c.e1[A], e2 = c.e2[A];
  const T nc2 = -c2;
  auto d1 = [&](T fm2, T fm1, T fp1, T fp2) { return mad(c1, fp1 - fm1, nc2 * (fp2 - fm2)); };

  T r[4][NV];
#pragma unroll
  for (int k = 0; k < 4; ++k) ldrec(k, r[k]);
  T s[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) s[k] = sfun(k, r[k]);
#define SBLI_D1(V) d1(r[0][V], r[1][V], r[2][V], r[3][V])
  const T ua = uc[A];
  // stencil weights times (u_A + u_A^c):  D1(f w) = f+1 W1 - f-1 V1 - f+2 W2 + f-2 V2
  const T W1 = c1 * (r[2][V_U0 + A] + ua), V1 = c1 * (r[1][V_U0 + A] + ua);
  const T W2 = c2 * (r[3][V_U0 + A] + ua), V2 = c2 * (r[0][V_U0 + A] + ua);
  const T nV1 = -V1, nW2 = -W2;
  auto d1w = [&](int V) { return mad(r[0][V], V2, mad(r[3][V], nW2, mad(r[1][V], nV1, r[2][V] * W1))); };
  // stencil weights times u_A:  D1(f u_A)
  const T X1 = c1 * r[2][V_U0 + A], Y1 = c1 * r[1][V_U0 + A];
  const T X2 = c2 * r[3][V_U0 + A], Y2 = c2 * r[0][V_U0 + A];
  const T mY1 = -Y1, mX2 = -X2;
#pragma unroll
  for (int i = 0; i < 3; ++i) t.rM[i] += d1w(V_M0 + i);
  t.rM[A] = t.rM[A] + SBLI_D1(V_P);  // D_A (2 p')
  t.rE += mad(r[0][V_P], Y2, mad(r[3][V_P], mX2, mad(r[1][V_P], mY1, r[2][V_P] * X1))) + d1w(V_E);
  t.rrho += d1(fma(ua, r[0][V_RHO], r[0][V_M0 + A]), fma(ua, r[1][V_RHO], r[1][V_M0 + A]),
               fma(ua, r[2][V_RHO], r[2][V_M0 + A]), fma(ua, r[3][V_RHO], r[3][V_M0 + A]));
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const T off = mad(e1, r[2][V_U0 + i] + r[1][V_U0 + i], e2 * (r[3][V_U0 + i] + r[0][V_U0 + i]));
    t.lap[i] += off;
    if (i == A) {
      t.G[A] = fma(e0, uc[A], off) + d1(s[0], s[1], s[2], s[3]);
    } else {
      t.g[i][A] = SBLI_D1(V_U0 + i);
    }
  }
  t.lapT += mad(e1, r[2][V_T] + r[1][V_T], e2 * (r[3][V_T] + r[0][V_T]));
#undef SBLI_D1
}

// The same terms with the four neighbours streamed through registers one at
// a time: each neighbour's record is folded into the accumulators with its
// stencil weights (Eq. 6: +c2, -c1, +c1, -c2; Eq. 7 off-centre: e2, e1, e1,
// e2 for offsets -2, -1, +1, +2), so only one record is live.  Fewer
// operations than the difference-first form for hardware FMA types; the
// double-float type keeps the difference-first form (its products cost more
// than its sums).
// a + b, never contracted with the product that formed b (so its rounding
// does not depend on how the compiler schedules that product)
__device__ __forceinline__ float add_nc(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ f32x2 add_nc(f32x2 a, f32x2 b) { return a + b; }
template <typename T>
__device__ __forceinline__ T add_nc(T a, T b) {
  return a + b;
}

// No x2-regrouped mixed terms (every axis but the binary32 x2 axis).
struct NoXTerms {
  template <typename T>
  __device__ void operator()(int, T&, T&) const {}
};

// ZX (binary32, A = 2): the mixed derivatives that involve x2 are taken with
// the x2 derivative last, D1_z(D1_x u2) and D1_z(D1_y u2) from xfun(k, ...)
// (the neighbours' in-plane gradients of u2), added to G_0 and G_1; the
// stream also forms D1_z u2 at the centre (g_22).
template <int A, bool ZX = false, typename T, typename LD, typename SF, typename XF = NoXTerms>
__device__ __forceinline__ void axis_terms_stream(const LD& ldrec, const SF& sfun, const Coef<T>& c,
                                                  const T (&uc)[3], Terms<T>& t, const XF& xfun = XF()) {
  static_assert(!ZX || A == 2, "x2-last mixed terms belong to the x2 axis");
  const T c1 = c.c1[A], c2 = c.c2[A], e1 = c.e1[A], e2 = c.e2[A];
  const T ua = uc[A];
  T gz0 = T(0), gz1 = T(0), g22 = T(0);  // ZX only
  T lAA = T(0);                       // sum_k e_k u_A,k: D2_A u_A without its centre term
  T gA = T(0);                        // sum_k c_k s_k = D1_A s_A
  T gI[3] = {T(0), T(0), T(0)};      // D1_A u_i, i != A
  // the per-axis products c u_A^c once, so that each neighbour's two
  // weights are one multiply and one fused multiply-add
  const T cu1 = c1 * ua, cu2 = c2 * ua;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const T cd = (k == 0) ? c2 : (k == 1) ? -c1 : (k == 2) ? c1 : -c2;
    const T ed = (k == 0 || k == 3) ? e2 : e1;
    const T cdu = (k == 0) ? cu2 : (k == 1) ? -cu1 : (k == 2) ? cu1 : -cu2;
    T r[NV];
    ldrec(k, r);
    const T sk = sfun(k, r);
    const T w = fma(cd, r[V_U0 + A], cdu);  // D1(f (u_A + u_A^c)) weight
    const T x = cd * r[V_U0 + A];          // D1(f u_A) weight (times 2 p' below)
#pragma unroll
    for (int i = 0; i < 3; ++i) t.rM[i] = mad(w, r[V_M0 + i], t.rM[i]);
    t.rM[A] = mad(cd, r[V_P], t.rM[A]);
    t.rE = mad(w, r[V_E], mad(x, r[V_P], t.rE));
    t.rrho = mad(cd, fma(ua, r[V_RHO], r[V_M0 + A]), t.rrho);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      if (i != A) {
        t.lap[i] = mad(ed, r[V_U0 + i], t.lap[i]);
        gI[i] = mad(cd, r[V_U0 + i], gI[i]);
      }
    }
    lAA = mad(ed, r[V_U0 + A], lAA);  // shared by the Laplacian of u_A and G_A
    gA = mad(cd, sk, gA);
    t.lapT = mad(ed, r[V_T], t.lapT);
    if constexpr (ZX) {
      T x02, x12;
      xfun(k, x02, x12);
      gz0 = mad(cd, x02, gz0);
      gz1 = mad(cd, x12, gz1);
      g22 = add_nc(g22, x);  // x = cd u_2 (above): an add the compiler may not contract
    }
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
    if (i != A) t.g[i][A] = gI[i];
  t.lap[A] += lAA;
  t.G[A] = fma(c.e0[A], uc[A], lAA + gA);  // D2_A u_A + D1_A s_A (Eq. 7 on j = A, D1 o D1 otherwise)
  if constexpr (ZX) {
    t.G[0] = t.G[0] + gz0;
    t.G[1] = t.G[1] + gz1;
    t.g[2][2] = g22;
  }
}

// Eqs. 1-3 at one point from the accumulated derivative terms and the
// centre values (deviation form: rho' = rho - 1, E' = rho E - (rho E)_ref).
template <typename T>
__device__ __forceinline__ void assemble_residual(const Terms<T>& t, T rho_p, const T (&mc)[3], T Ec, const T (&uc)[3],
                                                  T Tc, const Coef<T>& c, T (&R)[5]) {
  const T e0sum = c.e0[0] + c.e0[1] + c.e0[2];  // centre coefficient of the Laplacian
  const T div = t.g[0][0] + t.g[1][1] + t.g[2][2];
  const T rho = T(1) + rho_p;
  R[0] = T(-0.5) * mad(rho, div, t.rrho);
  T uvisc = T(0);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const T lap = fma(e0sum, uc[i], t.lap[i]);
    const T visc = mad(t.G[i], T(1.0 / 3.0), lap);  // Laplacian + G - (2/3) G
    uvisc = mad(uc[i], visc, uvisc);
    R[1 + i] = mad(c.inv_re, visc, T(-0.5) * mad(mc[i], div, t.rM[i]));
  }
  // viscous dissipation du_i/dx_j (du_i/dx_j + du_j/dx_i - 2/3 div delta_ij)
  const T a01 = t.g[0][1] + t.g[1][0], a02 = t.g[0][2] + t.g[2][0], a12 = t.g[1][2] + t.g[2][1];
  const T sq = mad(t.g[2][2], t.g[2][2], mad(t.g[1][1], t.g[1][1], t.g[0][0] * t.g[0][0]));
  const T diss = mad(T(2), sq, mad(a12, a12, mad(a02, a02, mad(a01, a01, T(-2.0 / 3.0) * div * div))));
  const T lapT = fma(e0sum, Tc, t.lapT);
  R[4] = mad(c.kappa, lapT, mad(c.inv_re, uvisc + diss, mad(-c.H0, div, T(-0.5) * mad(Ec, div, t.rE))));
}

template <int A, bool ZX = false, typename T, typename LD, typename SF, typename XF = NoXTerms>
__device__ __forceinline__ void axis_terms_any(const LD& ldrec, const SF& sfun, const Coef<T>& c, const T (&uc)[3],
                                               Terms<T>& t, const XF& xfun = XF()) {
  if constexpr (std::is_same<T, dfloat>::value) {
    static_assert(!ZX, "double-float keeps the s_i helpers");
    axis_terms<A>(ldrec, sfun, c, uc, t);
  } else {
    axis_terms_stream<A, ZX>(ldrec, sfun, c, uc, t, xfun);
  }
}

// TIN: type of the stage input in HBM; TOUT: type of the stage output.
// CTAs per SM the launch bounds plan for: shared memory allows two 32 x 8
// binary32 CTAs per SM with the 5-slot ring (113 KiB each) and three with
// the TMEM queue and 3-slot ring (59 KiB each, 80 registers); binary64 and
// double-float (194.5 KiB) and 32 x 16 tiles take one.
template <typename T, int TY, bool ZT = false>
constexpr int fused_min_blocks() {
  return (sizeof(T) == 4 && TY <= 8) ? (ZT ? 3 : 2) : 1;
}
// tile width in points: 32 columns per warp row, times the columns per thread
template <typename T>
constexpr int tile_width() {
  return TX * Lanes<T>::N;
}

// The z march of one CTA over the 32 x TY column tile (bx, by), output
// planes [zbeg, min(zend, n2)), for the grid and stage described by `a`.
// Adds the stage input's kinetic energy and enstrophy of the tile's points
// to ke_acc / ens_acc when WITH_KE.  Ends with a barrier, so the shared
// memory can be reused by the caller.
template <typename T, typename TIN, typename TOUT, int TY, bool RHS_ONLY, bool WITH_KE, bool DF = false,
          bool ZT = false>
__device__ __forceinline__ void fused_march(const StageArgs& a, const Coef<T>& c, int bx, int by, int zbeg, int zend_req,
                                            FusedSmem<T, TY, ZT>& sm, double& ke_acc, double& ens_acc,
                                            uint32_t tmem_base = 0, uint32_t tmem_base2 = 0) {
  using S = FusedSmem<T, TY, ZT>;
  constexpr bool MIXZ = S::MIXZ;
  constexpr int SY = S::SY;
  constexpr int NT = TX * TY;
  constexpr int PTS = SX * SY;
  constexpr int NHALO = PTS - NT;                  // haloed points outside the tile
  constexpr int LPT = 1 + (NHALO + NT - 1) / NT;   // own point + halo points per thread

  constexpr int PP = Lanes<T>::N;  // columns per thread: tx and tx + 32
  const int n0 = a.g.n0, n1 = a.g.n1, n2 = a.g.n2;
  const unsigned plane = (unsigned)n0 * (unsigned)n1;
  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;
  const int x0 = bx * (TX * PP), y0 = by * TY;
  const int zend = min(zend_req, n2);
  const int gy = y0 + ty;
  bool valid[PP];
  unsigned own[PP];
#pragma unroll
  for (int j = 0; j < PP; ++j) {
    const int gx = x0 + tx + TX * j;
    valid[j] = (gx < n0) && (gy < n1);
    own[j] = valid[j] ? (unsigned)gx + (unsigned)n0 * (unsigned)gy : 0u;
  }
  const bool valid_xy = valid[0];  // column tx (the second column is valid only if the first is)
  // per-field base pointers; offsets inside a field are 32-bit (P < 2^32)
  const TIN* qf[NF];
  const double* accf[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    qf[f] = static_cast<const TIN*>(a.q_in) + (long long)f * a.g.P;
    accf[f] = a.acc_in ? a.acc_in + (long long)f * a.g.P : nullptr;
  }

  // points this thread loads on every plane (periodic wrap): its own tile
  // point first, then at most LPT-1 points of the halo ring (the two rows
  // above and below the tile at full haloed width, then the two columns on
  // each side of the tile rows)
  int ld_off[LPT][PP], ld_s[LPT];
#pragma unroll
  for (int l = 0; l < LPT; ++l) {
    int sy = -1, sx = -1;
    if (l == 0) {
      sy = ty + HALO;
      sx = tx + HALO;
    } else {
      const int h = tid + (l - 1) * NT;
      if (h < 4 * SX) {
        const int r = h / SX;
        sy = (r < 2) ? r : TY + r;
        sx = h % SX;
      } else if (h < NHALO) {
        const int h2 = h - 4 * SX;
        const int k = h2 & 3;
        sy = HALO + (h2 >> 2);
        sx = (k < 2) ? k : TX + k;
      }
    }
    if (sy >= 0) {
#pragma unroll
      for (int j = 0; j < PP; ++j)
        ld_off[l][j] = wrapi(x0 - HALO + sx + TX * j, n0) + n0 * wrapi(y0 - HALO + sy, n1);
      ld_s[l] = sy * SX + sx;
    } else {
#pragma unroll
      for (int j = 0; j < PP; ++j) ld_off[l][j] = -1;
      ld_s[l] = 0;
    }
  }

  const int nplanes = zend - zbeg;
  const int nit = nplanes + 4;
  // the window address is warp-uniform; broadcasting lane 0's copy lets the
  // compiler keep it in a uniform register for the tcgen05 operands
  const uint32_t twin = ZT ? __shfl_sync(0xffffffffu, tmem_window<T>(tmem_base), 0) : 0u;
  const uint32_t twin2 = (ZT && MIXZ) ? __shfl_sync(0xffffffffu, tmem_window2(tmem_base2), 0) : 0u;
  T d22 = T(0);
  T g00c = T(0), g11c = T(0);  // D1_x u0, D1_y u1 at the centre point

  // halo tasks of phase 2b, fixed for the whole z march: s_0 on the x0-halo
  // columns (4*TY points) and s_1 on the x1-halo rows (4*TX points)
  constexpr int NHT = 4 * (TX + TY);
  constexpr int HPT = (NHT + NT - 1) / NT;  // tasks per thread
  int hk[HPT], hxy[HPT], hdst[HPT];         // kind (0 none, 1 s_0, 2 s_1), packed (hy, hx), buffer index
#pragma unroll
  for (int j = 0; j < HPT; ++j) {
    const int h = tid + j * NT;
    if (h < 4 * TY) {
      const int r = h >> 2, k = h & 3;
      const int hx = (k < 2) ? k : TX + k;  // 0, 1, TX+2, TX+3
      hk[j] = 1;
      hxy[j] = ((r + HALO) << 8) | hx;
      hdst[j] = r * SX + hx;
    } else if (h < NHT) {
      const int h2 = h - 4 * TY;
      const int col = h2 % TX, k = h2 / TX;
      const int hy = (k < 2) ? k : TY + k;
      hk[j] = 2;
      hxy[j] = (hy << 8) | (col + HALO);
      hdst[j] = hy * TX + col;
    } else {
      hk[j] = 0;
      hxy[j] = 0;
      hdst[j] = 0;
    }
  }
  // ring slots of planes e-4 .. e (e = entering plane), rotated each iteration
  int rs[NSLOT];
#pragma unroll
  for (int k = 0; k < NSLOT; ++k) rs[k] = (k + 1) % NSLOT;  // any permutation; warm-up fills all slots
  // full-record slots (ZT; otherwise the ring slots): planes e-2, e-1, e, and
  // e-3 in front of them when there are four
  constexpr int NFULL = S::NFULL;
  constexpr bool LAST_BARRIER = !ZT || NFULL < 4;  // the barrier that ends each plane
  int rf[ZT ? NFULL : 1];
#pragma unroll
  for (int k = 0; k < (ZT ? NFULL : 1); ++k) rf[k] = (k + 1) % (ZT ? NFULL : 1);
  // binary32 helper-buffer slots of planes e-2, e-1, e
  int rb[3] = {1, 2, 0};

  TIN pf[LPT][NF][PP];
  int zl = wrapi(zbeg - HALO, n2);  // next plane to load (periodic), advanced one plane per load
  auto issue_loads = [&]() {
    const unsigned zoff = (unsigned)zl * plane;
    zl = (zl + 1 == n2) ? 0 : zl + 1;
#pragma unroll
    for (int l = 0; l < LPT; ++l) {
      if (l == 0 || ld_off[l][0] >= 0) {  // the own point always exists
#pragma unroll
        for (int j = 0; j < PP; ++j) {
          const unsigned o = zoff + (unsigned)ld_off[l][j];
#pragma unroll
          for (int f = 0; f < NF; ++f) pf[l][f][j] = qf[f][o];
        }
      }
    }
  };
  issue_loads();

  for (int it = 0; it < nit; ++it) {
    // ---------------------------------------------------------------- phase 1
    // plane e = zbeg - 2 + it enters slot it % 5: derive primitives (Eqs. 4-5
    // in deviation form) on the haloed tile from the prefetched Q'.
    {
      const int t0 = rs[0];
#pragma unroll
      for (int k = 0; k < NSLOT - 1; ++k) rs[k] = rs[k + 1];
      rs[NSLOT - 1] = t0;
    }
    const int se = rs[NSLOT - 1];
    if constexpr (ZT) {
      const int t0 = rf[0];
#pragma unroll
      for (int k = 0; k < NFULL - 1; ++k) rf[k] = rf[k + 1];
      rf[NFULL - 1] = t0;
    }
    const int fe = ZT ? rf[ZT ? NFULL - 1 : 0] : se;  // full-record slot of the entering plane
    if constexpr (MIXZ) {
      const int t0 = rb[0];
      rb[0] = rb[1];
      rb[1] = rb[2];
      rb[2] = t0;
    }
    {
      T* ring = &sm.ring[fe][0][0][0];
#pragma unroll
      for (int l = 0; l < LPT; ++l) {
        if (l == 0 || ld_off[l][0] >= 0) {  // the own point is always loaded
          T rec[NV];
          const T rho_p = from_lanes<T, TIN>(pf[l][0]);
          const T m0 = from_lanes<T, TIN>(pf[l][1]);
          const T m1 = from_lanes<T, TIN>(pf[l][2]);
          const T m2 = from_lanes<T, TIN>(pf[l][3]);
          const T E_p = from_lanes<T, TIN>(pf[l][4]);
          const T rinv = recip<T>(T(1) + rho_p);
          const T u0 = m0 * rinv, u1 = m1 * rinv, u2 = m2 * rinv;
          const T mu = mad(m2, u2, mad(m1, u1, m0 * u0));
          const T p2 = c.gm1x2 * mad(T(-0.5), mu, E_p);  // Eq. 4: 2 (p - p_ref)
          const T T_p = mad(c.hgM2, p2, -rho_p) * rinv;  // Eq. 5: T - 1
          rec[V_RHO] = rho_p;
          rec[V_M0] = m0;
          rec[V_M1] = m1;
          rec[V_M2] = m2;
          rec[V_E] = E_p;
          rec[V_U0] = u0;
          rec[V_U1] = u1;
          rec[V_U2] = u2;
          rec[V_P] = p2;
          rec[V_T] = T_p;
          store_rec(ring + ld_s[l] * NV, rec);
          if constexpr (S::U2) (&sm.u2ring[se][0][0])[ld_s[l]] = u2;
          if constexpr (ZT) {
            if (l == 0) tmem_store_rec(twin, se, rec);  // l == 0: every thread
          }
        }
      }
    }
    if (it + 1 < nit) issue_loads();
    __syncthreads();
    // --------------------------------------------------------------- phase 2a
    // in-plane diagonal gradients of the entering plane, kept for s_2 and
    // for the velocity gradient when the plane is the centre.
    {
      const T(*R)[SX][NV] = sm.ring[fe];
      const int sy = ty + HALO, sx = tx + HALO;
      const T d00 = mad(c.c1[0], R[sy][sx + 1][V_U0] - R[sy][sx - 1][V_U0],
                        -c.c2[0] * (R[sy][sx + 2][V_U0] - R[sy][sx - 2][V_U0]));
      // u1 and u2 of the x1 neighbours (adjacent fields: one 8-byte load each
      // in binary32, whose records sit at 8-byte multiples)
      T y1[4], y2[4];
      {
        const int oy[4] = {-2, -1, 1, 2};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          if constexpr (std::is_same<T, float>::value && MIXZ) {
            const float2 v = *reinterpret_cast<const float2*>(&R[sy + oy[k]][sx][V_U1]);
            y1[k] = v.x;
            y2[k] = v.y;
          } else {
            y1[k] = R[sy + oy[k]][sx][V_U1];
            y2[k] = R[sy + oy[k]][sx][V_U2];
          }
        }
      }
      const T d11 = mad(c.c1[1], y1[2] - y1[1], -c.c2[1] * (y1[3] - y1[0]));
      if constexpr (ZT) {
        tmem_store_diag(twin, se, d00, d11);  // this thread's column only
      } else {
        sm.dring[se][0][ty][tx] = d00;
        sm.dring[se][1][ty][tx] = d11;
      }
      if constexpr (MIXZ) {
        // binary32: the in-plane gradients of u2 (for D1_z of them at the
        // centre, from this thread's own column) and the helpers D1_y u1 on
        // the x0-haloed rows and D1_x u0 on the x1-haloed columns of the
        // entering plane, read when it becomes the centre
        const T d02 = mad(c.c1[0], R[sy][sx + 1][V_U2] - R[sy][sx - 1][V_U2],
                          -c.c2[0] * (R[sy][sx + 2][V_U2] - R[sy][sx - 2][V_U2]));
        const T d12 = mad(c.c1[1], y2[2] - y2[1], -c.c2[1] * (y2[3] - y2[0]));
        if constexpr (ZT) {
          tmem_store_xdiag(twin2, se, d02, d12);
        } else {
          sm.dring[se][2][ty][tx] = d02;
          sm.dring[se][3][ty][tx] = d12;
        }
        const int sbe = rb[2];
        sm.s0buf[sbe][ty][sx] = d11;
        sm.s1buf[sbe][sy][tx] = d00;
#pragma unroll
        for (int j = 0; j < HPT; ++j) {
          const int hy = hxy[j] >> 8, hx = hxy[j] & 0xFF;
          if (hk[j] == 1) {
            (&sm.s0buf[sbe][0][0])[hdst[j]] = mad(c.c1[1], R[hy + 1][hx][V_U1] - R[hy - 1][hx][V_U1],
                                                  -c.c2[1] * (R[hy + 2][hx][V_U1] - R[hy - 2][hx][V_U1]));
          } else if (hk[j] == 2) {
            (&sm.s1buf[sbe][0][0])[hdst[j]] = mad(c.c1[0], R[hy][hx + 1][V_U0] - R[hy][hx - 1][V_U0],
                                                  -c.c2[0] * (R[hy][hx + 2][V_U0] - R[hy][hx - 2][V_U0]));
          }
        }
      }
    }
    if (it < 4) continue;  // ring not yet full; slots written so far are not read again before the next sync

    const int zc = zbeg + it - 4;  // centre plane
    // slot of plane zc + o, o = -2..2
    const int sl[5] = {rs[0], rs[1], rs[2], rs[3], rs[4]};
    const int scen = sl[2];
    const int fc = ZT ? rf[ZT ? NFULL - 3 : 0] : scen;  // full-record slot of the centre plane
    unsigned oc[PP];  // offsets of the thread's centre points
#pragma unroll
    for (int j = 0; j < PP; ++j) oc[j] = (unsigned)zc * plane + own[j];

    // accumulator of the centre points (fetched as phase 3 starts, so that
    // its latency overlaps the derivative terms)
    double accv[NF][PP];
    float dhi[NF][PP], dlo[NF][PP];  // double-float accumulator (DF mode)
    auto fetch_acc = [&]() {
      if (!RHS_ONLY) {
#pragma unroll
        for (int j = 0; j < PP; ++j) {
          if (!valid[j]) continue;
          if (DF) {
#pragma unroll
            for (int f = 0; f < NF; ++f) {
              dhi[f][j] = a.dacc_in[(long long)f * a.g.P + oc[j]];
              dlo[f][j] = a.dacc_in[(long long)(NF + f) * a.g.P + oc[j]];
            }
          } else {
#pragma unroll
            for (int f = 0; f < NF; ++f) accv[f][j] = accf[f][oc[j]];
          }
        }
      }
    };

    // --------------------------------------------------------------- phase 2b
    // binary64 / double-float: s_0 and s_1 on the centre plane's tile and
    // halo; binary32 has its helpers already (phase 2a of the plane's entry)
    // and needs only the centre's in-plane gradients.
    if constexpr (MIXZ) {
      if constexpr (ZT) {
        tmem_load_diag(twin, scen, g00c, g11c);
      } else {
        g00c = sm.dring[scen][0][ty][tx];
        g11c = sm.dring[scen][1][ty][tx];
      }
    } else {
      const int sy = ty + HALO, sx = tx + HALO;
      auto u2at = [&](int slot, int yy, int xx) {
        if constexpr (ZT)
          return sm.u2ring[slot][yy][xx];
        else
          return sm.ring[slot][yy][xx][V_U2];
      };
      auto u2z = [&](int yy, int xx) {
        return mad(c.c1[2], u2at(sl[3], yy, xx) - u2at(sl[1], yy, xx),
                   -c.c2[2] * (u2at(sl[4], yy, xx) - u2at(sl[0], yy, xx)));
      };
      d22 = u2z(sy, sx);
      if constexpr (ZT) {
        tmem_load_diag(twin, scen, g00c, g11c);
      } else {
        g00c = sm.dring[scen][0][ty][tx];
        g11c = sm.dring[scen][1][ty][tx];
      }
      sm.s0buf[0][ty][sx] = g11c + d22;
      sm.s1buf[0][sy][tx] = g00c + d22;
      const T(*R)[SX][NV] = sm.ring[fc];
#pragma unroll
      for (int j = 0; j < HPT; ++j) {
        const int hy = hxy[j] >> 8, hx = hxy[j] & 0xFF;
        if (hk[j] == 1) {
          const T d11 = mad(c.c1[1], R[hy + 1][hx][V_U1] - R[hy - 1][hx][V_U1],
                            -c.c2[1] * (R[hy + 2][hx][V_U1] - R[hy - 2][hx][V_U1]));
          (&sm.s0buf[0][0][0])[hdst[j]] = d11 + u2z(hy, hx);
        } else if (hk[j] == 2) {
          const T d00 = mad(c.c1[0], R[hy][hx + 1][V_U0] - R[hy][hx - 1][V_U0],
                            -c.c2[0] * (R[hy][hx + 2][V_U0] - R[hy][hx - 2][V_U0]));
          (&sm.s1buf[0][0][0])[hdst[j]] = d00 + u2z(hy, hx);
        }
      }
      __syncthreads();
    }
    // ---------------------------------------------------------------- phase 3
    {
      fetch_acc();
      const int sy = ty + HALO, sx = tx + HALO;
      const T(*C)[SX][NV] = sm.ring[fc];
      T cen[NV];
      if constexpr (ZT)
        tmem_load_rec(twin, scen, cen);
      else
        load_rec(&C[sy][sx][0], cen);
      const T rho_p = cen[V_RHO];
      const T mc[3] = {cen[V_M0], cen[V_M1], cen[V_M2]};
      const T Ec = cen[V_E];
      const T uc[3] = {cen[V_U0], cen[V_U1], cen[V_U2]};
      const T Tc = cen[V_T];

      Terms<T> t;
      t.rrho = t.rE = t.lapT = T(0);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        t.rM[i] = T(0);
        t.lap[i] = T(0);
      }
      t.g[0][0] = g00c;
      t.g[1][1] = g11c;
      t.g[2][2] = d22;

      // x0 group first (SN2 ordering), then x1, x2
      const int sbc = MIXZ ? rb[0] : 0;  // helper buffers of the centre plane
      {
        const int off[4] = {-2, -1, 1, 2};
        auto ld = [&](int k, T(&r)[NV]) { load_rec(&C[sy][sx + off[k]][0], r); };
        auto sf = [&](int k, const T(&)[NV]) { return sm.s0buf[sbc][ty][sx + off[k]]; };
        axis_terms_any<0>(ld, sf, c, uc, t);
      }
      {
        const int off[4] = {-2, -1, 1, 2};
        auto ld = [&](int k, T(&r)[NV]) { load_rec(&C[sy + off[k]][sx][0], r); };
        auto sf = [&](int k, const T(&)[NV]) { return sm.s1buf[sbc][sy + off[k]][tx]; };
        axis_terms_any<1>(ld, sf, c, uc, t);
      }
      {
        const int zs[4] = {sl[0], sl[1], sl[3], sl[4]};
        auto ld = [&](int k, T(&r)[NV]) {
          if constexpr (ZT)
            tmem_load_rec(twin, zs[k], r);
          else
            load_rec(&sm.ring[zs[k]][sy][sx][0], r);
        };
        auto sf = [&](int k, const T(&)[NV]) {
          if constexpr (ZT) {
            T a, b;
            tmem_load_diag(twin, zs[k], a, b);
            return a + b;
          } else {
            return sm.dring[zs[k]][0][ty][tx] + sm.dring[zs[k]][1][ty][tx];
          }
        };
        // binary32: D1_x u2 and D1_y u2 of the x2 neighbours
        auto xf = [&](int k, T& d02, T& d12) {
          if constexpr (MIXZ) {
            if constexpr (ZT) {
              tmem_load_xdiag(twin2, zs[k], d02, d12);
            } else {
              d02 = sm.dring[zs[k]][2][ty][tx];
              d12 = sm.dring[zs[k]][3][ty][tx];
            }
          }
        };
        axis_terms_any<2, MIXZ>(ld, sf, c, uc, t, xf);
      }

      const T rho = T(1) + rho_p;
      T R[5];
      assemble_residual(t, rho_p, mc, Ec, uc, Tc, c, R);

#pragma unroll
      for (int j = 0; j < PP; ++j) {
        if (!valid[j]) continue;
        const unsigned o = oc[j];
        TOUT qo[NF];
        if constexpr (RHS_ONLY) {
#pragma unroll
          for (int f = 0; f < NF; ++f) a.r_out[(long long)f * a.g.P + o] = double(lane(R[f], j));
        } else if constexpr (DF) {
          // binary32 stage, double-float accumulator (hi + lo, binary32
          // each): acc' = acc + (b dt R) by Dekker's Fast2Sum of hi and the
          // increment x = fl(b dt R), the error folded into lo; Q_{k+1} = hi'
          // + (lo' + (a - b) dt R).  Fast2Sum is exact when |hi| >= |x|;
          // otherwise (hi crossing zero) the pair misses hi + x by at most
          // about half an ulp of x, the size of the rounding x already
          // carries, so the accumulator keeps its precision where it
          // matters.  The pair (hi', lo') represents acc' whether or not it
          // is normalised; the last stage of a step renormalises it, so that
          // the state's hi fields are its binary32 rounding (the next step's
          // stage-0 input), the others leave it as it is.
          // Fields are updated two at a time with packed two-lane
          // instructions (the same correctly rounded binary32 operations as
          // one field at a time), the last field alone.
          const float bdt = a.b_dt32, ambdt = a.amb_dt32;
          float hi3[NF], lo3[NF], rr[NF];
#pragma unroll
          for (int f = 0; f < NF; ++f) rr[f] = float(lane(R[f], j));
          const float2 bdt2 = make_float2(bdt, bdt), ambdt2 = make_float2(ambdt, ambdt);
#pragma unroll
          for (int f = 0; f < NF; f += 2) {
            if (f + 1 < NF) {
              const float2 r2 = make_float2(rr[f], rr[f + 1]);
              const float2 h2 = make_float2(dhi[f][j], dhi[f + 1][j]);
              const float2 x2 = __fmul2_rn(bdt2, r2);
              const float2 s2 = __fadd2_rn(h2, x2);
              const float2 d2 = __fadd2_rn(s2, make_float2(-h2.x, -h2.y));
              const float2 e2 = __fadd2_rn(x2, make_float2(-d2.x, -d2.y));
              float2 l2 = __fadd2_rn(make_float2(dlo[f][j], dlo[f + 1][j]), e2);
              float2 hn = s2;
              if (a.df_normalize) {
                hn = __fadd2_rn(s2, l2);
                const float2 g2 = __fadd2_rn(hn, make_float2(-s2.x, -s2.y));
                l2 = __fadd2_rn(l2, make_float2(-g2.x, -g2.y));
              }
              const float2 q2 = __fadd2_rn(hn, __ffma2_rn(ambdt2, r2, l2));
              hi3[f] = hn.x;
              hi3[f + 1] = hn.y;
              lo3[f] = l2.x;
              lo3[f + 1] = l2.y;
              qo[f] = TOUT(q2.x);
              qo[f + 1] = TOUT(q2.y);
            } else {
              const float x = bdt * rr[f];
              const float s = __fadd_rn(dhi[f][j], x);
              const float err = __fsub_rn(x, __fsub_rn(s, dhi[f][j]));
              float h = s, l = __fadd_rn(dlo[f][j], err);
              if (a.df_normalize) {
                h = __fadd_rn(s, l);
                l = __fsub_rn(l, __fsub_rn(h, s));
              }
              hi3[f] = h;
              lo3[f] = l;
              qo[f] = TOUT(h + fmaf(ambdt, rr[f], l));
            }
          }
#pragma unroll
          for (int f = 0; f < NF; ++f) {
            a.dacc_out[(long long)f * a.g.P + o] = hi3[f];
            a.dacc_out[(long long)(NF + f) * a.g.P + o] = lo3[f];
          }
        } else if constexpr (is_f64_class<T>()) {
          // binary64 (or double-float) stage: acc + b dt R and acc + a dt R,
          // binary64 fused multiply-adds
#pragma unroll
          for (int f = 0; f < NF; ++f) {
            const double r = as_double(R[f]);
            a.acc_out[(long long)f * a.g.P + o] = fma(a.b_dt, r, accv[f][j]);
            qo[f] = to_output<TOUT>(fma(a.a_dt, r, accv[f][j]));
          }
        } else {
          // binary32 stage, binary64 accumulator: one DADD per field,
          //   acc' = acc + (b dt R),  Q_{k+1} = float(acc') + (a - b) dt R
          // (conversions by integer re-packing, fpconv.cuh; the narrowing
          // rounds to nearest, ties away from zero)
          const float bdt = a.b_dt32, ambdt = a.amb_dt32;
#pragma unroll
          for (int f = 0; f < NF; ++f) {
            const float r = float(lane(R[f], j));
            const double accn = accv[f][j] + widen_f32_fast(bdt * r);
            a.acc_out[(long long)f * a.g.P + o] = accn;
            qo[f] = TOUT(narrow_f64_rna(accn) + ambdt * r);
          }
        }
        if constexpr (!RHS_ONLY) {
          if (a.q_out) {  // the stage field (absent on the last stage)
#pragma unroll
            for (int f = 0; f < NF; ++f) static_cast<TOUT*>(a.q_out)[(long long)f * a.g.P + o] = qo[f];
          }
        }
        if (WITH_KE) {
          const T w0 = t.g[2][1] - t.g[1][2], w1 = t.g[0][2] - t.g[2][0], w2 = t.g[1][0] - t.g[0][1];
          const T ke_t = T(0.5) * (mc[0] * uc[0] + mc[1] * uc[1] + mc[2] * uc[2]);
          const T ens_t = T(0.5) * rho * (w0 * w0 + w1 * w1 + w2 * w2);
          ke_acc += double(lane(ke_t, j));
          ens_acc += double(lane(ens_t, j));
        }
      }
    }
    // with four full-record slots the next plane writes the slot of plane
    // e-3, last read before this plane's first barrier
    if constexpr (LAST_BARRIER) __syncthreads();
  }
  if constexpr (!LAST_BARRIER) __syncthreads();  // the caller may reuse shared memory
}

// Fixed-order block reduction of (ke, ens) into out[0..1]: warp shuffles,
// then thread 0 over the warps.
template <int NT>
__device__ __forceinline__ void block_reduce_pair(double (&red)[2][32], double ke, double ens, double* out) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ke += __shfl_down_sync(0xffffffffu, ke, o);
    ens += __shfl_down_sync(0xffffffffu, ens, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = ke;
    red[1][threadIdx.x >> 5] = ens;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double k = 0.0, e = 0.0;
    for (int w = 0; w < NT / 32; ++w) {
      k += red[0][w];
      e += red[1][w];
    }
    out[0] = k;
    out[1] = e;
  }
  __syncthreads();
}

// Single grid: one CTA per (tile, z chunk).  ZT: x2-neighbour records in TMEM.
template <typename T, typename TIN, typename TOUT, int TY, bool RHS_ONLY, bool WITH_KE, bool DF = false,
          bool ZT = false>
__global__ void __launch_bounds__(TX* TY, fused_min_blocks<T, TY, ZT>())
    fused_stage_kernel(const StageArgs a, const Coef<T> c) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  FusedSmem<T, TY, ZT>& sm = *reinterpret_cast<FusedSmem<T, TY, ZT>*>(smem_raw);
  constexpr int NCOL = tmem_columns<TY, T>();  // TX*TY/32 = TY warps
  constexpr int NCOL2 = tmem_columns2<TY, T>();
  uint32_t tbase = 0, tbase2 = 0;
  if (ZT) tmem_acquire<NCOL, NCOL2>(sm.tmem_base, tbase, tbase2);
  double ke = 0.0, ens = 0.0;
  const int zbeg = blockIdx.z * a.zc;
  fused_march<T, TIN, TOUT, TY, RHS_ONLY, WITH_KE, DF, ZT>(a, c, blockIdx.x, blockIdx.y, zbeg, zbeg + a.zc, sm, ke,
                                                          ens, tbase, tbase2);
  if (WITH_KE) {
    const long long b = blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
    block_reduce_pair<TX * TY>(sm.red, ke, ens, a.ke_partials + 2 * b);
  }
  if (ZT) tmem_release<NCOL, NCOL2>(tbase, tbase2);
}

template <int TY, int W = TX>
inline dim3 fused_grid(const Geom& g, int zc) {
  return dim3((g.n0 + W - 1) / W, (g.n1 + TY - 1) / TY, (g.n2 + zc - 1) / zc);
}

// The dynamic shared-memory limit is a per-device attribute of a kernel: set
// it on the current device the first time a kernel launches there (bit d of
// `done`).  Concurrent first launches may both set it, which is harmless.
template <typename K>
cudaError_t ensure_smem_limit(K kernel, size_t bytes, std::atomic<unsigned long long>& done) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = dev < 64 ? (1ull << dev) : 0ull;
  if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_acq_rel);
  return e;
}

template <typename T, typename TIN, typename TOUT, int TY, bool RHS_ONLY, bool WITH_KE, bool DF = false,
          bool ZT = false>
cudaError_t launch_fused_t(const StageArgs& a, const Coef<T>& c, cudaStream_t s) {
  auto k = fused_stage_kernel<T, TIN, TOUT, TY, RHS_ONLY, WITH_KE, DF, ZT>;
  const size_t smem = sizeof(FusedSmem<T, TY, ZT>);
  static std::atomic<unsigned long long> done{0};  // devices this instantiation is configured on
  if (cudaError_t e = ensure_smem_limit(k, smem, done)) return e;
  k<<<fused_grid<TY, tile_width<T>()>(a.g, a.zc), TX * TY, smem, s>>>(a, c);
  return cudaGetLastError();
}

}  // namespace sbli
