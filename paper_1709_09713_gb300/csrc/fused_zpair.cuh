// fused_zpair.cuh -- binary32 fused residual + RK stage (arXiv:1709.09713,
// Eqs. 1-8, §2.2 Fig. 1) with two x2 planes per thread.
//
// Same method and data layout as fused_march (fused_stage.cuh): a CTA owns a
// 32 x 8 column tile and marches along x2; one thread per column.  Here a
// thread advances two consecutive planes (z, z+1) of its column at once and
// carries their values as the two lanes of one packed FP32x2 value (f32x2),
// so every arithmetic instruction, every shared-memory access and all the
// per-plane bookkeeping (ring rotation, barriers, addresses) serve two
// points:
//   * shared memory keeps "pair records": the 10 primitives of a haloed
//     point for planes z and z+1 side by side (80 bytes, 16-byte accesses
//     move two values of both planes), for two plane pairs -- the entering
//     pair and the centre pair -- plus u_2 pairs of three plane pairs (the
//     six planes z-2 .. z+3 that D1_z u_2 needs on the halo);
//   * the x2 neighbours of a column come from tensor memory (TMEM), where
//     each thread keeps its own column's pair records: "aligned" pairs
//     (z, z+1) of the last three entering pairs and "shifted" pairs
//     (z-1, z) of the last two, so that every x2 neighbour pair of the
//     centre pair (zc+o, zc+1+o), o = -2, -1, +1, +2, is one contiguous
//     TMEM load: aligned for o = -2, +2, shifted for o = -1, +1;
//   * per entering pair: primitives (Eqs. 4-5) on the haloed tile,
//     D1_x u0 and D1_y u1 at the own column, the mixed-term helpers s_0, s_1
//     on the centre pair's halo, then all derivatives (Eqs. 6-7), the
//     residual (Eqs. 1-3) and the RK update of both centre planes.
// Each lane performs exactly the binary32 operations of the one-plane
// kernel's explicit FMA form (packed instructions round each lane
// correctly), so results agree with it within binary32 rounding.
#pragma once

#include "fused_stage.cuh"

namespace sbli {
namespace zp {

constexpr int TY = 8;
constexpr int SY = TY + 2 * HALO;
constexpr int NT = TX * TY;  // 256 threads, 8 warps

struct Smem {
  f32x2 ring[2][SY][SX][NV];  // pair records of the entering and the centre plane pair
  f32x2 u2ring[3][SY][SX];    // u_2 pairs of the last three entering plane pairs
  f32x2 s0buf[TY][SX];        // s_0 = D1_y u1 + D1_z u2, centre pair, x0-haloed rows
  f32x2 s1buf[SY][TX];        // s_1 = D1_x u0 + D1_z u2, centre pair, x1-haloed columns
  double red[2][32];
  uint32_t tmem_base;
};

// TMEM columns of one thread's window (32-bit columns; every access is
// aligned to its own width).  Aligned slots s = 0..2 (entering pair j at
// slot j % 3), shifted and diagonal slots s = 0..1 (slot j % 2).
//   AREC  fields 0-7 of an aligned pair record, interleaved (f(z), f(z+1))
//   SREC  the same for a shifted pair (f(z-1), f(z))
//   ATAIL, STAIL  fields 8-9 of those records
//   DIAG  (D1_x u0, D1_y u1) of the aligned pair, both lanes
//   SA, SS  s_2 = D1_x u0 + D1_y u1 of the aligned and the shifted pair
struct Tm {
  static constexpr uint32_t AREC = 0, SREC = 48, ATAIL = 80, STAIL = 92, DIAG = 100, SA = 108, SS = 114;
  static constexpr int COLS = 128;  // window width; 118 used
};
constexpr int NCOL = 2 * Tm::COLS;  // 8 warps: two lane-quarter windows -> 256 columns per CTA

__device__ __forceinline__ uint32_t u32(float x) { return __float_as_uint(x); }
__device__ __forceinline__ float f32(uint32_t x) { return __uint_as_float(x); }

// pair record (20 words, interleaved) to / from TMEM
__device__ __forceinline__ void tm_store_rec(uint32_t a16, uint32_t a4, const f32x2 (&r)[NV]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16};\n\t"
      "tcgen05.st.sync.aligned.32x32b.x4.b32 [%17], {%18, %19, %20, %21};\n\t"
      "tcgen05.wait::st.sync.aligned;" ::"r"(a16),
      "r"(u32(r[0].x)), "r"(u32(r[0].y)), "r"(u32(r[1].x)), "r"(u32(r[1].y)), "r"(u32(r[2].x)), "r"(u32(r[2].y)),
      "r"(u32(r[3].x)), "r"(u32(r[3].y)), "r"(u32(r[4].x)), "r"(u32(r[4].y)), "r"(u32(r[5].x)), "r"(u32(r[5].y)),
      "r"(u32(r[6].x)), "r"(u32(r[6].y)), "r"(u32(r[7].x)), "r"(u32(r[7].y)), "r"(a4), "r"(u32(r[8].x)),
      "r"(u32(r[8].y)), "r"(u32(r[9].x)), "r"(u32(r[9].y))
      : "memory");
}
// shifted pair (lane 0 = lane 1 of the previous aligned pair, lane 1 = lane 0 of the new one)
__device__ __forceinline__ void tm_store_shifted(uint32_t a16, uint32_t a4, const f32x2 (&prev)[NV],
                                                 const f32x2 (&cur)[NV]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16};\n\t"
      "tcgen05.st.sync.aligned.32x32b.x4.b32 [%17], {%18, %19, %20, %21};\n\t"
      "tcgen05.wait::st.sync.aligned;" ::"r"(a16),
      "r"(u32(prev[0].y)), "r"(u32(cur[0].x)), "r"(u32(prev[1].y)), "r"(u32(cur[1].x)), "r"(u32(prev[2].y)),
      "r"(u32(cur[2].x)), "r"(u32(prev[3].y)), "r"(u32(cur[3].x)), "r"(u32(prev[4].y)), "r"(u32(cur[4].x)),
      "r"(u32(prev[5].y)), "r"(u32(cur[5].x)), "r"(u32(prev[6].y)), "r"(u32(cur[6].x)), "r"(u32(prev[7].y)),
      "r"(u32(cur[7].x)), "r"(a4), "r"(u32(prev[8].y)), "r"(u32(cur[8].x)), "r"(u32(prev[9].y)), "r"(u32(cur[9].x))
      : "memory");
}
__device__ __forceinline__ void tm_load_rec(uint32_t a16, uint32_t a4, f32x2 (&r)[NV]) {
  uint32_t v[2 * NV];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%20];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%16, %17, %18, %19}, [%21];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
        "=r"(v[17]), "=r"(v[18]), "=r"(v[19])
      : "r"(a16), "r"(a4)
      : "memory");
#pragma unroll
  for (int i = 0; i < NV; ++i) r[i] = f32x2(f32(v[2 * i]), f32(v[2 * i + 1]));
}
__device__ __forceinline__ void tm_store4(uint32_t a, f32x2 p, f32x2 q) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};\n\t"
      "tcgen05.wait::st.sync.aligned;" ::"r"(a),
      "r"(u32(p.x)), "r"(u32(p.y)), "r"(u32(q.x)), "r"(u32(q.y))
      : "memory");
}
__device__ __forceinline__ void tm_load4(uint32_t a, f32x2& p, f32x2& q) {
  uint32_t v0, v1, v2, v3;
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(v0), "=r"(v1), "=r"(v2), "=r"(v3)
      : "r"(a)
      : "memory");
  p = f32x2(f32(v0), f32(v1));
  q = f32x2(f32(v2), f32(v3));
}
__device__ __forceinline__ void tm_store2(uint32_t a, f32x2 p) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1, %2};\n\t"
      "tcgen05.wait::st.sync.aligned;" ::"r"(a),
      "r"(u32(p.x)), "r"(u32(p.y))
      : "memory");
}
__device__ __forceinline__ f32x2 tm_load2(uint32_t a) {
  uint32_t v0, v1;
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%2];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(v0), "=r"(v1)
      : "r"(a)
      : "memory");
  return f32x2(f32(v0), f32(v1));
}

// Coefficients with both lanes equal.
inline Coef<f32x2> pair_coef(const Coef<float>& cf) {
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
  c.inv_re = f32x2(cf.inv_re, cf.inv_re);
  c.kappa = f32x2(cf.kappa, cf.kappa);
  c.H0 = f32x2(cf.H0, cf.H0);
  return c;
}

// The z march of one CTA over the 32 x 8 column tile (bx, by), output
// planes [zbeg, min(zend, n2)), binary32 stage input and output.  DF: the
// accumulator is a double-float pair (else binary64).  WITH_KE: adds the
// stage input's kinetic energy and enstrophy of the tile's points to
// ke_acc / ens_acc.  Ends with a barrier (shared memory reusable).
template <bool DF, bool WITH_KE>
__device__ __forceinline__ void march(const StageArgs& a, const Coef<f32x2>& c, int bx, int by, int zbeg, int zend_req,
                                      Smem& sm, double& ke_acc, double& ens_acc, uint32_t tmem_base) {
  using T = f32x2;
  constexpr int PTS = SX * SY;
  constexpr int NHALO = PTS - NT;
  constexpr int LPT = 1 + (NHALO + NT - 1) / NT;  // own point + halo points per thread (2)

  const int n0 = a.g.n0, n1 = a.g.n1, n2 = a.g.n2;
  const unsigned plane = (unsigned)n0 * (unsigned)n1;
  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;
  const int x0 = bx * TX, y0 = by * TY;
  const int zend = min(zend_req, n2);
  const int gx = x0 + tx, gy = y0 + ty;
  const bool valid_xy = (gx < n0) && (gy < n1);
  const unsigned own = valid_xy ? (unsigned)gx + (unsigned)n0 * (unsigned)gy : 0u;
  const float* q_in = static_cast<const float*>(a.q_in);
  const long long P = a.g.P;

  // points this thread loads on every plane (periodic wrap folded in): its
  // own tile point, then at most one point of the halo ring
  int ld_off[LPT], ld_s[LPT];
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
      ld_off[l] = wrapi(x0 - HALO + sx, n0) + n0 * wrapi(y0 - HALO + sy, n1);
      ld_s[l] = sy * SX + sx;
    } else {
      ld_off[l] = -1;
      ld_s[l] = 0;
    }
  }

  // halo tasks of the s-helpers: s_0 on the x0-halo columns (4 TY points),
  // s_1 on the x1-halo rows (4 TX points); one packed word per task:
  // kind (0 none, 1 s_0, 2 s_1) | hx << 2 | hy << 8 | buffer index << 12
  constexpr int NHT = 4 * (TX + TY);
  constexpr int HPT = (NHT + NT - 1) / NT;
  int htask[HPT];
#pragma unroll
  for (int j = 0; j < HPT; ++j) {
    const int h = tid + j * NT;
    htask[j] = 0;
    if (h < 4 * TY) {
      const int r = h >> 2, k = h & 3;
      const int hx = (k < 2) ? k : TX + k;
      htask[j] = 1 | (hx << 2) | ((r + HALO) << 8) | ((r * SX + hx) << 12);
    } else if (h < NHT) {
      const int h2 = h - 4 * TY;
      const int col = h2 % TX, k = h2 / TX;
      const int hy = (k < 2) ? k : TY + k;
      htask[j] = 2 | ((col + HALO) << 2) | (hy << 8) | ((hy * TX + col) << 12);
    }
  }

  const int nplanes = zend - zbeg;
  const int npairs = (nplanes + 1) / 2;
  const int nit = npairs + 2;  // two warm-up pairs (planes zbeg-2 .. zbeg+1)
  const uint32_t twin = __shfl_sync(0xffffffffu, tmem_base + ((((threadIdx.x >> 5) & 3u) * 32u) << 16) +
                                                     (threadIdx.x >> 7) * (uint32_t)Tm::COLS, 0);

  // per-field bases of the stage input (uniform over the CTA)
  const float* qb[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) qb[f] = q_in + (long long)f * P;
  // prefetched stage input of the entering pair: [point][field][lane]; the
  // next plane to load is zl (wrapped periodically, advanced by two planes)
  float pf[LPT][NF][2];
  int zl = wrapi(zbeg - HALO, n2);
  auto issue_loads = [&]() {
    const int z1 = (zl + 1 == n2) ? 0 : zl + 1;
    const unsigned zo0 = (unsigned)zl * plane, zo1 = (unsigned)z1 * plane;
    zl = (z1 + 1 == n2) ? 0 : z1 + 1;
#pragma unroll
    for (int l = 0; l < LPT; ++l) {
      if (l == 0 || ld_off[l] >= 0) {
        const unsigned o0 = zo0 + (unsigned)ld_off[l], o1 = zo1 + (unsigned)ld_off[l];
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          pf[l][f][0] = qb[f][o0];
          pf[l][f][1] = qb[f][o1];
        }
      }
    }
  };
  issue_loads();

  // ring slots, rotated each iteration: aligned TMEM / u_2 slots of the
  // entering pair (as), the previous one (ap) and the one before (a2)
  int as = 0, ap = 2, a2 = 1;
  for (int it = 0; it < nit; ++it) {
    const int fs = it & 1;  // full pair slot of the entering pair (and its shifted / diagonal TMEM slots)
    if (it > 0) {
      const int t = a2;
      a2 = ap;
      ap = as;
      as = t;
    }
    // ---------------------------------------------------------------- phase 1
    {
      T* ring = &sm.ring[fs][0][0][0];
#pragma unroll
      for (int l = 0; l < LPT; ++l) {
        if (l == 0 || ld_off[l] >= 0) {
          T rec[NV];
          const T rho_p(pf[l][0][0], pf[l][0][1]);
          const T m0(pf[l][1][0], pf[l][1][1]);
          const T m1(pf[l][2][0], pf[l][2][1]);
          const T m2(pf[l][3][0], pf[l][3][1]);
          const T E_p(pf[l][4][0], pf[l][4][1]);
          const T rho = T(1) + rho_p;
          const T rinv(rcp_approx_f32(rho.x), rcp_approx_f32(rho.y));
          const T u0 = m0 * rinv, u1 = m1 * rinv, u2 = m2 * rinv;
          const T mu = fma(m2, u2, fma(m1, u1, m0 * u0));
          const T p_p = c.gm1 * fma(T(-0.5), mu, E_p);    // Eq. 4: p - p_ref
          const T T_p = fma(c.gM2, p_p, -rho_p) * rinv;  // Eq. 5: T - 1
          rec[V_RHO] = rho_p;
          rec[V_M0] = m0;
          rec[V_M1] = m1;
          rec[V_M2] = m2;
          rec[V_E] = E_p;
          rec[V_U0] = u0;
          rec[V_U1] = u1;
          rec[V_U2] = u2;
          rec[V_P] = p_p;
          rec[V_T] = T_p;
          store_rec(ring + ld_s[l] * NV, rec);
          (&sm.u2ring[as][0][0])[ld_s[l]] = u2;
          if (l == 0) {
            tm_store_rec(twin + Tm::AREC + 16u * as, twin + Tm::ATAIL + 4u * as, rec);
            if (it > 0) {
              T prev[NV];
              tm_load_rec(twin + Tm::AREC + 16u * ap, twin + Tm::ATAIL + 4u * ap, prev);
              tm_store_shifted(twin + Tm::SREC + 16u * fs, twin + Tm::STAIL + 4u * fs, prev, rec);
            }
          }
        }
      }
    }
    if (it + 1 < nit) issue_loads();
    __syncthreads();
    // --------------------------------------------------------------- phase 2a
    // D1_x u0, D1_y u1 and s_2 of the entering pair at the own column
    {
      const T(*R)[SX][NV] = sm.ring[fs];
      const int sy = ty + HALO, sx = tx + HALO;
      const T d00 = fma(c.c1[0], R[sy][sx + 1][V_U0] - R[sy][sx - 1][V_U0],
                        -c.c2[0] * (R[sy][sx + 2][V_U0] - R[sy][sx - 2][V_U0]));
      const T d11 = fma(c.c1[1], R[sy + 1][sx][V_U1] - R[sy - 1][sx][V_U1],
                        -c.c2[1] * (R[sy + 2][sx][V_U1] - R[sy - 2][sx][V_U1]));
      const T s2 = d00 + d11;
      tm_store4(twin + Tm::DIAG + 4u * fs, d00, d11);
      tm_store2(twin + Tm::SA + 2u * as, s2);
      if (it > 0) {
        const T sp = tm_load2(twin + Tm::SA + 2u * ap);
        tm_store2(twin + Tm::SS + 2u * fs, T(sp.y, s2.x));
      }
    }
    if (it < 2) continue;

    // centre pair: planes zc, zc + 1 (the previous entering pair)
    const int zc = zbeg + 2 * (it - 2);
    const int fc = fs ^ 1;  // a2: aligned slot of the pair before the centre pair (planes zc-2, zc-1)
    const bool v0 = valid_xy, v1 = valid_xy && (zc + 1 < zend);
    const unsigned oc0 = (unsigned)zc * plane + own;
    const unsigned oc1 = oc0 + plane;
    T g00c, g11c, d22;
    // --------------------------------------------------------------- phase 2b
    // s_0 and s_1 of both centre planes on the tile and halo
    {
      const int sy = ty + HALO, sx = tx + HALO;
      // D1_z u_2 for both lanes from the u_2 pairs of planes zc-2 .. zc+3
      auto u2z = [&](int yy, int xx) {
        const T lo = sm.u2ring[a2][yy][xx], mi = sm.u2ring[ap][yy][xx], hi = sm.u2ring[as][yy][xx];
        return fma(c.c1[2], T(mi.y, hi.x) - T(lo.y, mi.x), -c.c2[2] * (hi - lo));
      };
      d22 = u2z(sy, sx);
      tm_load4(twin + Tm::DIAG + 4u * fc, g00c, g11c);
      sm.s0buf[ty][sx] = g11c + d22;
      sm.s1buf[sy][tx] = g00c + d22;
      const T(*R)[SX][NV] = sm.ring[fc];
#pragma unroll
      for (int j = 0; j < HPT; ++j) {
        const int kind = htask[j] & 3, hx = (htask[j] >> 2) & 63, hy = (htask[j] >> 8) & 15, dst = htask[j] >> 12;
        if (kind == 1) {
          const T d11 = fma(c.c1[1], R[hy + 1][hx][V_U1] - R[hy - 1][hx][V_U1],
                            -c.c2[1] * (R[hy + 2][hx][V_U1] - R[hy - 2][hx][V_U1]));
          (&sm.s0buf[0][0])[dst] = d11 + u2z(hy, hx);
        } else if (kind == 2) {
          const T d00 = fma(c.c1[0], R[hy][hx + 1][V_U0] - R[hy][hx - 1][V_U0],
                            -c.c2[0] * (R[hy][hx + 2][V_U0] - R[hy][hx - 2][V_U0]));
          (&sm.s1buf[0][0])[dst] = d00 + u2z(hy, hx);
        }
      }
    }
    __syncthreads();
    // ---------------------------------------------------------------- phase 3
    {
      const int sy = ty + HALO, sx = tx + HALO;
      const T(*C)[SX][NV] = sm.ring[fc];
      T uc[3];  // centre velocities (the rest of the centre record is read again for the assembly)
      {
        T cen[NV];
        tm_load_rec(twin + Tm::AREC + 16u * ap, twin + Tm::ATAIL + 4u * ap, cen);
        uc[0] = cen[V_U0];
        uc[1] = cen[V_U1];
        uc[2] = cen[V_U2];
      }

      Terms<T> t;
      t.rrho = t.rE = t.lapT = T(0.0f, 0.0f);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        t.rM[i] = T(0.0f, 0.0f);
        t.lap[i] = T(0.0f, 0.0f);
      }
      t.g[0][0] = g00c;
      t.g[1][1] = g11c;
      t.g[2][2] = d22;

      {
        const int off[4] = {-2, -1, 1, 2};
        auto ld = [&](int k, T(&r)[NV]) { load_rec(&C[sy][sx + off[k]][0], r); };
        auto sf = [&](int k, const T(&)[NV]) { return sm.s0buf[ty][sx + off[k]]; };
        axis_terms_stream<0>(ld, sf, c, uc, t);
      }
      {
        const int off[4] = {-2, -1, 1, 2};
        auto ld = [&](int k, T(&r)[NV]) { load_rec(&C[sy + off[k]][sx][0], r); };
        auto sf = [&](int k, const T(&)[NV]) { return sm.s1buf[sy + off[k]][tx]; };
        axis_terms_stream<1>(ld, sf, c, uc, t);
      }
      // accumulator of both centre points (fetched now so that its latency
      // overlaps the x2 terms)
      float ah[NF][2], al[NF][2];  // DF: hi, lo; else unused
      double ad[NF][2];            // binary64 accumulator
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        if (DF) {
          ah[f][0] = v0 ? a.dacc_in[(long long)f * P + oc0] : 0.f;
          al[f][0] = v0 ? a.dacc_in[(long long)(NF + f) * P + oc0] : 0.f;
          ah[f][1] = v1 ? a.dacc_in[(long long)f * P + oc1] : 0.f;
          al[f][1] = v1 ? a.dacc_in[(long long)(NF + f) * P + oc1] : 0.f;
        } else {
          ad[f][0] = v0 ? a.acc_in[(long long)f * P + oc0] : 0.0;
          ad[f][1] = v1 ? a.acc_in[(long long)f * P + oc1] : 0.0;
        }
      }
      {
        // x2 neighbours (zc+o, zc+1+o): o = -2 aligned pair before the
        // centre, o = -1 shifted pair of the centre, o = +1 shifted pair of
        // the entering pair, o = +2 the entering pair
        auto ld = [&](int k, T(&r)[NV]) {
          if (k == 0) tm_load_rec(twin + Tm::AREC + 16u * a2, twin + Tm::ATAIL + 4u * a2, r);
          else if (k == 1) tm_load_rec(twin + Tm::SREC + 16u * fc, twin + Tm::STAIL + 4u * fc, r);
          else if (k == 2) tm_load_rec(twin + Tm::SREC + 16u * fs, twin + Tm::STAIL + 4u * fs, r);
          else tm_load_rec(twin + Tm::AREC + 16u * as, twin + Tm::ATAIL + 4u * as, r);
        };
        auto sf = [&](int k, const T(&)[NV]) {
          if (k == 0) return tm_load2(twin + Tm::SA + 2u * a2);
          if (k == 1) return tm_load2(twin + Tm::SS + 2u * fc);
          if (k == 2) return tm_load2(twin + Tm::SS + 2u * fs);
          return tm_load2(twin + Tm::SA + 2u * as);
        };
        axis_terms_stream<2>(ld, sf, c, uc, t);
      }
      T cen[NV];
      tm_load_rec(twin + Tm::AREC + 16u * ap, twin + Tm::ATAIL + 4u * ap, cen);
      const T rho_p = cen[V_RHO];
      const T mc[3] = {cen[V_M0], cen[V_M1], cen[V_M2]};
      T R[5];
      assemble_residual(t, rho_p, mc, cen[V_E], uc, cen[V_T], c, R);

      // Runge-Kutta stage of both planes (§2.2, Fig. 1)
      float* q_out = static_cast<float*>(a.q_out);
      if constexpr (DF) {
        // acc' = acc + b dt R by an error-free two-sum of hi and the
        // increment, the error folded into lo and renormalised;
        // Q_{k+1} = hi' + (lo' + (a - b) dt R)
        const T bdt(a.b_dt32, a.b_dt32), ambdt(a.amb_dt32, a.amb_dt32);
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          const T hi(ah[f][0], ah[f][1]), lo(al[f][0], al[f][1]);
          const T x = bdt * R[f];
          const T s = hi + x;
          const T bb = s - hi;
          const T err = (hi - (s - bb)) + (x - bb);
          const T lo2 = lo + err;
          const T hi3 = s + lo2;
          const T lo3 = lo2 - (hi3 - s);
          const T qo = hi3 + fma(ambdt, R[f], lo3);
          if (v0) {
            a.dacc_out[(long long)f * P + oc0] = hi3.x;
            a.dacc_out[(long long)(NF + f) * P + oc0] = lo3.x;
            if (q_out) q_out[(long long)f * P + oc0] = qo.x;
          }
          if (v1) {
            a.dacc_out[(long long)f * P + oc1] = hi3.y;
            a.dacc_out[(long long)(NF + f) * P + oc1] = lo3.y;
            if (q_out) q_out[(long long)f * P + oc1] = qo.y;
          }
        }
      } else {
        // binary64 accumulator: acc' = acc + (b dt R) (one DADD per value),
        // Q_{k+1} = float(acc') + (a - b) dt R
        const T bdt(a.b_dt32, a.b_dt32), ambdt(a.amb_dt32, a.amb_dt32);
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          const T x = bdt * R[f];
          const double n0v = ad[f][0] + widen_f32_fast(x.x);
          const double n1v = ad[f][1] + widen_f32_fast(x.y);
          const T qo = fma(ambdt, R[f], T(narrow_f64_fast(n0v), narrow_f64_fast(n1v)));
          if (v0) {
            a.acc_out[(long long)f * P + oc0] = n0v;
            if (q_out) q_out[(long long)f * P + oc0] = qo.x;
          }
          if (v1) {
            a.acc_out[(long long)f * P + oc1] = n1v;
            if (q_out) q_out[(long long)f * P + oc1] = qo.y;
          }
        }
      }
      if (WITH_KE) {
        const T w0 = t.g[2][1] - t.g[1][2], w1 = t.g[0][2] - t.g[2][0], w2 = t.g[1][0] - t.g[0][1];
        const T rho = T(1) + rho_p;
        const T ke_t = T(0.5f, 0.5f) * fma(mc[2], uc[2], fma(mc[1], uc[1], mc[0] * uc[0]));
        const T ens_t = T(0.5f, 0.5f) * rho * fma(w2, w2, fma(w1, w1, w0 * w0));
        if (v0) {
          ke_acc += (double)ke_t.x;
          ens_acc += (double)ens_t.x;
        }
        if (v1) {
          ke_acc += (double)ke_t.y;
          ens_acc += (double)ens_t.y;
        }
      }
    }
    __syncthreads();  // the next entering pair overwrites this centre pair's slot
  }
}

}  // namespace zp

// Single grid, binary32 stage fields, two planes per thread (z queue mode 2).
template <bool DF, bool WITH_KE>
__global__ void __launch_bounds__(zp::NT, 2) fused_zpair_kernel(const StageArgs a, const Coef<f32x2> c) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  zp::Smem& sm = *reinterpret_cast<zp::Smem*>(smem_raw);
  const uint32_t tbase = tmem_acquire<zp::NCOL>(&sm.tmem_base);
  double ke = 0.0, ens = 0.0;
  const int zbeg = blockIdx.z * a.zc;
  zp::march<DF, WITH_KE>(a, c, blockIdx.x, blockIdx.y, zbeg, zbeg + a.zc, sm, ke, ens, tbase);
  if (WITH_KE) {
    const long long b = blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
    block_reduce_pair<zp::NT>(sm.red, ke, ens, a.ke_partials + 2 * b);
  }
  tmem_release<zp::NCOL>(tbase);
}

}  // namespace sbli
