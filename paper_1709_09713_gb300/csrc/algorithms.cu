// algorithms.cu -- the paper's other evaluation strategies for the residual
// of Eqs. 1-3 (§2.4 intermediate storage, §2.5 minimal storage), in binary64,
// as comparison variants beside the store-all (BL) variant and the tiled
// fused kernel:
//
//   RS  Recompute Some: the 9 velocity gradients D_j u_i are stored to global
//       arrays first (velocity arrays, then one derivative launch each, as BL
//       does); every other derivative is a stencil written into the residual
//       expressions, evaluated again at each place it occurs.
//   SS  Store Some: the same 9 stored arrays; every other derivative is
//       evaluated once into a thread-local variable and reused.
//   RA  Recompute All: nothing stored; every derivative, velocity gradients
//       and the mixed derivatives built on them included, is a stencil at each
//       place it occurs in one large expression per residual.
//   SN  Store None: nothing stored; all 60 derivatives evaluated once into
//       thread-local variables, in the order they are listed (by kind).
//   SN2 as SN, with the evaluations grouped by velocity index i (every
//       derivative of a quantity holding u_i), then the remaining group.
//
// The primitives u_i, p and T (Eqs. 4-5) are evaluated into arrays once per
// stage before the residual, for every class (the derivative-storage classes
// of Table 1 count derivative arrays only; its operation counts leave no room
// for recomputing a division-bearing primitive at every stencil point).  The
// residual kernel runs one thread per grid point; stencil values come from
// global memory (through L1/L2) and the differentiated products are formed
// at each stencil point they are needed.  The Runge-Kutta update of Fig. 1
// is written in the same kernel.
// All strategies share one assembly of Eqs. 1-3 over derivative identifiers,
// and differ only in how a derivative reaches it; whether the compiler
// merges repeated evaluations is what the comparison measures.
//
// Variables are deviations from the reference state, as in the other paths.
#include <utility>

#include "sbli_internal.cuh"

namespace sbli {

namespace {

// the 60 distinct derivatives of Eqs. 1-3
enum DerivId {
  D_RHOU = 0,    // D_j m_i          [i][j]  9
  D_U = 9,       // D_j u_i          [i][j]  9
  D_RHOUU = 18,  // D_j (m_i u_j)    [i][j]  9
  D_RHO = 27,    // D_j rho'                 3
  D_P = 30,      // D_j p'                   3
  D_E = 33,      // D_j E'                   3
  D_EU = 36,     // D_j (E' u_j)             3
  D_PU = 39,     // D_j (p' u_j)             3
  D2_U = 42,     // D2_j u_i         [i][j]  9
  DD_U = 51,     // D_i D_j u_j, i != j      6 (01,02,10,12,20,21)
  D2_T = 57,     // D2_j T'                  3
  N_DERIV = 60
};

constexpr int offd_c(int i, int j) { return 2 * i + (j > i ? j - 1 : j); }
constexpr int dd_i(int o) { return o / 2; }
constexpr int dd_j(int o) { return (o % 2) + ((o % 2) >= o / 2 ? 1 : 0); }
static_assert(dd_i(offd_c(2, 1)) == 2 && dd_j(offd_c(2, 1)) == 1 && dd_j(offd_c(0, 2)) == 2, "mixed index map");

template <int B, int E, class F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    static_for<B + 1, E>(f);
  }
}

// Conserved variables and primitive arrays at the stencil points of one
// grid point (periodic).
struct PointQ {
  const double* __restrict__ q;
  const double* __restrict__ w;  // u_0, u_1, u_2, p', T' (5 arrays of P)
  long long P;
  long long n0;
  int xo[5], yo[5];
  long long zo[5];
  const Coef<double>* c;

  __device__ long long at(int s0, int s1, int s2) const { return xo[s0 + 2] + n0 * yo[s1 + 2] + zo[s2 + 2]; }
  template <int A>
  __device__ long long along(int s) const {
    return at(A == 0 ? s : 0, A == 1 ? s : 0, A == 2 ? s : 0);
  }
  template <int A, int B>
  __device__ long long along2(int sa, int sb) const {
    return at((A == 0 ? sa : 0) + (B == 0 ? sb : 0), (A == 1 ? sa : 0) + (B == 1 ? sb : 0),
              (A == 2 ? sa : 0) + (B == 2 ? sb : 0));
  }
  __device__ double rho_p(long long n) const { return __ldg(q + n); }
  __device__ double m(int i, long long n) const { return __ldg(q + (1 + i) * P + n); }
  __device__ double E(long long n) const { return __ldg(q + 4 * P + n); }
  __device__ double u(int i, long long n) const { return __ldg(w + i * P + n); }
  __device__ double p(long long n) const { return __ldg(w + 3 * P + n); }
  __device__ double temp(long long n) const { return __ldg(w + 4 * P + n); }
};

// Eq. 6 along axis A of the quantity f(n)
template <int A, class F>
__device__ __forceinline__ double d1(const PointQ& Q, F f) {
  const Coef<double>& c = *Q.c;
  return c.c1[A] * (f(Q.along<A>(1)) - f(Q.along<A>(-1))) - c.c2[A] * (f(Q.along<A>(2)) - f(Q.along<A>(-2)));
}
// Eq. 7 along axis A
template <int A, class F>
__device__ __forceinline__ double d2(const PointQ& Q, F f) {
  const Coef<double>& c = *Q.c;
  return c.e0[A] * f(Q.at(0, 0, 0)) + c.e1[A] * (f(Q.along<A>(1)) + f(Q.along<A>(-1))) +
         c.e2[A] * (f(Q.along<A>(2)) + f(Q.along<A>(-2)));
}
// D_A (D_B f), A != B: Eq. 6 along A of Eq. 6 along B
template <int A, int B, class F>
__device__ __forceinline__ double dd(const PointQ& Q, F f) {
  const Coef<double>& c = *Q.c;
  auto inner = [&](int sa) {
    return c.c1[B] * (f(Q.along2<A, B>(sa, 1)) - f(Q.along2<A, B>(sa, -1))) -
           c.c2[B] * (f(Q.along2<A, B>(sa, 2)) - f(Q.along2<A, B>(sa, -2)));
  };
  return c.c1[A] * (inner(1) - inner(-1)) - c.c2[A] * (inner(2) - inner(-2));
}

// Derivative ID evaluated on the fly from the conserved variables.
template <int ID>
__device__ __forceinline__ double on_the_fly(const PointQ& Q) {
  if constexpr (ID >= D_RHOU && ID < D_U) {
    constexpr int i = (ID - D_RHOU) / 3, j = (ID - D_RHOU) % 3;
    return d1<j>(Q, [&](long long n) { return Q.m(i, n); });
  } else if constexpr (ID >= D_U && ID < D_RHOUU) {
    constexpr int i = (ID - D_U) / 3, j = (ID - D_U) % 3;
    return d1<j>(Q, [&](long long n) { return Q.u(i, n); });
  } else if constexpr (ID >= D_RHOUU && ID < D_RHO) {
    constexpr int i = (ID - D_RHOUU) / 3, j = (ID - D_RHOUU) % 3;
    return d1<j>(Q, [&](long long n) { return Q.m(i, n) * Q.u(j, n); });
  } else if constexpr (ID >= D_RHO && ID < D_P) {
    return d1<ID - D_RHO>(Q, [&](long long n) { return Q.rho_p(n); });
  } else if constexpr (ID >= D_P && ID < D_E) {
    return d1<ID - D_P>(Q, [&](long long n) { return Q.p(n); });
  } else if constexpr (ID >= D_E && ID < D_EU) {
    return d1<ID - D_E>(Q, [&](long long n) { return Q.E(n); });
  } else if constexpr (ID >= D_EU && ID < D_PU) {
    constexpr int j = ID - D_EU;
    return d1<j>(Q, [&](long long n) { return Q.E(n) * Q.u(j, n); });
  } else if constexpr (ID >= D_PU && ID < D2_U) {
    constexpr int j = ID - D_PU;
    return d1<j>(Q, [&](long long n) { return Q.p(n) * Q.u(j, n); });
  } else if constexpr (ID >= D2_U && ID < DD_U) {
    constexpr int i = (ID - D2_U) / 3, j = (ID - D2_U) % 3;
    return d2<j>(Q, [&](long long n) { return Q.u(i, n); });
  } else if constexpr (ID >= DD_U && ID < D2_T) {
    constexpr int i = dd_i(ID - DD_U), j = dd_j(ID - DD_U);
    return dd<i, j>(Q, [&](long long n) { return Q.u(j, n); });
  } else {
    static_assert(ID >= D2_T && ID < N_DERIV, "derivative id");
    return d2<ID - D2_T>(Q, [&](long long n) { return Q.temp(n); });
  }
}

// Derivative ID with the velocity gradients taken from the 9 stored arrays
// G[3i+j] = D_j u_i (the mixed derivatives are Eq. 6 applied to them).
template <int ID>
__device__ __forceinline__ double with_stored_gradients(const PointQ& Q, const double* __restrict__ G) {
  if constexpr (ID >= D_U && ID < D_RHOUU) {
    return __ldg(G + (long long)(ID - D_U) * Q.P + Q.at(0, 0, 0));
  } else if constexpr (ID >= DD_U && ID < D2_T) {
    constexpr int i = dd_i(ID - DD_U), j = dd_j(ID - DD_U);
    const double* Gjj = G + (long long)(3 * j + j) * Q.P;
    return d1<i>(Q, [&](long long n) { return __ldg(Gjj + n); });
  } else {
    return on_the_fly<ID>(Q);
  }
}

// Derivative providers: get<ID>() is called at every place ID occurs.
struct RecomputeAll {
  const PointQ& Q;
  template <int ID>
  __device__ __forceinline__ double get() const {
    return on_the_fly<ID>(Q);
  }
};
struct RecomputeSome {
  const PointQ& Q;
  const double* G;
  template <int ID>
  __device__ __forceinline__ double get() const {
    return with_stored_gradients<ID>(Q, G);
  }
};
struct Locals {
  double v[N_DERIV];
  template <int ID>
  __device__ __forceinline__ double get() const {
    return v[ID];
  }
};

// SN2 evaluation order: for i = 0, 1, 2 every derivative of a quantity that
// holds u_i (D_j u_i, D2_j u_i, D_a D_i u_i, D_i (m_k u_i), D_i (E' u_i),
// D_i (p' u_i)), then the rest (D_j m_i, D_j rho', D_j p', D_j E', D2_j T').
struct Sn2Order {
  int id[N_DERIV];
  constexpr Sn2Order() : id{} {
    int n = 0;
    for (int i = 0; i < 3; ++i) {
      for (int j = 0; j < 3; ++j) id[n++] = D_U + 3 * i + j;
      for (int j = 0; j < 3; ++j) id[n++] = D2_U + 3 * i + j;
      for (int a = 0; a < 3; ++a)
        if (a != i) id[n++] = DD_U + offd_c(a, i);
      for (int k = 0; k < 3; ++k) id[n++] = D_RHOUU + 3 * k + i;
      id[n++] = D_EU + i;
      id[n++] = D_PU + i;
    }
    for (int x = 0; x < 9; ++x) id[n++] = D_RHOU + x;
    for (int j = 0; j < 3; ++j) id[n++] = D_RHO + j;
    for (int j = 0; j < 3; ++j) id[n++] = D_P + j;
    for (int j = 0; j < 3; ++j) id[n++] = D_E + j;
    for (int j = 0; j < 3; ++j) id[n++] = D2_T + j;
  }
};
constexpr Sn2Order SN2_ORDER{};

constexpr bool sn2_is_permutation() {
  bool seen[N_DERIV] = {};
  for (int k = 0; k < N_DERIV; ++k) {
    const int v = SN2_ORDER.id[k];
    if (v < 0 || v >= N_DERIV || seen[v]) return false;
    seen[v] = true;
  }
  return true;
}
static_assert(sn2_is_permutation(), "SN2 order lists each derivative once");

// Residual of Eqs. 1-3 at the centre point from a derivative provider.  Every
// derivative is requested at each place it occurs in the equations.
template <class DP>
__device__ __forceinline__ void assemble(const DP& d, double rho, const double (&m)[3], const double (&u)[3],
                                         double E, const Coef<double>& c, double (&R)[5]) {
  auto div = [&]() { return d.template get<D_U + 0>() + d.template get<D_U + 4>() + d.template get<D_U + 8>(); };
  // Eq. 1
  double conv = 0.0;
  static_for<0, 3>([&](auto J) {
    constexpr int j = J;
    conv += d.template get<D_RHOU + 3 * j + j>() + rho * d.template get<D_U + 3 * j + j>() +
            u[j] * d.template get<D_RHO + j>();
  });
  R[0] = -0.5 * conv;
  // Eq. 2: viscous part sd_i = sum_j D2_j u_i + (1/3) sum_j D_i D_j u_j
  auto sd = [&](auto I) {
    constexpr int i = I;
    double lap = 0.0, cross = 0.0;
    static_for<0, 3>([&](auto J) {
      constexpr int j = J;
      lap += d.template get<D2_U + 3 * i + j>();
      if constexpr (j == i)
        cross += d.template get<D2_U + 3 * i + i>();
      else
        cross += d.template get<DD_U + offd_c(i, j)>();
    });
    return lap + cross - (2.0 / 3.0) * cross;
  };
  static_for<0, 3>([&](auto I) {
    constexpr int i = I;
    double cv = 0.0;
    static_for<0, 3>([&](auto J) {
      constexpr int j = J;
      cv += d.template get<D_RHOUU + 3 * i + j>() + m[i] * d.template get<D_U + 3 * j + j>() +
            u[j] * d.template get<D_RHOU + 3 * i + j>();
    });
    R[1 + i] = -0.5 * cv - d.template get<D_P + i>() + c.inv_re * sd(I);
  });
  // Eq. 3 (the reference enthalpy H0 carries the constant parts of rho E and p)
  conv = 0.0;
  double pw = 0.0, heat = 0.0, vw = 0.0, diss = 0.0;
  static_for<0, 3>([&](auto J) {
    constexpr int j = J;
    conv += d.template get<D_EU + j>() + E * d.template get<D_U + 3 * j + j>() + u[j] * d.template get<D_E + j>();
    pw += d.template get<D_PU + j>();
    heat += d.template get<D2_T + j>();
  });
  static_for<0, 3>([&](auto I) {
    constexpr int i = I;
    vw += u[i] * c.inv_re * sd(I);
    static_for<0, 3>([&](auto J) {
      constexpr int j = J;
      const double g = d.template get<D_U + 3 * i + j>();
      diss += g * (g + d.template get<D_U + 3 * j + i>() - (i == j ? (2.0 / 3.0) * div() : 0.0));
    });
  });
  R[4] = -0.5 * conv - c.H0 * div() - pw + vw + c.inv_re * diss + c.kappa * heat;
}

template <int ALG>
__global__ void __launch_bounds__(256) algorithm_stage_kernel(Geom g, const __grid_constant__ Coef<double> c,
                                                              const double* __restrict__ q,
                                                              const double* __restrict__ W,
                                                              const double* __restrict__ G, const double* acc_in,
                                                              double* acc_out, double* __restrict__ q_out,
                                                              double* __restrict__ r_out, double a_dt, double b_dt) {
  const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y, k = blockIdx.z;
  if (i >= g.n0 || j >= g.n1) return;
  PointQ Q;
  Q.q = q;
  Q.w = W;
  Q.P = g.P;
  Q.n0 = g.n0;
  Q.c = &c;
  const long long pl = (long long)g.n0 * g.n1;
#pragma unroll
  for (int s = -2; s <= 2; ++s) {
    Q.xo[s + 2] = wrapi(i + s, g.n0);
    Q.yo[s + 2] = wrapi(j + s, g.n1);
    Q.zo[s + 2] = pl * wrapi(k + s, g.n2);
  }
  const long long n = Q.at(0, 0, 0);
  const double rho = 1.0 + Q.rho_p(n);
  const double m[3] = {Q.m(0, n), Q.m(1, n), Q.m(2, n)};
  const double u[3] = {Q.u(0, n), Q.u(1, n), Q.u(2, n)};
  const double E = Q.E(n);
  double R[5];
  if constexpr (ALG == SBLI_RA) {
    assemble(RecomputeAll{Q}, rho, m, u, E, c, R);
  } else if constexpr (ALG == SBLI_RS) {
    assemble(RecomputeSome{Q, G}, rho, m, u, E, c, R);
  } else if constexpr (ALG == SBLI_SS) {
    Locals L;
    static_for<0, N_DERIV>([&](auto I) { L.v[I] = with_stored_gradients<I>(Q, G); });
    assemble(L, rho, m, u, E, c, R);
  } else if constexpr (ALG == SBLI_SN) {
    Locals L;
    static_for<0, N_DERIV>([&](auto I) { L.v[I] = on_the_fly<I>(Q); });
    assemble(L, rho, m, u, E, c, R);
  } else {
    static_assert(ALG == SBLI_SN2, "algorithm");
    Locals L;
    static_for<0, N_DERIV>([&](auto I) {
      constexpr int id = SN2_ORDER.id[I];
      L.v[id] = on_the_fly<id>(Q);
    });
    assemble(L, rho, m, u, E, c, R);
  }
  if (r_out) {
#pragma unroll
    for (int f = 0; f < 5; ++f) r_out[f * g.P + n] = R[f];
    return;
  }
  // Fig. 1 stage update: Q_k+1 = Q_acc + a_k dt R, Q_acc += b_k dt R
#pragma unroll
  for (int f = 0; f < 5; ++f) {
    const double a = acc_in[f * g.P + n];
    acc_out[f * g.P + n] = fma(b_dt, R[f], a);
    if (q_out) q_out[f * g.P + n] = fma(a_dt, R[f], a);
  }
}

// Primitives of Eqs. 4-5 into arrays: u_i = m_i / rho, p' (deviation of
// p), T' (deviation of T), from the deviation-form conserved variables.
__global__ void primitives_kernel(long long P, const __grid_constant__ Coef<double> c, const double* __restrict__ q,
                                  double* __restrict__ w) {
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < P; n += (long long)gridDim.x * blockDim.x) {
    const double rho_p = q[n], rho = 1.0 + rho_p;
    double u[3];
    for (int i = 0; i < 3; ++i) u[i] = q[(1 + i) * P + n] / rho;
    const double p_p = c.gm1 * (q[4 * P + n] - 0.5 * rho * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]));  // Eq. 4
    for (int i = 0; i < 3; ++i) w[i * P + n] = u[i];
    w[3 * P + n] = p_p;
    w[4 * P + n] = (c.gM2 * p_p - rho_p) / rho;  // Eq. 5
  }
}

template <int ALG>
cudaError_t launch_alg(const Geom& g, const Coef<double>& c, const double* q, const double* W, const double* G,
                       const double* acc_in, double* acc_out, double* q_out, double* r_out, double a_dt, double b_dt,
                       cudaStream_t s) {
  dim3 blk(32, 8), grd((g.n0 + 31) / 32, (g.n1 + 7) / 8, g.n2);
  algorithm_stage_kernel<ALG><<<grd, blk, 0, s>>>(g, c, q, W, G, acc_in, acc_out, q_out, r_out, a_dt, b_dt);
  return cudaGetLastError();
}

}  // namespace

bool algorithm_stores_gradients(int alg) { return alg == SBLI_RS || alg == SBLI_SS; }

size_t algorithm_scratch_doubles(const Geom& g, int alg) {
  if (alg < SBLI_RS || alg > SBLI_SN2) return 0;
  // u_i, p', T' (5), plus D_j u_i (9) for the intermediate-storage classes
  return (size_t)(algorithm_stores_gradients(alg) ? 14 : 5) * g.P;
}

cudaError_t launch_algorithm_stage(int alg, const Geom& g, const Coef<double>& c, const double* q_in,
                                   const double* acc_in, double* acc_out, double* q_out, double* r_out, double a_dt,
                                   double b_dt, double* scratch, cudaStream_t s) {
  const double* G = nullptr;
  double* W = scratch;
  const long long blocks = (g.P + 255) / 256;
  primitives_kernel<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(g.P, c, q_in, W);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (algorithm_stores_gradients(alg)) {
    // the 9 velocity-gradient arrays, one derivative launch each
    const double* U = W;
    double* Gw = scratch + 5 * g.P;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        e = launch_derivative_fp64(g, c, U + i * g.P, Gw + (3 * i + j) * g.P, j, 1, s);
        if (e != cudaSuccess) return e;
      }
    G = Gw;
  }
  switch (alg) {
    case SBLI_RS: return launch_alg<SBLI_RS>(g, c, q_in, W, G, acc_in, acc_out, q_out, r_out, a_dt, b_dt, s);
    case SBLI_SS: return launch_alg<SBLI_SS>(g, c, q_in, W, G, acc_in, acc_out, q_out, r_out, a_dt, b_dt, s);
    case SBLI_RA: return launch_alg<SBLI_RA>(g, c, q_in, W, G, acc_in, acc_out, q_out, r_out, a_dt, b_dt, s);
    case SBLI_SN: return launch_alg<SBLI_SN>(g, c, q_in, W, G, acc_in, acc_out, q_out, r_out, a_dt, b_dt, s);
    case SBLI_SN2: return launch_alg<SBLI_SN2>(g, c, q_in, W, G, acc_in, acc_out, q_out, r_out, a_dt, b_dt, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace sbli
