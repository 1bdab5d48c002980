/*
 * sbli_oracle.c -- plain, slow FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline and
 * reference legs may load this library.  It shares no code with the CUDA
 * library and is compiled with -ffp-contract=off (no fused multiply-adds), so
 * every operation below rounds exactly as written.
 *
 * Source: Jammy, Jacobs, Lusher & Sandham, "Energy efficiency of finite
 * difference algorithms on multicore CPUs, GPUs, and Intel Xeon Phi
 * processors", arXiv:1709.09713.  Each function names the equation or
 * section it follows.  Where the paper is garbled or silent the reading taken
 * is stated at the point of use (R1..R7 below):
 *
 *  R1  Eq. 3's energy convection bracket is printed with two minus signs that
 *      turn it into +u_j d(rhoE)/dx_j.  It is read as the Blaisdell skew form
 *      the text names (same form as Eqs. 1-2):
 *        -1/2 ( d(rhoE u_j)/dx_j + rhoE du_j/dx_j + u_j d(rhoE)/dx_j ).
 *      energy_form = 1 evaluates the printed signs, only for the test that
 *      shows the printed form does not conserve total energy.
 *  R2  Eq. 8 is printed implicit and without coefficients.  It is read as the
 *      explicit two-register scheme of Fig. 1 (save Q^n; per stage evaluate R,
 *      update the stage solution, advance the n+1 level) with the
 *      third-order coefficients a = (2/3, 5/12, 3/5) (stage) and
 *      b = (1/4, 3/20, 3/5) (accumulator).
 *  R3  The mixed derivative d2 f/dx_a dx_b (a != b) is D1_a(D1_b f); a pure
 *      second derivative, including d2 u_i/dx_i dx_i inside the stress
 *      divergence, uses the Eq. 7 stencil.
 *  R4  The initial density is not printed: T = 1 everywhere (T_ref from the
 *      equation of state, Eq. 5), so rho = gamma M^2 p.
 *  R5  A velocity amplitude A multiplies u0, u1 and A^2 the pressure
 *      fluctuation (A = 1 is the paper's field).
 *  R6  Grid points x_i = i h, h = 2 pi L / n, no duplicated periodic end point.
 *  R7  KE = <rho |u|^2 / 2>, enstrophy = <rho |omega|^2 / 2> (volume averages,
 *      omega = curl u with Eq. 6); the paper names the quantities only.
 */
#include "sbli_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------- helpers */

static int wrap(int i, int n) {
  int r = i % n;
  return r < 0 ? r + n : r;
}

static size_t npoints(const orc_params* p) { return (size_t)p->n[0] * p->n[1] * p->n[2]; }

static size_t at(const orc_params* p, int i, int j, int k) {
  return (size_t)wrap(i, p->n[0]) + (size_t)p->n[0] * ((size_t)wrap(j, p->n[1]) + (size_t)p->n[1] * wrap(k, p->n[2]));
}

/* index of the point shifted by s along axis a */
static size_t at_shift(const orc_params* p, int i, int j, int k, int a, int s) {
  if (a == 0) return at(p, i + s, j, k);
  if (a == 1) return at(p, i, j + s, k);
  return at(p, i, j, k + s);
}

double orc_h(const orc_params* p, int axis) { return 2.0 * M_PI * p->L / (double)p->n[axis]; }

static double inv_reynolds(const orc_params* p) { return isinf(p->Re) ? 0.0 : 1.0 / p->Re; }

void orc_set_threads(int nthreads) {
#ifdef _OPENMP
  omp_set_num_threads(nthreads > 0 ? nthreads : 1);
#else
  (void)nthreads;
#endif
}

int orc_get_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------- stencils (Eqs. 6 and 7) */

/* Eq. 6: df/dx = ( f_{i-2}/12 - 2 f_{i-1}/3 + 2 f_{i+1}/3 - f_{i+2}/12 ) / h */
static double stencil_d1(double fm2, double fm1, double fp1, double fp2, double h) {
  return (fm2 / 12.0 - 2.0 * fm1 / 3.0 + 2.0 * fp1 / 3.0 - fp2 / 12.0) / h;
}

/* Eq. 7: d2f/dx2 = ( -f_{i-2}/12 + 4 f_{i-1}/3 - 5 f_i/2 + 4 f_{i+1}/3 - f_{i+2}/12 ) / h^2 */
static double stencil_d2(double fm2, double fm1, double f0, double fp1, double fp2, double h) {
  return (-fm2 / 12.0 + 4.0 * fm1 / 3.0 - 5.0 * f0 / 2.0 + 4.0 * fp1 / 3.0 - fp2 / 12.0) / (h * h);
}

void orc_d1(const orc_params* p, const double* f, int axis, double* out) {
  const double h = orc_h(p, axis);
#pragma omp parallel for schedule(static)
  for (int k = 0; k < p->n[2]; ++k)
    for (int j = 0; j < p->n[1]; ++j)
      for (int i = 0; i < p->n[0]; ++i)
        out[at(p, i, j, k)] = stencil_d1(f[at_shift(p, i, j, k, axis, -2)], f[at_shift(p, i, j, k, axis, -1)],
                                         f[at_shift(p, i, j, k, axis, 1)], f[at_shift(p, i, j, k, axis, 2)], h);
}

void orc_d2(const orc_params* p, const double* f, int axis, double* out) {
  const double h = orc_h(p, axis);
#pragma omp parallel for schedule(static)
  for (int k = 0; k < p->n[2]; ++k)
    for (int j = 0; j < p->n[1]; ++j)
      for (int i = 0; i < p->n[0]; ++i)
        out[at(p, i, j, k)] =
            stencil_d2(f[at_shift(p, i, j, k, axis, -2)], f[at_shift(p, i, j, k, axis, -1)], f[at(p, i, j, k)],
                       f[at_shift(p, i, j, k, axis, 1)], f[at_shift(p, i, j, k, axis, 2)], h);
}

/* R3: d2 f / dx_a dx_b = D1_a ( D1_b f ) */
void orc_mixed(const orc_params* p, const double* f, int a, int b, double* out) {
  double* tmp = (double*)malloc(npoints(p) * sizeof(double));
  orc_d1(p, f, b, tmp);
  orc_d1(p, tmp, a, out);
  free(tmp);
}

/* ------------------------------------------------ equation of state (4, 5) */

typedef struct {
  double rho, rhou[3], rhoE, u[3], p, T;
} point_state;

static point_state primitive_at(const orc_params* p, const double* q, size_t n) {
  const size_t P = npoints(p);
  point_state s;
  s.rho = q[n];
  for (int i = 0; i < 3; ++i) s.rhou[i] = q[(size_t)(1 + i) * P + n];
  s.rhoE = q[4 * P + n];
  for (int i = 0; i < 3; ++i) s.u[i] = s.rhou[i] / s.rho;
  /* Eq. 4: p = (gamma - 1)(rho E - rho u_j u_j / 2) */
  s.p = (p->gamma - 1.0) * (s.rhoE - 0.5 * s.rho * (s.u[0] * s.u[0] + s.u[1] * s.u[1] + s.u[2] * s.u[2]));
  /* Eq. 5: T = gamma M^2 p / rho */
  s.T = p->gamma * p->Mach * p->Mach * s.p / s.rho;
  return s;
}

void orc_primitives(const orc_params* p, const double* q, double* u, double* pr, double* T) {
  const size_t P = npoints(p);
#pragma omp parallel for schedule(static)
  for (size_t n = 0; n < P; ++n) {
    point_state s = primitive_at(p, q, n);
    for (int i = 0; i < 3; ++i) u[(size_t)i * P + n] = s.u[i];
    pr[n] = s.p;
    T[n] = s.T;
  }
}

/* --------------------------------------------- residual assembly (Eqs. 1-3) */

/* Every quantity the residual of Eqs. 1-3 needs at one point. */
typedef struct {
  point_state s;
  double d_rhou[3][3];  /* d(rho u_i)/dx_j            [i][j] */
  double d_u[3][3];     /* du_i/dx_j                  [i][j] */
  double d_rho[3];      /* drho/dx_j                  [j]    */
  double d_rhouu[3][3]; /* d(rho u_i u_j)/dx_j        [i][j] */
  double d_p[3];        /* dp/dx_i                    [i]    */
  double d2_u[3][3];    /* d2 u_i/dx_j^2              [i][j] */
  double dd_u[3][3];    /* d2 u_j/dx_i dx_j (R3)      [i][j] */
  double d_rhoE[3];     /* d(rho E)/dx_j              [j]    */
  double d_rhoEu[3];    /* d(rho E u_j)/dx_j          [j]    */
  double d_pu[3];       /* d(p u_j)/dx_j              [j]    */
  double d2_T[3];       /* d2 T/dx_j^2                [j]    */
} local_terms;

static void assemble(const orc_params* p, const local_terms* L, double r[5]) {
  const double inv_re = inv_reynolds(p);
  const double kappa = inv_re / ((p->gamma - 1.0) * p->Mach * p->Mach * p->Pr);
  const point_state* s = &L->s;
  const double div_u = L->d_u[0][0] + L->d_u[1][1] + L->d_u[2][2];

  /* Eq. 1: drho/dt = -1/2 ( d(rho u_j)/dx_j + rho du_j/dx_j + u_j drho/dx_j ) */
  double conv = 0.0;
  for (int j = 0; j < 3; ++j) conv += L->d_rhou[j][j] + s->rho * L->d_u[j][j] + s->u[j] * L->d_rho[j];
  r[0] = -0.5 * conv;

  /* Eq. 2, and the bracket (u_i/Re)(...) of Eq. 3 which repeats it */
  double stress_div[3];
  for (int i = 0; i < 3; ++i) {
    conv = 0.0;
    for (int j = 0; j < 3; ++j) conv += L->d_rhouu[i][j] + s->rhou[i] * L->d_u[j][j] + s->u[j] * L->d_rhou[i][j];
    /* d2 u_i/dx_j^2 + d2 u_j/dx_i dx_j - 2/3 d2 u_k/dx_j dx_k delta_ij,
       the delta_ij contraction leaving the k sum at j = i */
    double lap = 0.0, cross = 0.0, dil = 0.0;
    for (int j = 0; j < 3; ++j) lap += L->d2_u[i][j];
    for (int j = 0; j < 3; ++j) cross += L->dd_u[i][j];
    for (int k = 0; k < 3; ++k) dil += L->dd_u[i][k];
    stress_div[i] = lap + cross - 2.0 / 3.0 * dil;
    r[1 + i] = -0.5 * conv - L->d_p[i] + inv_re * stress_div[i];
  }

  /* Eq. 3 */
  double econv = 0.0;
  if (p->energy_form == 0) {
    /* R1: skew-symmetric reading */
    for (int j = 0; j < 3; ++j) econv += L->d_rhoEu[j] + s->rhoE * L->d_u[j][j] + s->u[j] * L->d_rhoE[j];
  } else {
    /* signs exactly as printed in Eq. 3 */
    for (int j = 0; j < 3; ++j) econv += s->rhoE * L->d_u[j][j] - s->u[j] * L->d_rhoE[j] - L->d_rhoEu[j];
  }
  double pwork = 0.0;
  for (int j = 0; j < 3; ++j) pwork += L->d_pu[j];
  double vwork = 0.0;
  for (int i = 0; i < 3; ++i) vwork += s->u[i] * inv_re * stress_div[i];
  double vdiss = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      vdiss += L->d_u[i][j] * (L->d_u[i][j] + L->d_u[j][i] - (i == j ? 2.0 / 3.0 * div_u : 0.0));
  double heat = 0.0;
  for (int j = 0; j < 3; ++j) heat += L->d2_T[j];
  r[4] = -0.5 * econv - pwork + vwork + inv_re * vdiss + kappa * heat;
}

/* ------------------------------------- full-grid residual, store-all (§2.3.1) */

/* (a) primitives and products into arrays, (b) every derivative into its own
 * array (the BL organisation of §2.3.1), (c) the residual point by point. */
void orc_rhs(const orc_params* p, const double* q, double* r) {
  const size_t P = npoints(p);
  const double* rho = q;
  const double* rhou[3] = {q + P, q + 2 * P, q + 3 * P};
  const double* rhoE = q + 4 * P;

  /* (a) primitives and the products that are differentiated */
  double* u = (double*)malloc(3 * P * sizeof(double));
  double* pr = (double*)malloc(P * sizeof(double));
  double* T = (double*)malloc(P * sizeof(double));
  orc_primitives(p, q, u, pr, T);
  double* rhouu = (double*)malloc(9 * P * sizeof(double)); /* rho u_i u_j [i][j] */
  double* rhoEu = (double*)malloc(3 * P * sizeof(double));
  double* pu = (double*)malloc(3 * P * sizeof(double));
#pragma omp parallel for schedule(static)
  for (size_t n = 0; n < P; ++n) {
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) rhouu[(size_t)(3 * i + j) * P + n] = rhou[i][n] * u[(size_t)j * P + n];
    for (int j = 0; j < 3; ++j) {
      rhoEu[(size_t)j * P + n] = rhoE[n] * u[(size_t)j * P + n];
      pu[(size_t)j * P + n] = pr[n] * u[(size_t)j * P + n];
    }
  }

  /* (b) derivative arrays */
  double* d_rhou = (double*)malloc(9 * P * sizeof(double));
  double* d_u = (double*)malloc(9 * P * sizeof(double));
  double* d_rhouu = (double*)malloc(9 * P * sizeof(double));
  double* d2_u = (double*)malloc(9 * P * sizeof(double));
  double* dd_u = (double*)malloc(9 * P * sizeof(double));
  double* d_rho = (double*)malloc(3 * P * sizeof(double));
  double* d_p = (double*)malloc(3 * P * sizeof(double));
  double* d_rhoE = (double*)malloc(3 * P * sizeof(double));
  double* d_rhoEu = (double*)malloc(3 * P * sizeof(double));
  double* d_pu = (double*)malloc(3 * P * sizeof(double));
  double* d2_T = (double*)malloc(3 * P * sizeof(double));
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      orc_d1(p, rhou[i], j, d_rhou + (size_t)(3 * i + j) * P);
      orc_d1(p, u + (size_t)i * P, j, d_u + (size_t)(3 * i + j) * P);
      orc_d1(p, rhouu + (size_t)(3 * i + j) * P, j, d_rhouu + (size_t)(3 * i + j) * P);
      orc_d2(p, u + (size_t)i * P, j, d2_u + (size_t)(3 * i + j) * P);
    }
  /* R3: dd_u[i][j] = d2 u_j / dx_i dx_j: Eq. 7 when i == j, D1_i(D1_j u_j) otherwise */
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      if (i == j)
        orc_d2(p, u + (size_t)j * P, i, dd_u + (size_t)(3 * i + j) * P);
      else
        orc_d1(p, d_u + (size_t)(3 * j + j) * P, i, dd_u + (size_t)(3 * i + j) * P);
    }
  for (int j = 0; j < 3; ++j) {
    orc_d1(p, rho, j, d_rho + (size_t)j * P);
    orc_d1(p, pr, j, d_p + (size_t)j * P);
    orc_d1(p, rhoE, j, d_rhoE + (size_t)j * P);
    orc_d1(p, rhoEu + (size_t)j * P, j, d_rhoEu + (size_t)j * P);
    orc_d1(p, pu + (size_t)j * P, j, d_pu + (size_t)j * P);
    orc_d2(p, T, j, d2_T + (size_t)j * P);
  }

  /* (c) residual */
#pragma omp parallel for schedule(static)
  for (size_t n = 0; n < P; ++n) {
    local_terms L;
    L.s = primitive_at(p, q, n);
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        const size_t f = (size_t)(3 * i + j) * P + n;
        L.d_rhou[i][j] = d_rhou[f];
        L.d_u[i][j] = d_u[f];
        L.d_rhouu[i][j] = d_rhouu[f];
        L.d2_u[i][j] = d2_u[f];
        L.dd_u[i][j] = dd_u[f];
      }
    for (int j = 0; j < 3; ++j) {
      L.d_rho[j] = d_rho[(size_t)j * P + n];
      L.d_p[j] = d_p[(size_t)j * P + n];
      L.d_rhoE[j] = d_rhoE[(size_t)j * P + n];
      L.d_rhoEu[j] = d_rhoEu[(size_t)j * P + n];
      L.d_pu[j] = d_pu[(size_t)j * P + n];
      L.d2_T[j] = d2_T[(size_t)j * P + n];
    }
    double rr[5];
    assemble(p, &L, rr);
    for (int f = 0; f < 5; ++f) r[(size_t)f * P + n] = rr[f];
  }

  free(u); free(pr); free(T); free(rhouu); free(rhoEu); free(pu);
  free(d_rhou); free(d_u); free(d_rhouu); free(d2_u); free(dd_u);
  free(d_rho); free(d_p); free(d_rhoE); free(d_rhoEu); free(d_pu); free(d2_T);
}

/* ------------------------------------------------ residual at a single point */

enum { Q_RHO, Q_RHOU0, Q_RHOU1, Q_RHOU2, Q_RHOE, Q_U0, Q_U1, Q_U2, Q_P, Q_T,
       Q_RHOUU /* + 3i + j */ = 10, Q_RHOEU /* + j */ = 19, Q_PU /* + j */ = 22 };

/* Value of a primitive or product at a point, computed exactly as orc_rhs
 * computes its arrays. */
static double value_at(const orc_params* p, const double* q, int id, size_t n) {
  const size_t P = npoints(p);
  if (id <= Q_RHOE) return q[(size_t)id * P + n];
  const point_state s = primitive_at(p, q, n);
  if (id <= Q_U2) return s.u[id - Q_U0];
  if (id == Q_P) return s.p;
  if (id == Q_T) return s.T;
  if (id < Q_RHOEU) {
    const int m = id - Q_RHOUU;
    return s.rhou[m / 3] * s.u[m % 3];
  }
  if (id < Q_PU) return s.rhoE * s.u[id - Q_RHOEU];
  return s.p * s.u[id - Q_PU];
}

static double point_d1(const orc_params* p, const double* q, int id, int axis, int i, int j, int k) {
  return stencil_d1(value_at(p, q, id, at_shift(p, i, j, k, axis, -2)), value_at(p, q, id, at_shift(p, i, j, k, axis, -1)),
                    value_at(p, q, id, at_shift(p, i, j, k, axis, 1)), value_at(p, q, id, at_shift(p, i, j, k, axis, 2)),
                    orc_h(p, axis));
}

static double point_d2(const orc_params* p, const double* q, int id, int axis, int i, int j, int k) {
  return stencil_d2(value_at(p, q, id, at_shift(p, i, j, k, axis, -2)), value_at(p, q, id, at_shift(p, i, j, k, axis, -1)),
                    value_at(p, q, id, at(p, i, j, k)), value_at(p, q, id, at_shift(p, i, j, k, axis, 1)),
                    value_at(p, q, id, at_shift(p, i, j, k, axis, 2)), orc_h(p, axis));
}

/* R3 at a point: D1_a applied to the values of D1_b f at the four neighbours */
static double point_mixed(const orc_params* p, const double* q, int id, int a, int b, int i, int j, int k) {
  double v[4];
  const int offs[4] = {-2, -1, 1, 2};
  for (int m = 0; m < 4; ++m) {
    int ii = i, jj = j, kk = k;
    if (a == 0) ii += offs[m];
    else if (a == 1) jj += offs[m];
    else kk += offs[m];
    v[m] = point_d1(p, q, id, b, ii, jj, kk);
  }
  return stencil_d1(v[0], v[1], v[2], v[3], orc_h(p, a));
}

static void local_terms_at(const orc_params* p, const double* q, int i, int j, int k, local_terms* L) {
  L->s = primitive_at(p, q, at(p, i, j, k));
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      L->d_rhou[a][b] = point_d1(p, q, Q_RHOU0 + a, b, i, j, k);
      L->d_u[a][b] = point_d1(p, q, Q_U0 + a, b, i, j, k);
      L->d_rhouu[a][b] = point_d1(p, q, Q_RHOUU + 3 * a + b, b, i, j, k);
      L->d2_u[a][b] = point_d2(p, q, Q_U0 + a, b, i, j, k);
      L->dd_u[a][b] = (a == b) ? point_d2(p, q, Q_U0 + b, a, i, j, k) : point_mixed(p, q, Q_U0 + b, a, b, i, j, k);
    }
  for (int b = 0; b < 3; ++b) {
    L->d_rho[b] = point_d1(p, q, Q_RHO, b, i, j, k);
    L->d_p[b] = point_d1(p, q, Q_P, b, i, j, k);
    L->d_rhoE[b] = point_d1(p, q, Q_RHOE, b, i, j, k);
    L->d_rhoEu[b] = point_d1(p, q, Q_RHOEU + b, b, i, j, k);
    L->d_pu[b] = point_d1(p, q, Q_PU + b, b, i, j, k);
    L->d2_T[b] = point_d2(p, q, Q_T, b, i, j, k);
  }
}

void orc_rhs_point(const orc_params* p, const double* q, int i, int j, int k, double r[5]) {
  local_terms L;
  local_terms_at(p, q, i, j, k, &L);
  assemble(p, &L, r);
}

/* ------------------------------------------- time integration (§2.2, Fig. 1) */

/* R2: stage coefficients a_k and accumulator coefficients b_k */
static const double RK_A[3] = {2.0 / 3.0, 5.0 / 12.0, 3.0 / 5.0};
static const double RK_B[3] = {1.0 / 4.0, 3.0 / 20.0, 3.0 / 5.0};

void orc_rk_coefficients(double a[3], double b[3]) {
  for (int k = 0; k < 3; ++k) {
    a[k] = RK_A[k];
    b[k] = RK_B[k];
  }
}

/* Fig. 1: save Q^n; for each stage evaluate R(Q^k), evaluate Q^{k+1} and
 * advance the n+1 level.  After the third stage Q^{n+1} = Q^3 (a_3 = b_3). */
void orc_lsrk3_step(size_t n, double* q, double dt, orc_rhs_fn f, void* ctx, double* work) {
  double* acc = work;    /* n+1 level being advanced, starts at Q^n */
  double* r = work + n;  /* R(Q^k) */
  memcpy(acc, q, n * sizeof(double));
  for (int k = 0; k < 3; ++k) {
    f(ctx, q, r);
    for (size_t m = 0; m < n; ++m) {
      q[m] = acc[m] + RK_A[k] * dt * r[m];
      acc[m] = acc[m] + RK_B[k] * dt * r[m];
    }
  }
}

void orc_stage(const orc_params* p, int k, double dt, const double* q_in, double* acc, double* q_out) {
  const size_t n = 5 * npoints(p);
  double* r = (double*)malloc(n * sizeof(double));
  orc_rhs(p, q_in, r);
  for (size_t m = 0; m < n; ++m) {
    q_out[m] = acc[m] + RK_A[k] * dt * r[m];
    acc[m] = acc[m] + RK_B[k] * dt * r[m];
  }
  free(r);
}

void orc_stage_point(const orc_params* p, int k, double dt, const double* q_in, const double* acc_in,
                     int i, int j, int kk, double q_out[5], double acc_out[5]) {
  const size_t P = npoints(p);
  const size_t n = at(p, i, j, kk);
  double r[5];
  orc_rhs_point(p, q_in, i, j, kk, r);
  for (int f = 0; f < 5; ++f) {
    const double a = acc_in[(size_t)f * P + n];
    q_out[f] = a + RK_A[k] * dt * r[f];
    acc_out[f] = a + RK_B[k] * dt * r[f];
  }
}

static void ns_rhs(void* ctx, const double* q, double* r) { orc_rhs((const orc_params*)ctx, q, r); }

void orc_step(const orc_params* p, double* q, double dt, int nsteps) {
  const size_t n = 5 * npoints(p);
  double* work = (double*)malloc(2 * n * sizeof(double));
  for (int s = 0; s < nsteps; ++s) orc_lsrk3_step(n, q, dt, ns_rhs, (void*)p, work);
  free(work);
}

/* ------------------------------------------------- Taylor-Green field (§4) */

/* Eqs. 9-12 at global point (i, j, k) with amplitude A (R5): rho, rho u_0..2, rho E */
static void tgv_point(const orc_params* p, double A, int i, int j, int k, double out[5]) {
  const double g = p->gamma, M = p->Mach, L = p->L;
  /* R6: x = i h */
  const double x = i * orc_h(p, 0), y = j * orc_h(p, 1), z = k * orc_h(p, 2);
  const double u0 = A * sin(x / L) * cos(y / L) * cos(z / L);
  const double u1 = -A * cos(x / L) * sin(y / L) * cos(z / L);
  const double u2 = 0.0;
  const double pr = 1.0 / (g * M * M) + A * A / 16.0 * (cos(2.0 * x / L) + cos(2.0 * y / L)) * (2.0 + cos(2.0 * z / L));
  /* R4: T = 1, so rho = gamma M^2 p by Eq. 5 */
  const double rho = g * M * M * pr;
  /* Eq. 4 solved for rho E */
  const double rhoE = pr / (g - 1.0) + 0.5 * rho * (u0 * u0 + u1 * u1 + u2 * u2);
  out[0] = rho;
  out[1] = rho * u0;
  out[2] = rho * u1;
  out[3] = rho * u2;
  out[4] = rhoE;
}

void orc_init_tgv(const orc_params* p, double A, double* q) {
  const size_t P = npoints(p);
#pragma omp parallel for schedule(static)
  for (int k = 0; k < p->n[2]; ++k)
    for (int j = 0; j < p->n[1]; ++j)
      for (int i = 0; i < p->n[0]; ++i) {
        double v[5];
        tgv_point(p, A, i, j, k, v);
        const size_t n = at(p, i, j, k);
        for (int f = 0; f < 5; ++f) q[(size_t)f * P + n] = v[f];
      }
}

void orc_init_tgv_window(const orc_params* p, double A, const int origin[3], const int width[3], double* q) {
  const size_t W = (size_t)width[0] * width[1] * width[2];
  for (int c = 0; c < width[2]; ++c)
    for (int b = 0; b < width[1]; ++b)
      for (int a = 0; a < width[0]; ++a) {
        double v[5];
        /* the periodic image of the window point inside the grid */
        tgv_point(p, A, wrap(origin[0] + a, p->n[0]), wrap(origin[1] + b, p->n[1]), wrap(origin[2] + c, p->n[2]), v);
        const size_t n = (size_t)a + (size_t)width[0] * ((size_t)b + (size_t)width[1] * c);
        for (int f = 0; f < 5; ++f) q[(size_t)f * W + n] = v[f];
      }
}

/* ------------------------------------------------------- diagnostics (R7) */

/* Neumaier-compensated running sum */
typedef struct {
  double s, c;
} csum;

static void csum_add(csum* a, double x) {
  const double t = a->s + x;
  if (fabs(a->s) >= fabs(x))
    a->c += (a->s - t) + x;
  else
    a->c += (x - t) + a->s;
  a->s = t;
}

void orc_ke_enstrophy(const orc_params* p, const double* q, double* ke, double* ens) {
  const size_t P = npoints(p);
  double* u = (double*)malloc(3 * P * sizeof(double));
  double* pr = (double*)malloc(P * sizeof(double));
  double* T = (double*)malloc(P * sizeof(double));
  double* du = (double*)malloc(9 * P * sizeof(double)); /* du_i/dx_j [i][j] */
  orc_primitives(p, q, u, pr, T);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      if (i != j) orc_d1(p, u + (size_t)i * P, j, du + (size_t)(3 * i + j) * P);
  csum k_sum = {0.0, 0.0}, e_sum = {0.0, 0.0};
  for (size_t n = 0; n < P; ++n) {
    const double rho = q[n];
    const double u0 = u[n], u1 = u[P + n], u2 = u[2 * P + n];
    /* omega = curl u */
    const double w0 = du[(size_t)(3 * 2 + 1) * P + n] - du[(size_t)(3 * 1 + 2) * P + n];
    const double w1 = du[(size_t)(3 * 0 + 2) * P + n] - du[(size_t)(3 * 2 + 0) * P + n];
    const double w2 = du[(size_t)(3 * 1 + 0) * P + n] - du[(size_t)(3 * 0 + 1) * P + n];
    csum_add(&k_sum, 0.5 * rho * (u0 * u0 + u1 * u1 + u2 * u2));
    csum_add(&e_sum, 0.5 * rho * (w0 * w0 + w1 * w1 + w2 * w2));
  }
  *ke = (k_sum.s + k_sum.c) / (double)P;
  *ens = (e_sum.s + e_sum.c) / (double)P;
  free(u); free(pr); free(T); free(du);
}
