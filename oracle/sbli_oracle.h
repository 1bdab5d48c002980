/*
 * sbli_oracle.h -- plain FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline and
 * reference legs may load the library built from this directory.  It shares
 * no code, header, table or constant with the CUDA library under
 * paper_1709_09713_gb300/csrc, and the CUDA library never calls it.
 *
 * What it computes (Jammy, Jacobs, Lusher & Sandham, arXiv:1709.09713):
 *   - the residual R(Q) of the non-dimensional compressible Navier-Stokes
 *     equations, Eqs. 1-3 (§2), skew-symmetric convection and Laplacian
 *     viscous terms, with the equation of state of Eqs. 4-5;
 *   - derivatives by the fourth-order central stencils of Eqs. 6-7 (§2.1),
 *     periodic in all three directions;
 *   - the three-stage low-storage Runge-Kutta update of Eq. 8 / Fig. 1 (§2.2);
 *   - the Taylor-Green vortex initial field of §4 (Eqs. 9-12);
 *   - kinetic energy and enstrophy averages (the quantities of the TGV
 *     validation dataset named in §4).
 *
 * Layout: a field is n0*n1*n2 doubles, x0 fastest (index i + n0*(j + n1*k)),
 * the loop order of Listing 1.  A state Q is 5 consecutive fields
 * (rho, rho*u0, rho*u1, rho*u2, rho*E).
 */
#ifndef SBLI_ORACLE_H
#define SBLI_ORACLE_H
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int n[3];        /* grid points along x0, x1, x2 (each >= 5) */
  double Re;       /* Reynolds number; +INFINITY turns viscous and heat terms off */
  double Mach;     /* reference Mach number M */
  double Pr;       /* Prandtl number */
  double gamma;    /* ratio of specific heats */
  double L;        /* domain is [0, 2*pi*L)^3 */
  int energy_form; /* 0: skew-symmetric energy convection (the reading used);
                      1: the signs as printed in Eq. 3 (kept only so a test can
                         show that reading breaks energy conservation) */
} orc_params;

/* One RHS evaluation callback for the generic Runge-Kutta driver. */
typedef void (*orc_rhs_fn)(void* ctx, const double* q, double* r);

double orc_h(const orc_params* p, int axis);

/* Eq. 6 / Eq. 7 along one axis, and D1_a(D1_b f) for the mixed term. */
void orc_d1(const orc_params* p, const double* f, int axis, double* out);
void orc_d2(const orc_params* p, const double* f, int axis, double* out);
void orc_mixed(const orc_params* p, const double* f, int a, int b, double* out);

/* Eqs. 4-5 over the grid: u (3 fields), pressure, temperature. */
void orc_primitives(const orc_params* p, const double* q, double* u, double* pr, double* T);

/* R(Q) over the whole grid, store-all organisation of §2.3.1. */
void orc_rhs(const orc_params* p, const double* q, double* r);

/* R(Q) at one grid point, every stencil evaluated on the fly; bitwise equal
 * to orc_rhs at that point. */
void orc_rhs_point(const orc_params* p, const double* q, int i, int j, int k, double r[5]);

/* The three-stage low-storage scheme of §2.2 for any right-hand side.
 * work holds 2*n doubles. */
void orc_lsrk3_step(size_t n, double* q, double dt, orc_rhs_fn f, void* ctx, double* work);

/* One stage k (0,1,2) in two-register form:
 *   R = R(q_in);  q_out = acc + a_k*dt*R;  acc = acc + b_k*dt*R.
 * Before stage 0 the caller sets acc = q_in. */
void orc_stage(const orc_params* p, int k, double dt, const double* q_in, double* acc, double* q_out);

/* The same stage at one point (for sampled checks on large grids). */
void orc_stage_point(const orc_params* p, int k, double dt, const double* q_in, const double* acc_in,
                     int i, int j, int kk, double q_out[5], double acc_out[5]);

/* nsteps full time steps of the Navier-Stokes system, in place. */
void orc_step(const orc_params* p, double* q, double dt, int nsteps);

/* The Runge-Kutta coefficients used (stage a_k, accumulator b_k). */
void orc_rk_coefficients(double a[3], double b[3]);

/* Taylor-Green initial field of §4 with velocity amplitude A (A = 1 in the paper). */
void orc_init_tgv(const orc_params* p, double A, double* q);

/* The same field on a width[0] x width[1] x width[2] window of the grid p
 * whose first point is the global point origin (wrapped periodically; the
 * window may be wider than the grid), field-major with x0 fastest.  Each
 * value is the one orc_init_tgv gives the same global point.  With params
 * of n = width and L scaled by width/n, orc_step on the window reproduces
 * the full grid's step at every window point farther than 4 points per
 * stage from the window's edge (the reach of the residual, Eqs. 6-7). */
void orc_init_tgv_window(const orc_params* p, double A, const int origin[3], const int width[3], double* q);

/* Volume averages: ke = <rho |u|^2 / 2>, ens = <rho |omega|^2 / 2>, omega = curl u by Eq. 6. */
void orc_ke_enstrophy(const orc_params* p, const double* q, double* ke, double* ens);

void orc_set_threads(int nthreads);
int orc_get_threads(void);

#ifdef __cplusplus
}
#endif
#endif
