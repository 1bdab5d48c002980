"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test names the fact it pins.  None of them re-derives the oracle's own
formula: they use closed forms of the stencils' Fourier symbols, convergence
orders, discrete conservation identities, symmetries of the Taylor-Green
field, the Runge-Kutta amplification polynomial and an analytic viscous decay
rate.  Together they are chosen so that a dropped term, a wrong sign or
index, or a transposed operand anywhere in the oracle fails at least one.
"""
import math

import numpy as np
import pytest

from paper_1709_09713_gb300 import workloads

GAMMA, MACH, PR, RE = 1.4, 0.1, 0.71, 1600.0


def grid(p):
    """Physical coordinates (x0, x1, x2) broadcast to (n2, n1, n0)."""
    L = p.L
    x = np.arange(p.n[0]) * (2 * math.pi * L / p.n[0])
    y = np.arange(p.n[1]) * (2 * math.pi * L / p.n[1])
    z = np.arange(p.n[2]) * (2 * math.pi * L / p.n[2])
    return x[None, None, :], y[None, :, None], z[:, None, None]


def s1(k, h):
    """Fourier symbol of the Eq. 6 stencil: D1 exp(ikx) = i s1 exp(ikx)."""
    return (8.0 * math.sin(k * h) - math.sin(2 * k * h)) / (6.0 * h)


def lam2(k, h):
    """Minus the Fourier symbol of the Eq. 7 stencil: D2 exp(ikx) = -lam2 exp(ikx)."""
    return (30.0 - 32.0 * math.cos(k * h) + 2.0 * math.cos(2 * k * h)) / (12.0 * h * h)


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


# ---------------------------------------------------------------- T1 symbols

@pytest.mark.parametrize("L", [1.0, 0.5])
def test_T1_stencil_symbols_exact(orc, L):
    """Eq. 6 and Eq. 7 applied to single Fourier modes give exactly the
    closed-form symbols; D1_a(D1_b) gives the product of symbols (R3)."""
    p = orc.params((16, 12, 10), L=L)
    X = grid(p)
    for axis in range(3):
        h = orc.h(p, axis)
        assert h == pytest.approx(2 * math.pi * L / p.n[axis], rel=1e-15)
        for k in (1, 2, 3):
            ph = 0.3
            f = np.sin(k * X[axis] / L + ph) * np.ones((p.n[2], p.n[1], p.n[0]))
            # derivative w.r.t. the physical coordinate x = L * theta
            want1 = s1(k, h / L) / L * np.cos(k * X[axis] / L + ph) * np.ones_like(f)
            want2 = -lam2(k, h / L) / L**2 * f
            assert rel(orc.d1(p, f, axis), want1) < 1e-13
            assert rel(orc.d2(p, f, axis), want2) < 1e-12
    # mixed: d2/dx_a dx_b of sin(x_a) sin(x_b) = s1_a s1_b cos cos
    for a, b in [(0, 1), (1, 2), (0, 2), (2, 0)]:
        ha, hb = orc.h(p, a) / L, orc.h(p, b) / L
        f = np.sin(X[a] / L) * np.sin(2 * X[b] / L) * np.ones((p.n[2], p.n[1], p.n[0]))
        want = s1(1, ha) * s1(2, hb) / L**2 * np.cos(X[a] / L) * np.cos(2 * X[b] / L)
        assert rel(orc.mixed(p, f, a, b), want) < 1e-13


# ----------------------------------------------------------- T2 convergence

def test_T2_fourth_order_convergence(orc):
    """The stencils of Eqs. 6-7 and the mixed D1 o D1 converge at 4th order
    (§2.1) on a smooth non-polynomial periodic function."""
    errs = {"d1": [], "d2": [], "mx": []}
    ns = [32, 64, 128]
    for n in ns:
        p = orc.params((n, n, 5))
        x, y, _ = grid(p)
        g = np.exp(np.sin(x)) * np.exp(np.cos(y)) * np.ones((p.n[2], n, n))
        gx = np.cos(x) * g
        gxx = (np.cos(x) ** 2 - np.sin(x)) * g
        gxy = np.cos(x) * (-np.sin(y)) * g
        errs["d1"].append(np.max(np.abs(orc.d1(p, g, 0) - gx)))
        errs["d2"].append(np.max(np.abs(orc.d2(p, g, 0) - gxx)))
        errs["mx"].append(np.max(np.abs(orc.mixed(p, g, 0, 1) - gxy)))
    for key, e in errs.items():
        slopes = [math.log2(e[i] / e[i + 1]) for i in range(len(e) - 1)]
        assert all(3.8 < s < 4.3 for s in slopes), (key, slopes)


# -------------------------------------------------------------- T3 / T4 conservation

def _state(orc, n, seed, amp=1.0):
    e0 = 1.0 / (GAMMA * (GAMMA - 1.0) * MACH**2) + 0.5
    return workloads.smooth_state(n, seed, offsets=(1.0, 0.0, 0.0, 0.0, e0),
                                  amplitudes=(0.05, 0.5 * amp, 0.5 * amp, 0.5 * amp, 0.5))


def test_T3_mass_momentum_conserved(orc):
    """Skew-symmetric central differences on a periodic grid conserve sum(rho)
    and sum(rho u_i) to round-off (Eqs. 1-2), viscous terms included."""
    p = orc.params((12, 10, 9))
    q = _state(orc, (12, 10, 9), seed=3)
    r = orc.rhs(p, q)
    for f in range(4):
        scale = np.sum(np.abs(r[f])) + 1e-30
        assert abs(np.sum(r[f])) / scale < 1e-13, f
    q2 = orc.step(p, q, 2e-3, 3)
    for f in range(4):
        assert abs(np.sum(q2[f]) - np.sum(q[f])) / np.sum(np.abs(q[f]) + 1) < 1e-14


def test_T4_inviscid_energy_conserved_only_in_skew_reading(orc):
    """With 1/Re = 0, sum(rho E) is conserved to round-off by the skew form
    (reading R1); the signs printed in Eq. 3 are not conservative."""
    n = (12, 10, 9)
    q = _state(orc, n, seed=5)
    p = orc.params(n, Re=orc.INF)
    r = orc.rhs(p, q)
    assert abs(np.sum(r[4])) / np.sum(np.abs(r[4])) < 1e-13
    p_printed = orc.params(n, Re=orc.INF, energy_form=1)
    r_printed = orc.rhs(p_printed, q)
    # eight orders of magnitude above the round-off level of the skew form
    assert abs(np.sum(r_printed[4])) / np.sum(np.abs(r_printed[4])) > 1e-6


def test_T4_viscous_energy_drift_is_fourth_order(orc):
    """With viscosity, the discrete total-energy budget closes only up to
    D2 != D1.D1 on the diagonal: sum(R_rhoE)/P -> 0 at 4th order."""
    vals = []
    for n in (12, 24):
        p = orc.params(n, Re=10.0)
        q = orc.init_tgv(p) + workloads.perturbation(n, seed=9, scale=0.02, kmax=2)
        vals.append(abs(np.mean(orc.rhs(p, q)[4])))
    assert 12.0 < vals[0] / vals[1] < 20.0, vals


# --------------------------------------------- manufactured single-mode RHS pins

def _q_from(rho, mom, e):
    return np.stack([rho, mom[0], mom[1], mom[2], e])


def test_manufactured_uniform_advection(orc):
    """Uniform velocity U, density wave, constant pressure, 1/Re = 0:
    R = -U0 d/dx0 of (rho, rho u, rho E), with the exact symbol s1."""
    n = (16, 6, 5)
    p = orc.params(n, Re=orc.INF)
    x, _, _ = grid(p)
    one = np.ones((n[2], n[1], n[0]))
    eps, U = 0.01, (0.3, -0.2, 0.1)
    rho = (1.0 + eps * np.sin(x)) * one
    p0 = 1.0 / (GAMMA * MACH**2)
    U2 = sum(u * u for u in U)
    e = p0 / (GAMMA - 1.0) + 0.5 * rho * U2
    q = _q_from(rho, [rho * u for u in U], e)
    r = orc.rhs(p, q)
    s = s1(1, orc.h(p, 0))
    wave = eps * s * np.cos(x) * one
    assert np.max(np.abs(r[0] - (-U[0] * wave))) < 1e-12
    for i in range(3):
        assert np.max(np.abs(r[1 + i] - (-U[0] * U[i] * wave))) < 1e-11
    assert np.max(np.abs(r[4] - (-0.5 * U[0] * U2 * wave))) < 1e-10
    # printed Eq. 3 signs advect energy backwards
    r_pr = orc.rhs(orc.params(n, Re=orc.INF, energy_form=1), q)
    assert np.max(np.abs(r_pr[4] - (0.5 * U[0] * U2 * wave))) < 1e-10


def test_manufactured_pressure_wave_and_heat_flux(orc):
    """Fluid at rest, pressure wave along x1: R_rho = 0, R_rho u1 = -dp/dx1,
    R_rhoE = kappa d2T/dx1^2 with T = gamma M^2 p (Eq. 5) and
    kappa = 1/((gamma-1) M^2 Pr Re) (Eq. 3)."""
    n = (5, 16, 6)
    p = orc.params(n)
    _, y, _ = grid(p)
    one = np.ones((n[2], n[1], n[0]))
    eps = 0.05
    p0 = 1.0 / (GAMMA * MACH**2)
    pr = (p0 + eps * np.sin(y)) * one
    q = _q_from(one, [0 * one] * 3, pr / (GAMMA - 1.0))
    r = orc.rhs(p, q)
    h = orc.h(p, 1)
    assert np.max(np.abs(r[0])) < 1e-13
    assert np.max(np.abs(r[1])) < 1e-11 and np.max(np.abs(r[3])) < 1e-11
    assert np.max(np.abs(r[2] - (-eps * s1(1, h) * np.cos(y) * one))) < 1e-11
    kappa = 1.0 / ((GAMMA - 1.0) * MACH**2 * PR * RE)
    want = kappa * GAMMA * MACH**2 * eps * (-lam2(1, h)) * np.sin(y) * one
    assert rel(r[4], want) < 1e-9


def test_manufactured_shear_wave(orc):
    """u1 = eps sin x0: R_rho u1 = (1/Re) D2 u1, and R_rhoE = viscous work
    u1 D2 u1/Re + dissipation (D1 u1)^2/Re, each with its exact symbol."""
    n = (16, 5, 6)
    p = orc.params(n)
    x, _, _ = grid(p)
    one = np.ones((n[2], n[1], n[0]))
    eps = 0.1
    p0 = 1.0 / (GAMMA * MACH**2)
    u1 = eps * np.sin(x) * one
    q = _q_from(one, [0 * one, u1, 0 * one], p0 / (GAMMA - 1.0) + 0.5 * u1 * u1)
    r = orc.rhs(p, q)
    h = orc.h(p, 0)
    assert np.max(np.abs(r[0])) < 1e-13
    assert rel(r[2], -lam2(1, h) * u1 / RE) < 1e-9
    want_e = (eps**2 / RE) * (s1(1, h) ** 2 * np.cos(x) ** 2 - lam2(1, h) * np.sin(x) ** 2) * one
    assert np.max(np.abs(r[4] - want_e)) < 1e-9 * np.max(np.abs(want_e)) + 1e-11


def test_manufactured_dilatation(orc):
    """u0 = eps sin x0: the stress divergence is (4/3) D2 u0 (reading R3 puts
    Eq. 7 on the diagonal of d2u_j/dx_i dx_j); convection is
    -(eps^2/4)(s1(2) + 2 s1(1)) sin 2x0."""
    n = (16, 5, 5)
    p = orc.params(n)
    x, _, _ = grid(p)
    one = np.ones((n[2], n[1], n[0]))
    eps = 0.1
    p0 = 1.0 / (GAMMA * MACH**2)
    u0 = eps * np.sin(x) * one
    q = _q_from(one, [u0, 0 * one, 0 * one], p0 / (GAMMA - 1.0) + 0.5 * u0 * u0)
    r = orc.rhs(p, q)
    h = orc.h(p, 0)
    assert np.max(np.abs(r[0] - (-eps * s1(1, h) * np.cos(x) * one))) < 1e-13
    want = (-(eps**2) / 4.0 * (s1(2, h) + 2 * s1(1, h)) * np.sin(2 * x) - 4.0 / 3.0 * lam2(1, h) * u0 / RE) * one
    assert np.max(np.abs(r[1] - want)) < 1e-11


def test_manufactured_mixed_derivative(orc):
    """u1 = eps sin x0 sin x1: R_rho u0 = (1/3Re) D1_0 D1_1 u1 (mixed term,
    R3) and R_rho u1 = convection - (7/3) lam2 u1 / Re."""
    n = (12, 16, 5)
    p = orc.params(n)
    x, y, _ = grid(p)
    one = np.ones((n[2], n[1], n[0]))
    eps = 0.1
    p0 = 1.0 / (GAMMA * MACH**2)
    u1 = eps * np.sin(x) * np.sin(y) * one
    q = _q_from(one, [0 * one, u1, 0 * one], p0 / (GAMMA - 1.0) + 0.5 * u1 * u1)
    r = orc.rhs(p, q)
    hx, hy = orc.h(p, 0), orc.h(p, 1)
    want0 = eps * s1(1, hx) * s1(1, hy) * np.cos(x) * np.cos(y) / (3.0 * RE) * one
    assert np.max(np.abs(r[1] - want0)) < 1e-12
    conv = -(eps**2) / 4.0 * (s1(2, hy) + 2 * s1(1, hy)) * np.sin(x) ** 2 * np.sin(2 * y)
    visc = -(lam2(1, hx) + lam2(1, hy) + lam2(1, hy) / 3.0) * u1 / RE
    assert np.max(np.abs(r[2] - (conv + visc) * one)) < 1e-11


# ------------------------------------------------------------ T5 symmetries

def test_T5_translation_equivariance_bitwise(orc):
    """The periodic scheme commutes with grid translations bit for bit
    (a wrong wrap index near the boundary breaks this)."""
    n = (10, 8, 7)
    p = orc.params(n)
    q = _state(orc, n, seed=11)
    r = orc.rhs(p, q)
    for shift in [(3, 0, 0), (0, 5, 0), (0, 0, 6), (9, 7, 1)]:
        qs = np.roll(q, shift=(shift[2], shift[1], shift[0]), axis=(1, 2, 3))
        rs = orc.rhs(p, qs)
        assert np.array_equal(rs, np.roll(r, shift=(shift[2], shift[1], shift[0]), axis=(1, 2, 3)))


def test_T5_tgv_symmetries_preserved(orc):
    """The TGV (§4) is invariant under half-period shifts in two directions,
    under x0 -> -x0 with u0 odd, and under the swap-plus-shift isometry
    (x0, x1) -> (x1 + pi, x0) with (u0, u1) swapped; the scheme keeps all of
    them over time steps (to round-off)."""
    n = 16
    p = orc.params(n)
    q = orc.step(p, orc.init_tgv(p), 2e-3, 3)
    h = n // 2
    for sh in [(h, h, 0), (h, 0, h), (0, h, h)]:
        qs = np.roll(q, shift=(sh[2], sh[1], sh[0]), axis=(1, 2, 3))
        for f in range(5):
            assert rel(qs[f], q[f]) < 1e-12 or np.max(np.abs(qs[f] - q[f])) < 1e-13
    # reflection x0 -> -x0: index i -> (-i) mod n
    idx = (-np.arange(n)) % n
    qr = q[:, :, :, idx].copy()
    qr[1] *= -1.0
    for f in range(5):
        assert np.max(np.abs(qr[f] - q[f])) < 1e-12 * max(1.0, np.max(np.abs(q[f])))
    # swap-plus-shift: value at (i, j, k) equals the (u0 <-> u1)-swapped value at (j + n/2, i, k)
    qsw = np.empty_like(q)
    J, I = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    for f in range(5):
        qsw[f] = q[f][:, I, (J + h) % n]
    tmp = qsw[1].copy()
    qsw[1] = qsw[2]
    qsw[2] = tmp
    for f in range(5):
        assert np.max(np.abs(qsw[f] - q[f])) < 1e-12 * max(1.0, np.max(np.abs(q[f])))


# ------------------------------------------------------------------- T6 RK

def test_T6_rk_amplification_polynomial(orc):
    """For dq/dt = lambda q one step multiplies by 1 + z + z^2/2 + z^3/6,
    z = lambda dt (a three-stage third-order scheme, §2.2); a rotation
    (imaginary lambda) checks the complex case."""
    for lam, dt in [(-1.7, 0.3), (0.8, 0.25), (-10.0, 0.05)]:
        z = lam * dt
        q = orc.lsrk3_step(np.array([1.0, -2.0]), dt, lambda v: lam * v)
        assert np.allclose(q, np.array([1.0, -2.0]) * (1 + z + z * z / 2 + z**3 / 6), rtol=1e-14, atol=0)
    w, dt = 2.0, 0.4
    Jm = np.array([[0.0, -w], [w, 0.0]])
    q = orc.lsrk3_step(np.array([1.0, 0.5]), dt, lambda v: Jm @ v)
    Z = Jm * dt
    G = np.eye(2) + Z + Z @ Z / 2 + Z @ Z @ Z / 6
    assert np.allclose(q, G @ np.array([1.0, 0.5]), rtol=1e-14, atol=1e-15)


def test_T6_rk_third_order_nonlinear(orc):
    """On a nonlinear ODE the global error falls as dt^3."""
    a, b = orc.rk_coefficients()
    assert a[2] == b[2]
    f = lambda v: np.array([v[1], -math.sin(v[0]) - 0.1 * v[1] * v[0] ** 2])
    T = 2.0
    errs = []
    ref = None
    for nsteps in (640, 20, 40, 80):
        q = np.array([1.0, 0.0])
        dt = T / nsteps
        for _ in range(nsteps):
            q = orc.lsrk3_step(q, dt, f)
        if ref is None:
            ref = q
        else:
            errs.append(np.max(np.abs(q - ref)))
    slopes = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(2.8 < s < 3.3 for s in slopes), slopes


# ------------------------------------------------------- T7 closed forms

@pytest.mark.parametrize("n,A", [(8, 1.0), (16, 1.0), (32, 1.0), (16, 0.9)])
def test_T7_initial_ke_and_enstrophy(orc, n, A):
    """Initial KE = A^2/8 exactly on the grid; initial enstrophy with omega
    from Eq. 6 is s1(1)^2/2 (3A^2/4 - 5 gamma M^2 A^4/64) (the density
    correlation term comes from rho = gamma M^2 p, reading R4)."""
    p = orc.params(n)
    q = orc.init_tgv(p, A)
    ke, ens = orc.ke_enstrophy(p, q)
    assert ke == pytest.approx(A * A / 8.0, rel=1e-13)
    s = s1(1, orc.h(p, 0))
    want = 0.5 * s * s * (0.75 * A * A - 5.0 * GAMMA * MACH**2 * A**4 / 64.0)
    assert ens == pytest.approx(want, rel=1e-12)


def test_T7_initial_field_values(orc):
    """Eqs. 9-12 at a grid point, with T = 1 (R4)."""
    p = orc.params(8)
    q = orc.init_tgv(p)
    x, y, z = 1 * 2 * math.pi / 8, 2 * 2 * math.pi / 8, 3 * 2 * math.pi / 8
    u0 = math.sin(x) * math.cos(y) * math.cos(z)
    u1 = -math.cos(x) * math.sin(y) * math.cos(z)
    pr = 1 / (GAMMA * MACH**2) + (math.cos(2 * x) + math.cos(2 * y)) * (2 + math.cos(2 * z)) / 16
    rho = GAMMA * MACH**2 * pr
    assert q[0, 3, 2, 1] == pytest.approx(rho, rel=1e-15)
    assert q[1, 3, 2, 1] == pytest.approx(rho * u0, rel=1e-14, abs=1e-16)
    assert q[2, 3, 2, 1] == pytest.approx(rho * u1, rel=1e-14, abs=1e-16)
    assert q[3, 3, 2, 1] == 0.0
    assert q[4, 3, 2, 1] == pytest.approx(pr / (GAMMA - 1) + 0.5 * rho * (u0**2 + u1**2), rel=1e-15)
    u, prim_p, T = orc.primitives(p, q)
    assert np.max(np.abs(T - 1.0)) < 1e-13


@pytest.mark.parametrize("A", [1.0, 0.7])
def test_T7_initial_total_energy_and_pressure(orc, A):
    """Mean total energy of the initial field is 1/(gamma (gamma-1) M^2) +
    A^2/8 (the pressure fluctuation of Eq. 12 averages to zero on the grid,
    the kinetic part is A^2/8), and the pressure recovered through Eq. 4 is
    Eq. 12 at every point."""
    p = orc.params(12)
    q = orc.init_tgv(p, A)
    want = 1.0 / (GAMMA * (GAMMA - 1.0) * MACH**2) + A * A / 8.0
    assert float(np.mean(q[4])) == pytest.approx(want, rel=1e-14)
    x, y, z = grid(p)
    pr = 1 / (GAMMA * MACH**2) + A * A * (np.cos(2 * x) + np.cos(2 * y)) * (2 + np.cos(2 * z)) / 16
    _, prim_p, _ = orc.primitives(p, q)
    assert rel(prim_p, pr) < 1e-13


@pytest.mark.parametrize("a", [0, 1, 2])
def test_T7_enstrophy_of_a_shear_pair(orc, a):
    """With axes (a, b, c) cyclic, u_b = -sin(x_b + x_c), u_c = sin(x_b + x_c)
    and u_a = 0 is solenoidal and its only vorticity component is
    omega_a = du_c/dx_b - du_b/dx_c = 2 cos(x_b + x_c); with Eq. 6 each
    derivative carries s1(1), so at rho = 1 the enstrophy is s1(1)^2 and the
    kinetic energy 1/2.  Both terms of omega_a are nonzero and equal, so a
    sign slip inside the curl halves or cancels it (the Taylor-Green field,
    with one nonzero term per component, cannot show that)."""
    p = orc.params(10)
    X = grid(p)
    b, c = (a + 1) % 3, (a + 2) % 3
    phase = X[b] + X[c] + np.zeros((10, 10, 10))
    q = np.zeros((5, 10, 10, 10))
    q[0] = 1.0
    q[1 + b] = -np.sin(phase)
    q[1 + c] = np.sin(phase)
    q[4] = 1.0 / (GAMMA * (GAMMA - 1.0) * MACH**2) + 0.5 * (q[1 + b] ** 2 + q[1 + c] ** 2)
    ke, ens = orc.ke_enstrophy(p, q)
    assert ke == pytest.approx(0.5, rel=1e-14)
    assert ens == pytest.approx(s1(1, orc.h(p, 0)) ** 2, rel=1e-13)


@pytest.mark.parametrize("n", [(9, 10, 11), (12, 8, 10)])
def test_T7_enstrophy_identity_random_field(orc, n):
    """For any periodic velocity at rho = 1, sum |omega|^2 = sum |D u|^2 -
    sum (D . u)^2 holds for the Eq. 6 operators exactly up to rounding:
    the cross sum (D_j u_i)(D_i u_j) equals sum (D_i u_i)(D_j u_j) because
    the periodic stencils commute and are skew-adjoint (summation by parts).
    The right side uses only first derivatives, never the curl, so a sign or
    index slip in any vorticity component breaks the identity."""
    p = orc.params(n)
    # the three components share their wavevectors (random amplitudes and
    # phases each), so every cross product D_b u_c * D_c u_b has a nonzero sum
    rng = np.random.default_rng(41)
    X = grid(p)
    q = np.zeros((5, n[2], n[1], n[0]))
    q[0] = 1.0
    q[4] = 180.0
    for _ in range(8):
        k = rng.integers(-3, 4, size=3)
        if not k.any():
            k[0] = 1
        phase = k[0] * X[0] + k[1] * X[1] + k[2] * X[2]
        for i in range(3):
            q[1 + i] += rng.uniform(0.1, 0.3) * np.cos(phase + rng.uniform(0.0, 2.0 * math.pi))
    _, ens = orc.ke_enstrophy(p, q)
    du = [[orc.d1(p, np.ascontiguousarray(q[1 + i]), j) for j in range(3)] for i in range(3)]
    grad2 = sum(float(np.mean(du[i][j] ** 2)) for i in range(3) for j in range(3))
    div2 = float(np.mean((du[0][0] + du[1][1] + du[2][2]) ** 2))
    assert 2.0 * ens == pytest.approx(grad2 - div2, rel=1e-12)
    assert div2 > 0.1 * grad2  # the random field is not solenoidal: the identity is not trivial


# ------------------------------------------------------- T8 viscous decay

def test_T8_low_reynolds_kinetic_energy_decay(orc):
    """At low Re and small amplitude the TGV decays like a linear viscous
    mode: KE(t) = KE(0) exp(-6 nu lam2(1) t), lam2 the Eq. 7 symbol."""
    n, Re, A, dt, nsteps = 12, 20.0, 1e-3, 2e-3, 100
    p = orc.params(n, Re=Re)
    q = orc.init_tgv(p, A)
    ke0, ens0 = orc.ke_enstrophy(p, q)
    q = orc.step(p, q, dt, nsteps)
    ke, ens = orc.ke_enstrophy(p, q)
    t = dt * nsteps
    want = ke0 * math.exp(-6.0 * lam2(1, orc.h(p, 0)) * t / Re)
    assert ke == pytest.approx(want, rel=2e-4)
    # dKE/dt = -(2/Re) enstrophy at t = 0, up to the symbol ratio lam2/s1^2
    s = s1(1, orc.h(p, 0))
    rate = -6.0 * lam2(1, orc.h(p, 0)) / Re * ke0
    assert rate == pytest.approx(-2.0 / Re * ens0 * lam2(1, orc.h(p, 0)) / s**2, rel=2e-3)


# ----------------------------------------------------- T9 brute force (tiny grids)

def _dense_d1(n, h):
    D = np.zeros((n, n))
    for i in range(n):
        for off, c in [(-2, 1 / 12), (-1, -2 / 3), (1, 2 / 3), (2, -1 / 12)]:
            D[i, (i + off) % n] += c / h
    return D


def _dense_d2(n, h):
    D = np.zeros((n, n))
    for i in range(n):
        for off, c in [(-2, -1 / 12), (-1, 4 / 3), (0, -5 / 2), (1, 4 / 3), (2, -1 / 12)]:
            D[i, (i + off) % n] += c / (h * h)
    return D


def _brute_rhs(q, n, Re, M, Pr, g):
    """Eqs. 1-3 evaluated term by term with dense derivative matrices."""
    hs = [2 * math.pi / m for m in n]
    D1 = [_dense_d1(n[a], hs[a]) for a in range(3)]
    D2 = [_dense_d2(n[a], hs[a]) for a in range(3)]
    # field arrays are (z, y, x): axis a of the method is numpy axis 2 - a
    def d1(f, a):
        return np.moveaxis(np.tensordot(D1[a], f, axes=([1], [2 - a])), 0, 2 - a)

    def d2(f, a):
        return np.moveaxis(np.tensordot(D2[a], f, axes=([1], [2 - a])), 0, 2 - a)

    rho, m, E = q[0], q[1:4], q[4]
    u = m / rho
    p = (g - 1) * (E - 0.5 * rho * np.sum(u * u, axis=0))
    T = g * M * M * p / rho
    div = sum(d1(u[j], j) for j in range(3))

    def dd(j, i):  # d2 u_j / dx_i dx_j, reading R3
        return d2(u[j], i) if i == j else d1(d1(u[j], j), i)

    r = np.zeros_like(q)
    r[0] = -0.5 * sum(d1(m[j], j) + rho * d1(u[j], j) + u[j] * d1(rho, j) for j in range(3))
    sd = []
    for i in range(3):
        conv = sum(d1(m[i] * u[j], j) + m[i] * d1(u[j], j) + u[j] * d1(m[i], j) for j in range(3))
        s = sum(d2(u[i], j) for j in range(3)) + sum(dd(j, i) for j in range(3)) - 2 / 3 * sum(dd(k, i) for k in range(3))
        sd.append(s)
        r[1 + i] = -0.5 * conv - d1(p, i) + s / Re
    conv = sum(d1(E * u[j], j) + E * d1(u[j], j) + u[j] * d1(E, j) for j in range(3))
    work = sum(u[i] * sd[i] for i in range(3)) / Re
    diss = sum(d1(u[i], j) * (d1(u[i], j) + d1(u[j], i) - (2 / 3 * div if i == j else 0)) for i in range(3) for j in range(3))
    heat = sum(d2(T, j) for j in range(3)) / ((g - 1) * M * M * Pr * Re)
    r[4] = -0.5 * conv - sum(d1(p * u[j], j) for j in range(3)) + work + diss / Re + heat
    return r


@pytest.mark.parametrize("n", [(5, 5, 5), (5, 6, 7), (8, 6, 5)])
def test_T9_brute_force_tiny_grids(orc, n):
    """On the smallest grids the 5-point stencils allow, the oracle equals a
    dense-matrix term-by-term evaluation of Eqs. 1-3."""
    p = orc.params(n, Re=50.0)
    q = _state(orc, n, seed=sum(n))
    r = orc.rhs(p, q)
    rb = _brute_rhs(q, n, 50.0, MACH, PR, GAMMA)
    for f in range(5):
        assert rel(r[f], rb[f]) < 1e-11, f


def test_point_and_grid_rhs_agree_bitwise(orc):
    """The per-point evaluation used for sampled checks on large grids is the
    same arithmetic as the full-grid one."""
    n = (9, 7, 6)
    p = orc.params(n)
    q = _state(orc, n, seed=1)
    r = orc.rhs(p, q)
    for (i, j, k) in [(0, 0, 0), (8, 6, 5), (4, 1, 3), (1, 6, 0)]:
        assert np.array_equal(orc.rhs_point(p, q, i, j, k), r[:, k, j, i])
    acc = q + 0.01
    qo, ao = orc.stage(p, 1, 1e-3, q, acc)
    for (i, j, k) in [(0, 0, 0), (5, 3, 2)]:
        qp, ap = orc.stage_point(p, 1, 1e-3, q, acc, i, j, k)
        assert np.array_equal(qp, qo[:, k, j, i]) and np.array_equal(ap, ao[:, k, j, i])


def test_stage_chain_equals_rk_driver_bitwise(orc):
    """The single-stage oracle used for per-stage GPU parity, chained over
    stages 0, 1, 2, is the pinned three-stage driver (T6) bit for bit."""
    n = (9, 8, 7)
    p = orc.params(n, Re=200.0)
    q0 = _state(orc, n, seed=31)
    acc, q = q0.copy(), q0.copy()
    for k in range(3):
        q, acc = orc.stage(p, k, 2e-3, q, acc)
    assert np.array_equal(acc, orc.step(p, q0, 2e-3, 1))
    assert np.array_equal(q, acc)


def test_oracle_matches_its_golden_fixture(orc):
    """The oracle's 32^3 Taylor-Green history and sampled final state against
    tests/golden/tgv32_oracle.txt (written by tests/golden/make_golden.py from
    the oracle alone): guards the oracle's arithmetic against silent change.
    Tolerance 1e-13: the fixture holds exact decimal reprs, the only freedom is
    the thread partition of the oracle's compensated sums."""
    import os

    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "tgv32_oracle.txt")
    hist, pts = [], []
    for line in open(path):
        tok = line.split()
        if not tok or tok[0].startswith("#"):
            continue
        if tok[0] == "h":
            hist.append((float(tok[2]), float(tok[3])))
        elif tok[0] == "q":
            pts.append(((int(tok[1]), int(tok[2]), int(tok[3])), [float(x) for x in tok[4:9]]))
    assert len(hist) == 10 and len(pts) == 6
    p = orc.params(32)
    q = orc.init_tgv(p)
    for s in range(10):
        ke, ens = orc.ke_enstrophy(p, q)
        assert ke == pytest.approx(hist[s][0], rel=1e-13) and ens == pytest.approx(hist[s][1], rel=1e-13)
        q = orc.step(p, q, 1e-3, 1)
    for (i, j, k), want in pts:
        for f in range(5):
            assert q[f, k, j, i] == pytest.approx(want[f], rel=1e-13, abs=1e-15)


# ------------------------------------------------- windows of large grids

@pytest.mark.parametrize("origin,width", [((0, 0, 0), (12, 10, 9)), ((-3, 8, 7), (7, 6, 5)), ((5, -11, 20), (25, 4, 3))])
def test_window_init_is_the_grid_init_on_the_window(orc, origin, width):
    """Each window value is bitwise the full grid's value at the periodic image
    of its global point (windows may wrap, start negative, or be wider than
    the grid)."""
    p = orc.params((12, 10, 9))
    full = orc.init_tgv(p, 0.9)
    win = orc.init_tgv_window(p, 0.9, origin, width)
    ii = (origin[0] + np.arange(width[0])) % 12
    jj = (origin[1] + np.arange(width[1])) % 10
    kk = (origin[2] + np.arange(width[2])) % 9
    want = full[:, kk[:, None, None], jj[None, :, None], ii[None, None, :]]
    assert np.array_equal(win, want)


def test_window_step_reproduces_the_grid_step_at_its_centre(orc):
    """One step on a 25^3 window (reach 3 stages x 4 points = 12 each side)
    with the grid's spacing gives the full grid's step at the window centre:
    the dependency cone of the centre never meets the window's wrap.  Not
    bitwise: the window's h = 2 pi (L w/n)/w may differ from 2 pi L/n in the
    last bit."""
    p = orc.params(20)
    dt = 1e-3
    full = orc.step(p, orc.init_tgv(p), dt, 1)
    pw = orc.window_params(p, (25, 25, 25))
    assert orc.h(pw, 0) == pytest.approx(orc.h(p, 0), rel=1e-15)
    for c in [(0, 0, 0), (19, 3, 11), (7, 19, 19)]:
        origin = tuple(v - 12 for v in c)
        win = orc.step(pw, orc.init_tgv_window(p, 1.0, origin, (25, 25, 25)), dt, 1)
        got = win[:, 12, 12, 12]
        want = full[:, c[2], c[1], c[0]]
        assert np.max(np.abs(got - want) / np.array([1.0, 1.0, 1.0, 1.0, 200.0])) < 1e-14, (c, got - want)
    # an off-centre window point inside the reach of the wrap does differ
    win = orc.step(pw, orc.init_tgv_window(p, 1.0, (-12, -12, -12), (25, 25, 25)), dt, 1)
    assert np.max(np.abs(win[:, 12, 12, 1] - full[:, 0, 0, 9])) > 1e-8
