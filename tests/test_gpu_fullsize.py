"""Parity at the full benchmark sizes, in the launch configurations the
benchmark times.

* 256^3 (the binary64 single-solve workload): one whole step of every path
  (fused binary64, store-all binary64, binary32 and double-float accumulator)
  against one oracle step, every point of every field.
* 512^3 (the precision-comparison workload): stage 0 of each precision on
  sampled points, each sample computed by the oracle's single-point stage from
  the same full-size input, and 200 steps of the binary32 paths against the
  binary64 path on the 64^3 subsample (every 8th point per direction) with the
  per-step kinetic-energy history.

Inputs are the Taylor-Green field of Sec. 4 plus a seeded smooth perturbation
that breaks its symmetries (so that a swapped axis or a wrong neighbour cannot
hide behind them).  Tolerances: 1e-12 for binary64, 1e-5 per field and 1e-6 on
the kinetic-energy history for the binary32 storage paths.
"""
import numpy as np
import pytest

from paper_1709_09713_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1709_09713_gb300 import build

    build.build()
    from paper_1709_09713_gb300 import sbli

    sbli.lib()
    return sbli


def rel_fields(a, b):
    """Per-field relative max-norm error, momentum with a shared denominator."""
    out = []
    mom = max(np.max(np.abs(b[1:4])), 1e-300)
    for f in range(5):
        den = mom if 1 <= f <= 3 else max(np.max(np.abs(b[f])), 1e-300)
        out.append(float(np.max(np.abs(a[f] - b[f])) / den))
    return out


def perturbed_tgv(orc, n, seed):
    p = orc.params(n)
    q = orc.init_tgv(p)
    q += workloads.separable_perturbation(n, seed, 1e-2)
    return p, q


def tuned_or_default(g, tune):
    if tune:
        g.autotune(3)
    return g.config()


# ----------------------------------------------------------------- 256^3
N256, DT256 = 256, 1e-3


@pytest.fixture(scope="module")
def step256(orc):
    p, q0 = perturbed_tgv(orc, N256, seed=256)
    q1 = orc.step(p, q0, DT256, 1)
    return q0, q1


@pytest.mark.parametrize(
    "precision,variant,tune,tol",
    [(0, 0, False, 1e-12), (0, 1, False, 1e-12), (1, 0, True, 1e-5), (2, 0, True, 1e-5), (3, 0, False, 1e-12)],
    ids=["fp64-fused", "fp64-store-all", "fp32-fused", "fp32df-fused", "df64-fused"],
)
def test_256_one_step_every_point(S, step256, precision, variant, tune, tol):
    q0, q1 = step256
    g = S.Grid(N256, precision, variant)
    if variant == S.SBLI_FUSED:
        tuned_or_default(g, tune)
    g.set_state(torch.from_numpy(q0).cuda())
    g.step_n(1, DT256)
    got = g.get_state().cpu().numpy()
    g.close()
    errs = rel_fields(got, q1)
    assert max(errs) <= tol, errs
    # the step moved the state by far more than the tolerance
    assert max(rel_fields(q0, q1)) > 10 * tol


# ----------------------------------------------------------------- 512^3
N512, DT512 = 512, 5e-4  # dt 1e-3 is beyond the RK3 stability limit at 512^3


@pytest.fixture(scope="module")
def input512(orc):
    p, q0 = perturbed_tgv(orc, N512, seed=512)
    rng = np.random.default_rng(5120)
    pts = rng.integers(0, N512, size=(1500, 3))
    # the faces and edges of the periodic box (every wrap direction)
    edge = np.array([[0, 0, 0], [N512 - 1, N512 - 1, N512 - 1], [0, N512 - 1, 1], [N512 - 2, 1, N512 - 1],
                     [1, 0, N512 - 2], [N512 - 1, 0, 0], [0, N512 - 1, 0], [0, 0, N512 - 1]])
    return p, q0, np.concatenate([edge, pts])


@pytest.mark.parametrize(
    "precision,tune,tol,inc_tol",
    [(0, False, 1e-12, 1e-10), (1, True, 1e-5, 5e-3), (2, True, 1e-5, 5e-3), (3, False, 1e-12, 1e-8)],
    ids=["fp64", "fp32", "fp32df", "df64"],
)
def test_512_stage0_sampled(S, orc, input512, precision, tune, tol, inc_tol):
    """Stage outputs against the oracle relative to the field maxima (tol), and
    the stage increment a dt R relative to its own maximum (inc_tol: the
    residual's own accuracy).  In binary32 the energy residual keeps about
    three digits at 512^3: the second-derivative stencil of the temperature
    amplifies its rounding by ~5/h^2 = 3.5e4 while the residual itself is
    small; 1e-3 is what the binary32 path reaches, 5e-3 leaves a margin.
    Double-float arithmetic carries about 48 bits (2^-48 = 3.6e-15, 32 times
    the binary64 unit roundoff), so its increments get 1e-8 where binary64
    gets 1e-10."""
    p, q0, pts = input512
    g = S.Grid(N512, precision, S.SBLI_FUSED)
    tuned_or_default(g, tune)
    g.set_state(torch.from_numpy(q0).cuda())
    g.rk_stage(0, DT512)
    qs, qa = g.get_stage()
    idx = torch.from_numpy(pts).cuda()
    qs = qs[:, idx[:, 2], idx[:, 1], idx[:, 0]].cpu().numpy()
    qa = qa[:, idx[:, 2], idx[:, 1], idx[:, 0]].cpu().numpy()
    g.close()
    del g
    torch.cuda.empty_cache()
    want_s = np.empty_like(qs)
    want_a = np.empty_like(qa)
    for m, (i, j, k) in enumerate(pts):
        want_s[:, m], want_a[:, m] = orc.stage_point(p, 0, DT512, q0, q0, int(i), int(j), int(k))
    q0s = q0[:, pts[:, 2], pts[:, 1], pts[:, 0]]
    # denominators: the field maxima of the input (the stage moves them little)
    den = [np.max(np.abs(q0[0])), *([np.max(np.abs(q0[1:4]))] * 3), np.max(np.abs(q0[4]))]
    inc_err = []
    for f in range(5):
        assert np.max(np.abs(qs[f] - want_s[f])) / den[f] <= tol, (f, "stage field")
        assert np.max(np.abs(qa[f] - want_a[f])) / den[f] <= tol, (f, "accumulator")
        mom = slice(1, 4) if 1 <= f <= 3 else slice(f, f + 1)
        d_want = want_s - q0s
        inc_err.append(float(np.max(np.abs((qs[f] - q0s[f]) - d_want[f])) / np.max(np.abs(d_want[mom]))))
    print("stage-0 increment errors per field", inc_err)
    assert max(inc_err) <= inc_tol, inc_err


def test_512_fp32_paths_against_fp64_200_steps(S):
    """The precision workload: 200 steps at 512^3, dt 5e-4, from the
    Taylor-Green field.  binary32 storage (both accumulator kinds) against the
    binary64 path (itself tied to the oracle above and at small sizes): fields
    on the 64^3 subsample within 1e-5, kinetic-energy history within 1e-6."""
    steps = 200
    sub = (slice(None), slice(None, None, 8), slice(None, None, 8), slice(None, None, 8))
    g = S.Grid(N512, S.SBLI_FP64, S.SBLI_FUSED)
    g.init_tgv()
    h64 = g.step_n_history(steps, DT512).cpu().numpy()
    ref = g.get_state()[sub].cpu().numpy()
    g.close()
    del g
    torch.cuda.empty_cache()
    assert h64[-1, 0] < h64[0, 0]  # the vortex decays
    for precision in (S.SBLI_FP32, S.SBLI_FP32_DF):
        g = S.Grid(N512, precision, S.SBLI_FUSED)
        g.autotune(3)
        g.init_tgv()
        h = g.step_n_history(steps, DT512).cpu().numpy()
        got = g.get_state()[sub].cpu().numpy()
        g.close()
        del g
        torch.cuda.empty_cache()
        errs = rel_fields(got, ref)
        assert max(errs) <= 1e-5, (precision, errs)
        ke_err = np.max(np.abs(h[:, 0] - h64[:, 0]) / np.abs(h64[:, 0]))
        assert ke_err <= 1e-6, (precision, ke_err)
        ens_err = np.max(np.abs(h[:, 1] - h64[:, 1]) / np.abs(h64[:, 1]))
        assert ens_err <= 1e-5, (precision, ens_err)
