"""Batched ensembles (one persistent launch per stage over all members,
graph-captured step loops): every member's result is bitwise the result of
the same problem run alone, and the alone result is tied to the oracle by
test_gpu_parity."""
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


SIZES = [(32, 32, 32), (48, 48, 48), (20, 16, 12), (64, 40, 24), (5, 6, 7)]
RE = [1600.0, 300.0, 100.0, 900.0, 50.0]
MACH = [0.1, 0.25, 0.4, 0.15, 0.3]
AMP = [1.0, 0.95, 1.08, 0.9, 1.02]


@pytest.mark.parametrize("precision", [0, 1, 2, 3])
def test_batch_members_equal_single_grids_bitwise(S, precision):
    dt, steps = 1e-3, 7  # one captured 6-step graph plus one direct step
    b = S.Batch(SIZES, precision, Re=RE, Mach=MACH)
    b.init_tgv(AMP)
    b.step_n(steps, dt)
    for m, n in enumerate(SIZES):
        g = S.Grid(n, precision, S.SBLI_FUSED, Re=RE[m], Mach=MACH[m])
        g.set_config(8, min(32, n[2]))
        g.init_tgv(AMP[m])
        g.step_n(steps, dt)
        assert torch.equal(b.get_state(m), g.get_state()), m


@pytest.mark.parametrize("precision", [0, 3])
def test_batch_matches_oracle_fp64(S, orc, precision):
    """binary64 and double-float arithmetic members against the oracle."""
    dt, steps = 1e-3, 3
    b = S.Batch(SIZES[:3], precision, Re=RE[:3], Mach=MACH[:3])
    b.init_tgv(AMP[:3])
    b.step_n(steps, dt)
    for m, n in enumerate(SIZES[:3]):
        p = orc.params(n, Re=RE[m], Mach=MACH[m])
        want = orc.step(p, orc.init_tgv(p, AMP[m]), dt, steps)
        got = b.get_state(m).cpu().numpy()
        mom = np.max(np.abs(want[1:4]))
        for f in range(5):
            den = mom if 1 <= f <= 3 else np.max(np.abs(want[f]))
            assert np.max(np.abs(got[f] - want[f])) / den <= 1e-12, (m, f)


@pytest.mark.parametrize("prec", [1, 2])
def test_batch_history_and_set_state(S, prec):
    dt, steps = 1e-3, 3
    sizes = SIZES[:4]
    b = S.Batch(sizes, prec, Re=RE[:4], Mach=MACH[:4])
    rng = np.random.default_rng(5)
    for m, n in enumerate(sizes):
        e0 = 1.0 / (1.4 * 0.4 * MACH[m] ** 2) + 0.5
        q = workloads.smooth_state(n, 40 + m, offsets=(1.0, 0, 0, 0, e0), amplitudes=(0.05, 0.3, 0.3, 0.3, 0.3))
        b.set_state(m, torch.from_numpy(q).cuda())
    hist = b.step_n_history(steps, dt).cpu().numpy()
    ke, ens = b.kinetic_energy()
    for m, n in enumerate(sizes):
        g = S.Grid(n, prec, S.SBLI_FUSED, Re=RE[m], Mach=MACH[m])
        e0 = 1.0 / (1.4 * 0.4 * MACH[m] ** 2) + 0.5
        q = workloads.smooth_state(n, 40 + m, offsets=(1.0, 0, 0, 0, e0), amplitudes=(0.05, 0.3, 0.3, 0.3, 0.3))
        g.set_state(torch.from_numpy(q).cuda())
        h = g.step_n_history(steps, dt).cpu().numpy()
        assert np.allclose(hist[:, m, :], h, rtol=1e-12, atol=0)
        k1, e1 = g.kinetic_energy()
        assert ke[m] == pytest.approx(k1, rel=1e-13) and ens[m] == pytest.approx(e1, rel=1e-13)
        assert torch.equal(b.get_state(m), g.get_state())


def test_batch_ensemble_draws_build(S):
    members = workloads.ensemble(8, seed=1709, sizes=(32, 48))
    b = S.Batch([mm.n for mm in members], 1, Re=[mm.Re for mm in members], Mach=[mm.Mach for mm in members])
    b.init_tgv([mm.amplitude for mm in members])
    b.step_n(2, 1e-3)
    ke, _ = b.kinetic_energy()
    assert all(np.isfinite(ke)) and all(k > 0 for k in ke)
    with pytest.raises(S.SbliError):
        S.sbli_batch_workspace_bytes([(4, 8, 8)], 1)


@pytest.mark.parametrize("prec", [1, 2])
def test_full_ensemble_against_single_grids_and_oracle(S, orc, prec):
    """The benchmarked ensemble itself: 64 Taylor-Green members (N uniform
    over {32, 48, 64, 96, 128}, Re ~ U[100, 1600], M ~ U[0.1, 0.4], amplitude
    ~ U(0.9, 1.1), seed 1709), binary32 stages with a binary64 accumulator,
    one persistent launch per stage.  After one step every member equals the
    same problem solved alone, bit for bit, and sampled points of every
    member (corners and random points) match one oracle step on a 25^3
    window around them (the reach of one step is 12 points per side) within
    the binary32 bar."""
    dt = 1e-3
    members = workloads.ensemble(64, seed=1709)
    b = S.Batch([m.n for m in members], prec, Re=[m.Re for m in members], Mach=[m.Mach for m in members])
    b.init_tgv([m.amplitude for m in members])
    b.step_n(1, dt)
    rng = np.random.default_rng(64)
    worst = 0.0
    for k, m in enumerate(members):
        got = b.get_state(k)
        g = S.Grid(m.n, prec, S.SBLI_FUSED, Re=m.Re, Mach=m.Mach)
        g.init_tgv(m.amplitude)
        g.step_n(1, dt)
        assert torch.equal(got, g.get_state()), k
        g.close()
        q = got.cpu().numpy()
        p = orc.params(m.n, Re=m.Re, Mach=m.Mach)
        pw = orc.window_params(p, (25, 25, 25))
        pts = [(0, 0, 0), (m.n - 1, m.n - 1, m.n - 1)] + [tuple(int(v) for v in rng.integers(0, m.n, 3)) for _ in range(4)]
        want = np.empty((5, len(pts)))
        for s, (i, j, kk) in enumerate(pts):
            win = orc.init_tgv_window(p, m.amplitude, (i - 12, j - 12, kk - 12), (25, 25, 25))
            want[:, s] = orc.step(pw, win, dt, 1)[:, 12, 12, 12]
        have = np.stack([q[:, kk, j, i] for (i, j, kk) in pts], axis=1)
        mom = np.max(np.abs(want[1:4]))
        for f in range(5):
            den = mom if 1 <= f <= 3 else np.max(np.abs(want[f]))
            err = float(np.max(np.abs(have[f] - want[f])) / den)
            worst = max(worst, err)
            assert err <= 1e-5, (k, m, f, err)
    b.close()
    print(f"64-member ensemble, precision {prec}, one step: worst sampled field error {worst:.2e}")


@pytest.mark.parametrize("precision", [0, 1, 2, 3])
def test_batch_of_extreme_shapes_equals_single_grids(S, precision):
    """Members long in one axis and at the 5-point minimum in the others
    (partial tiles in x0 and x1, z chunks from 5 to 300 planes) in one
    persistent launch: each equals its solo run bit for bit."""
    sizes = [(5, 5, 300), (700, 5, 5), (9, 260, 5), (33, 17, 9)]
    b = S.Batch(sizes, precision, Re=[400.0, 900.0, 1600.0, 100.0], Mach=[0.1, 0.2, 0.3, 0.4])
    b.init_tgv([1.0, 0.95, 1.05, 0.9])
    b.step_n(3, 1e-3)
    for m, n in enumerate(sizes):
        g = S.Grid(n, precision, S.SBLI_FUSED, Re=[400.0, 900.0, 1600.0, 100.0][m], Mach=[0.1, 0.2, 0.3, 0.4][m])
        g.init_tgv([1.0, 0.95, 1.05, 0.9][m])
        g.step_n(3, 1e-3)
        assert torch.equal(b.get_state(m), g.get_state()), (m, n)
        g.close()
    b.close()


@pytest.mark.parametrize("precision", [0, 1, 2, 3])
def test_batch_set_state_mid_run(S, precision):
    """A member's state set after an odd number of steps (the other register
    of the rotation) steps on exactly like a fresh single grid given it."""
    sizes = [(24, 20, 16), (32, 16, 12)]
    b = S.Batch(sizes, precision)
    b.init_tgv([1.0, 0.9])
    b.step_n(1, 1e-3)
    e0 = 1.0 / (1.4 * 0.4 * 0.1**2) + 0.5
    q = workloads.smooth_state(sizes[0], 77, offsets=(1.0, 0, 0, 0, e0), amplitudes=(0.05, 0.3, 0.3, 0.3, 0.3))
    b.set_state(0, torch.from_numpy(q).cuda())
    b.step_n(2, 1e-3)
    g = S.Grid(sizes[0], precision, S.SBLI_FUSED)
    g.set_state(torch.from_numpy(q).cuda())
    g.step_n(2, 1e-3)
    assert torch.equal(b.get_state(0), g.get_state())
    g.close()
    b.close()


@pytest.mark.parametrize("precision", [0, 1, 2, 3])
def test_batch_schedules_are_bitwise_identical(S, precision):
    """The schedule (z-queue mode, planes per work item of each member)
    changes only the work decomposition: any schedule, and the one the
    autotuner picks, gives bitwise the state of the default schedule and of
    each member run alone; the autotuner leaves the state unchanged."""
    dt, steps = 1e-3, 7
    ref = S.Batch(SIZES, precision, Re=RE, Mach=MACH)
    ref.init_tgv(AMP)
    ref.step_n(steps, dt)
    want = [ref.get_state(m) for m in range(len(SIZES))]
    zq0, zc0 = ref.schedule()
    assert zq0 == (1 if precision in (1, 2) else 0)
    assert zc0 == [min(32, n[2]) for n in SIZES]
    ref.close()
    for sched in [(1 - zq0, [4, 9, 5, 24, 7]), (zq0, [16, 8, 12, 6, 4]), "tuned"]:
        b = S.Batch(SIZES, precision, Re=RE, Mach=MACH)
        b.init_tgv(AMP)
        if sched == "tuned":
            before = [b.get_state(m) for m in range(len(SIZES))]
            zq, ms = b.autotune(2)
            assert zq in (0, 1) and ms > 0
            for m in range(len(SIZES)):
                assert torch.equal(b.get_state(m), before[m]), m
            zq_now, zc_now = b.schedule()
            assert zq_now == zq and all(4 <= z <= n[2] or z == n[2] for z, n in zip(zc_now, SIZES))
        else:
            b.set_schedule(*sched)
            zq_now, zc_now = b.schedule()
            assert zq_now == sched[0] and zc_now == [min(z, n[2]) for z, n in zip(sched[1], SIZES)]
        b.step_n(steps, dt)
        for m in range(len(SIZES)):
            assert torch.equal(b.get_state(m), want[m]), (sched, m)
        b.close()


def test_batch_schedule_rejects_bad_values(S):
    b = S.Batch(SIZES, 1, Re=RE, Mach=MACH)
    with pytest.raises(S.SbliError) as e:
        b.set_schedule(2)
    assert e.value.code == S.SBLI_EINVAL
    with pytest.raises(S.SbliError) as e:
        b.set_schedule(1, [4, 4, 3, 4, 4])
    assert e.value.code == S.SBLI_EINVAL
    assert b.schedule() == (1, [min(32, n[2]) for n in SIZES])
