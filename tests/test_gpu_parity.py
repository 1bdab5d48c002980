"""GPU path (through the C ABI) against the CPU oracle on identical inputs.

Tolerances (relative max-norm per field; the three momentum fields share the
denominator max_i |rho u_i| because rho u2 starts at zero):
  * binary64 state after the stated steps: 1e-12 (the stated FP64 bar);
  * binary64 residual on random states: 1e-12;
  * binary32 stage storage and arithmetic with binary64 accumulation: state
    1e-5, kinetic-energy history 1e-6 (the stated FP32 bars); residual 1e-4
    (binary32 arithmetic: eps = 6e-8 times the ~1e3 amplification of the
    derivative stencils and cancellations in the energy equation).
"""
import math

import numpy as np
import pytest

from paper_1709_09713_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GAMMA, MACH = 1.4, 0.1


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


def random_state(n, seed):
    e0 = 1.0 / (GAMMA * (GAMMA - 1.0) * MACH**2) + 0.5
    return workloads.smooth_state(n, seed, offsets=(1.0, 0.0, 0.0, 0.0, e0), amplitudes=(0.05, 0.5, 0.5, 0.5, 0.5))


def to_dev(q):
    return torch.from_numpy(np.ascontiguousarray(q)).cuda()


GRIDS = [(32, 32, 32), (40, 24, 20), (37, 11, 9), (5, 5, 5), (5, 6, 7), (64, 16, 8)]


ALL_VARIANTS = [0, 1, 2, 3, 4, 5, 6]  # fused, BL, RS, SS, RA, SN, SN2


@pytest.mark.parametrize("variant", ALL_VARIANTS)
@pytest.mark.parametrize("n", GRIDS)
def test_rhs_fp64_matches_oracle(S, orc, n, variant):
    q = random_state(n, seed=sum(n))
    g = S.Grid(n, S.SBLI_FP64, variant)
    g.set_state(to_dev(q))
    r = g.rhs().cpu().numpy()
    want = orc.rhs(orc.params(n), q)
    errs = rel_fields(r, want)
    assert max(errs) <= 1e-12, errs


@pytest.mark.parametrize("n", GRIDS)
def test_rhs_df64_matches_oracle(S, orc, n):
    """Double-float stage arithmetic on binary64 registers: the residual to
    the binary64 bar."""
    q = random_state(n, seed=11 + sum(n))
    g = S.Grid(n, S.SBLI_DF64, S.SBLI_FUSED)
    g.set_state(to_dev(q))
    r = g.rhs().cpu().numpy()
    want = orc.rhs(orc.params(n), q)
    errs = rel_fields(r, want)
    print("df64 residual errors", errs)
    assert max(errs) <= 1e-12, errs


def test_tgv_32_df64_ten_steps_and_history(S, orc):
    """The 32^3 Taylor-Green case with double-float stage arithmetic: state
    after 10 steps and the kinetic-energy/enstrophy history against the
    oracle, <= 1e-12."""
    n, dt, steps = 32, 1e-3, 10
    g = S.Grid(n, S.SBLI_DF64, S.SBLI_FUSED)
    g.init_tgv(1.0)
    hist = g.step_n_history(steps, dt).cpu().numpy()
    got = g.get_state().cpu().numpy()
    p = orc.params(n)
    q = orc.init_tgv(p)
    for s in range(steps):
        ke_o, ens_o = orc.ke_enstrophy(p, q)
        assert abs(hist[s, 0] - ke_o) / ke_o <= 1e-12
        assert abs(hist[s, 1] - ens_o) / ens_o <= 1e-12
        q = orc.step(p, q, dt, 1)
    errs = rel_fields(got, q)
    print("df64 state errors", errs)
    assert max(errs) <= 1e-12, errs


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("n", [(32, 32, 32), (40, 24, 20), (5, 6, 7)])
def test_rhs_fp32_matches_oracle(S, orc, n, variant):
    q = random_state(n, seed=3 + sum(n))
    g = S.Grid(n, S.SBLI_FP32, variant)
    g.set_state(to_dev(q))
    r = g.rhs().cpu().numpy()
    want = orc.rhs(orc.params(n), q)
    errs = rel_fields(r, want)
    assert max(errs) <= 1e-4, errs


@pytest.mark.parametrize("precision", [0, 1])
def test_init_tgv_matches_oracle(S, orc, precision):
    n = (32, 24, 16)
    for A in (1.0, 0.93):
        g = S.Grid(n, precision, S.SBLI_FUSED)
        g.init_tgv(A)
        got = g.get_state().cpu().numpy()
        want = orc.init_tgv(orc.params(n), A)
        assert max(rel_fields(got, want)) <= 1e-14


@pytest.mark.parametrize("variant", ALL_VARIANTS)
def test_tgv_32_fp64_ten_steps(S, orc, variant):
    """The 32^3 Taylor-Green case (Re 1600, M 0.1, dt 1e-3, 10 steps):
    the fused path and every comparison algorithm (BL, RS, SS, RA, SN, SN2)
    against the oracle, <= 1e-12."""
    n, dt, steps = 32, 1e-3, 10
    g = S.Grid(n, S.SBLI_FP64, variant)
    g.init_tgv(1.0)
    g.step_n(steps, dt)
    got = g.get_state().cpu().numpy()
    p = orc.params(n)
    want = orc.step(p, orc.init_tgv(p), dt, steps)
    errs = rel_fields(got, want)
    assert max(errs) <= 1e-12, errs
    assert g.stage_count() == 3 * steps


def test_stages_one_by_one_match_oracle(S, orc):
    """Each stage's outputs (stage field and accumulator) against the oracle's
    two-register stage, on a random ragged grid, binary64."""
    n, dt = (24, 20, 12), 2e-3
    q0 = random_state(n, seed=77)
    g = S.Grid(n, S.SBLI_FP64, S.SBLI_FUSED)
    g.set_state(to_dev(q0))
    p = orc.params(n)
    q_in, acc = q0.copy(), q0.copy()
    for k in range(3):
        g.rk_stage(k, dt)
        q_out, acc = orc.stage(p, k, dt, q_in, acc)
        if k < 2:
            qs, qa = (t.cpu().numpy() for t in g.get_stage())
            assert max(rel_fields(qs, q_out)) <= 1e-13
            assert max(rel_fields(qa, acc)) <= 1e-13
        q_in = q_out
    got = g.get_state().cpu().numpy()
    assert max(rel_fields(got, acc)) <= 1e-13


@pytest.mark.parametrize("precision", [0, 1])
def test_graph_steps_equal_stage_calls(S, precision):
    """sbli_step_n (captured graph, 6-step chunks + remainder) is bitwise the
    same as calling the stages one by one."""
    n, dt, steps = (32, 16, 16), 1e-3, 8
    a = S.Grid(n, precision, S.SBLI_FUSED)
    b = S.Grid(n, precision, S.SBLI_FUSED)
    a.init_tgv()
    b.init_tgv()
    a.step_n(steps, dt)
    for _ in range(steps):
        for k in range(3):
            b.rk_stage(k, dt)
    assert torch.equal(a.get_state(), b.get_state())


def test_fused_and_storeall_agree(S):
    n, dt = (32, 24, 16), 1e-3
    a = S.Grid(n, S.SBLI_FP64, S.SBLI_FUSED)
    b = S.Grid(n, S.SBLI_FP64, S.SBLI_STORE_ALL)
    q = to_dev(random_state(n, 5))
    a.set_state(q)
    b.set_state(q)
    a.step_n(4, dt)
    b.step_n(4, dt)
    assert max(rel_fields(a.get_state().cpu().numpy(), b.get_state().cpu().numpy())) <= 1e-13


@pytest.mark.parametrize("variant", [0, 1])
def test_tgv_fp32_against_fp64_oracle(S, orc, variant):
    """Binary32 storage/arithmetic with binary64 accumulation, 32^3 TGV,
    10 steps: fields within 1e-5, KE within 1e-6 of the binary64 oracle."""
    n, dt, steps = 32, 1e-3, 10
    g = S.Grid(n, S.SBLI_FP32, variant)
    g.init_tgv(1.0)
    g.step_n(steps, dt)
    got = g.get_state().cpu().numpy()
    p = orc.params(n)
    want = orc.step(p, orc.init_tgv(p), dt, steps)
    errs = rel_fields(got, want)
    assert max(errs) <= 1e-5, errs
    ke, ens = g.kinetic_energy()
    ke_o, ens_o = orc.ke_enstrophy(p, want)
    assert abs(ke - ke_o) / ke_o <= 1e-6


@pytest.mark.parametrize("n", [(32, 32, 32), (20, 12, 28), (5, 5, 5)])
def test_kinetic_energy_matches_oracle(S, orc, n):
    q = random_state(n, seed=19)
    g = S.Grid(n, S.SBLI_FP64, S.SBLI_FUSED)
    g.set_state(to_dev(q))
    ke, ens = g.kinetic_energy()
    ke_o, ens_o = orc.ke_enstrophy(orc.params(n), q)
    assert ke == pytest.approx(ke_o, rel=1e-13)
    assert ens == pytest.approx(ens_o, rel=1e-12)


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-6)])
def test_history_matches_oracle(S, orc, precision, tol):
    """KE/enstrophy of Q^n before each step, fused into stage 0."""
    n, dt, steps = 24, 1e-3, 5
    g = S.Grid(n, precision, S.SBLI_FUSED)
    g.init_tgv()
    hist = g.step_n_history(steps, dt).cpu().numpy()
    p = orc.params(n)
    q = orc.init_tgv(p)
    for s in range(steps):
        ke_o, ens_o = orc.ke_enstrophy(p, q)
        assert abs(hist[s, 0] - ke_o) / ke_o <= tol
        assert abs(hist[s, 1] - ens_o) / ens_o <= tol * 10
        q = orc.step(p, q, dt, 1)


def test_error_paths_fault_nothing(S):
    g = S.Grid(16, S.SBLI_FP64, S.SBLI_FUSED)
    g.init_tgv()
    with pytest.raises(S.SbliError) as e:
        g.rk_stage(1, 1e-3)
    assert e.value.code == S.SBLI_EINVAL
    with pytest.raises(S.SbliError):
        g.rk_stage(0, -1.0)
    g.rk_stage(0, 1e-3)
    with pytest.raises(S.SbliError):
        g.get_state()
    with pytest.raises(S.SbliError):
        g.step_n(1, 1e-3)
    g.rk_stage(1, 1e-3)
    g.rk_stage(2, 1e-3)
    before = g.get_state()
    stages = S.sbli_stage_count(g.handle)
    g.step_n(0, 1e-3)  # zero steps: nothing runs
    assert torch.equal(g.get_state(), before) and S.sbli_stage_count(g.handle) == stages
    with pytest.raises(S.SbliError):
        g.step_n(-1, 1e-3)
    with pytest.raises(S.SbliError):
        g.step_n(1, float("nan"))
    with pytest.raises(S.SbliError):
        S.sbli_sample_state(g.handle, 0, -1, 0)  # negative count
    small = torch.empty(1024, dtype=torch.uint8, device="cuda")
    with pytest.raises(S.SbliError) as e:
        S.sbli_create_grid(16, 16, 16, 0, 0, S.params(), (small.data_ptr() + 255) // 256 * 256, 512, 0)
    assert e.value.code == S.SBLI_ENOMEM
    host = torch.empty(1 << 20, dtype=torch.uint8)
    with pytest.raises(S.SbliError) as e:
        S.sbli_create_grid(8, 8, 8, 0, 0, S.params(), (host.data_ptr() + 255) // 256 * 256, 1 << 19, 0)
    assert e.value.code in (S.SBLI_EINVAL, S.SBLI_ENOMEM)
    torch.cuda.synchronize()


@pytest.mark.parametrize(
    "precision,configs",
    [
        (1, [(8, 4, 0, 1), (8, 13, 0, 1), (16, 7, 0, 1), (16, 40, 0, 1), (8, 13, 1, 1), (16, 7, 1, 1),
             (16, 40, 1, 1), (8, 4, 1, 1), (16, 4, 1, 1), (8, 4, 0, 2), (8, 13, 0, 2), (8, 40, 0, 2)]),
        (2, [(8, 4, 0, 1), (16, 7, 0, 1), (8, 13, 1, 1), (16, 40, 1, 1), (16, 5, 1, 1), (8, 5, 0, 2),
             (8, 40, 0, 2)]),
        (0, [(8, 4, 0, 1), (8, 9, 0, 1), (8, 40, 0, 1), (8, 4, 1, 1), (8, 13, 1, 1)]),
        (3, [(8, 4, 0, 1), (8, 40, 0, 1), (8, 5, 1, 1), (8, 40, 1, 1)]),
    ],
)
@pytest.mark.parametrize("n", [(64, 48, 40), (96, 20, 12), (40, 9, 7)])
def test_launch_configs_are_bitwise_identical(S, precision, configs, n):
    """Tile height, planes per CTA and where the x2-neighbour records live
    (shared-memory ring or TMEM queue; 32 x 16 queue tiles with four
    full-record planes and two barriers per plane) change only the work
    decomposition and data movement: every point's arithmetic is the same, so the state (and
    the kinetic-energy history up to the order of its sums) is bitwise equal.
    Two columns per thread use packed two-lane instructions with their own
    multiply-add fusion: bitwise equal among themselves, within the binary32
    bar of the one-column kernels.  Grids with x0 extents that are not
    multiples of 64 cover the two-column tiles' ragged edge."""
    dt = 1e-3
    q = to_dev(random_state(n, 23))
    ref = {}
    for ty, zc, zq, px in configs:
        g = S.Grid(n, precision, S.SBLI_FUSED)
        g.set_config(ty, zc, zq, px)
        assert g.config() == (ty, min(zc, n[2]), zq, px)
        g.set_state(q)
        g.step_n(2, dt)
        hist = g.step_n_history(2, dt).cpu().numpy()
        out = g.get_state()
        if px not in ref:
            ref[px] = (out, hist)
        else:
            assert torch.equal(out, ref[px][0]), (ty, zc, zq, px)
            assert np.allclose(hist, ref[px][1], rtol=1e-13, atol=0), (ty, zc, zq, px)
    if 2 in ref:
        errs = rel_fields(ref[2][0].cpu().numpy(), ref[1][0].cpu().numpy())
        assert max(errs) <= 1e-5, errs
        assert np.allclose(ref[2][1], ref[1][1], rtol=1e-6, atol=0)


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("n", [(64, 32, 24), (96, 20, 12), (40, 9, 7)])
def test_two_column_tiles_match_oracle(S, orc, precision, n):
    """Two columns per thread (64 x 8 tiles, packed two-lane binary32
    arithmetic) against the oracle: residual within the binary32 residual
    bar, state after 5 steps within the binary32 state bar."""
    q = random_state(n, seed=41 + sum(n))
    g = S.Grid(n, precision, S.SBLI_FUSED)
    g.set_config(8, 8, 0, 2)
    g.set_state(to_dev(q))
    r = g.rhs().cpu().numpy()
    p = orc.params(n)
    assert max(rel_fields(r, orc.rhs(p, q))) <= 1e-4
    g.step_n(5, 1e-3)
    got = g.get_state().cpu().numpy()
    errs = rel_fields(got, orc.step(p, q, 1e-3, 5))
    assert max(errs) <= 1e-5, errs


def test_autotune_keeps_state_and_picks_a_valid_config(S):
    n = (64, 64, 64)
    g = S.Grid(n, S.SBLI_FP32, S.SBLI_FUSED)
    g.init_tgv()
    before = g.get_state()
    ty, zc, zq, px, ms = g.autotune(reps=2)
    assert ty in (8, 16) and 4 <= zc <= n[2] and zq in (0, 1) and px in (1, 2) and ms > 0
    assert torch.equal(g.get_state(), before)
    assert g.config() == (ty, zc, zq, px)
    g.step_n(1, 1e-3)
    with pytest.raises(S.SbliError):
        g.set_config(12, 8)
    with pytest.raises(S.SbliError):
        g.set_config(12, 8, 1)
    with pytest.raises(S.SbliError):
        g.set_config(8, 8, 2)
    d = S.Grid(n, S.SBLI_FP64, S.SBLI_FUSED)
    d.set_config(8, 8, 1)  # binary64 records in the TMEM queue
    with pytest.raises(S.SbliError):
        d.set_config(4, 8, 1)  # binary64 tiles are 32 x 8
    with pytest.raises(S.SbliError):
        d.set_config(16, 8, 1)
    with pytest.raises(S.SbliError):
        d.set_config(8, 8, 0, 2)  # two columns per thread: binary32 only
    with pytest.raises(S.SbliError):
        g.set_config(16, 8, 0, 2)  # two-column tiles are 64 x 8
    with pytest.raises(S.SbliError):
        g.set_config(8, 8, 1, 2)  # ... with the shared-memory ring


@pytest.mark.parametrize("precision", [0, 1, 2, 3])
def test_autotune_leaves_every_register_of_the_state(S, precision):
    """The autotuner's trial stages leave the state bitwise as it was, and
    with it every copy the next step reads (the binary32 copy, the (hi, lo)
    pair copy of a double-float grid whose state is updated in place): the
    steps after autotuning equal those of a grid that was never tuned."""
    n, dt = (40, 24, 20), 1e-3
    g = S.Grid(n, precision, S.SBLI_FUSED)
    g.init_tgv()
    g.step_n(2, dt)
    before = g.get_state()
    cfg = g.autotune(reps=1)[:4]
    assert torch.equal(g.get_state(), before)
    g.step_n(3, dt)
    ref = S.Grid(n, precision, S.SBLI_FUSED)
    ref.set_config(*cfg)
    ref.init_tgv()
    ref.step_n(5, dt)
    assert torch.equal(g.get_state(), ref.get_state())


def test_fp32_kinetic_energy_history_512_subsample_bound(S, orc):
    """FP32 path against the binary64 GPU path at a larger grid (64^3, 20
    steps): fields within 1e-5, KE history within 1e-6."""
    n, dt, steps = 64, 1e-3, 20
    a = S.Grid(n, S.SBLI_FP64, S.SBLI_FUSED)
    b = S.Grid(n, S.SBLI_FP32, S.SBLI_FUSED)
    a.init_tgv()
    b.init_tgv()
    ha = a.step_n_history(steps, dt).cpu().numpy()
    hb = b.step_n_history(steps, dt).cpu().numpy()
    assert np.max(np.abs(hb[:, 0] - ha[:, 0]) / ha[:, 0]) <= 1e-6
    errs = rel_fields(b.get_state().cpu().numpy(), a.get_state().cpu().numpy())
    assert max(errs) <= 1e-5, errs


# ------------------------------------------------- double-float accumulator

def test_fp32df_state_roundtrip(S):
    """set/get_state through the double-float register keeps about 48 bits."""
    n = (24, 16, 12)
    q = random_state(n, 91)
    g = S.Grid(n, S.SBLI_FP32_DF, S.SBLI_FUSED)
    g.set_state(to_dev(q))
    back = g.get_state().cpu().numpy()
    assert max(rel_fields(back, q)) <= 1e-13


def test_fp32df_against_fp64_oracle(S, orc):
    n, dt, steps = 32, 1e-3, 10
    g = S.Grid(n, S.SBLI_FP32_DF, S.SBLI_FUSED)
    g.init_tgv(1.0)
    hist = g.step_n_history(steps, dt).cpu().numpy()
    got = g.get_state().cpu().numpy()
    p = orc.params(n)
    q = orc.init_tgv(p)
    for s_ in range(steps):
        ke_o, _ = orc.ke_enstrophy(p, q)
        assert abs(hist[s_, 0] - ke_o) / ke_o <= 1e-6
        q = orc.step(p, q, dt, 1)
    errs = rel_fields(got, q)
    assert max(errs) <= 1e-5, errs
    ke, _ = g.kinetic_energy()
    assert abs(ke - orc.ke_enstrophy(p, q)[0]) / ke <= 1e-6


def test_fp32df_rhs_stages_and_graph(S, orc):
    n, dt = (40, 24, 20), 1e-3
    q = random_state(n, 17)
    g = S.Grid(n, S.SBLI_FP32_DF, S.SBLI_FUSED)
    g.set_state(to_dev(q))
    r = g.rhs().cpu().numpy()
    assert max(rel_fields(r, orc.rhs(orc.params(n), q))) <= 1e-4
    p = orc.params(n)
    g.rk_stage(0, dt)
    qs, qa = (t.cpu().numpy() for t in g.get_stage())
    q1, acc1 = orc.stage(p, 0, dt, q, q)
    assert max(rel_fields(qs, q1)) <= 1e-6 and max(rel_fields(qa, acc1)) <= 1e-6
    g.rk_stage(1, dt)
    g.rk_stage(2, dt)
    a = S.Grid(n, S.SBLI_FP32_DF, S.SBLI_FUSED)
    b = S.Grid(n, S.SBLI_FP32_DF, S.SBLI_FUSED)
    a.set_state(to_dev(q))
    b.set_state(to_dev(q))
    a.step_n(7, dt)
    for _ in range(7):
        for k in range(3):
            b.rk_stage(k, dt)
    assert torch.equal(a.get_state(), b.get_state())
    with pytest.raises(S.SbliError) as e:
        S.sbli_workspace_bytes(16, 16, 16, S.SBLI_FP32_DF, S.SBLI_STORE_ALL)
    assert e.value.code == S.SBLI_EUNSUPPORTED


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_init_then_get_state_every_precision(S, orc, precision):
    n = (20, 12, 8)
    g = S.Grid(n, precision, S.SBLI_FUSED)
    g.init_tgv(0.97)
    got = g.get_state().cpu().numpy()
    assert max(rel_fields(got, orc.init_tgv(orc.params(n), 0.97))) <= 1e-14


# (Re, Mach, Pr, gamma, L): the inviscid limit (Re = inf removes the viscous
# and heat-flux terms), a monatomic gas, unit Prandtl number, a half-size and
# a larger domain, on a grid that is not a cube
PHYSICS = [
    (math.inf, 0.1, 0.71, 1.4, 1.0),
    (400.0, 0.3, 1.0, 5.0 / 3.0, 0.5),
    (2500.0, 0.2, 0.71, 1.4, 1.7),
]


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (3, 1e-12), (1, 1e-5), (2, 1e-5)])
@pytest.mark.parametrize("phys", PHYSICS)
def test_physical_parameters_match_oracle(S, orc, phys, prec, tol):
    """Every precision, on random states, with the physical parameters the
    Taylor-Green workloads do not vary: residual (binary64 bar 1e-12,
    binary32 residual bar 1e-4) and three steps against the oracle."""
    Re, Mach, Pr, gamma, L = phys
    n = (24, 20, 16)
    e0 = 1.0 / (gamma * (gamma - 1.0) * Mach**2) + 0.5
    q = workloads.smooth_state(n, 90 + int(gamma * 10), offsets=(1.0, 0.0, 0.0, 0.0, e0),
                               amplitudes=(0.05, 0.4, 0.4, 0.4, 0.4))
    p = orc.params(n, Re=Re, Mach=Mach, Pr=Pr, gamma=gamma, L=L)
    dt = 2e-4 * L
    g = S.Grid(n, prec, S.SBLI_FUSED, Re=Re, Mach=Mach, Pr=Pr, gamma=gamma, L=L)
    g.set_state(to_dev(q))
    r = g.rhs().cpu().numpy()
    assert max(rel_fields(r, orc.rhs(p, q))) <= (tol if tol < 1e-6 else 1e-4), phys
    g.step_n(3, dt)
    got = g.get_state().cpu().numpy()
    errs = rel_fields(got, orc.step(p, q, dt, 3))
    assert max(errs) <= tol, (phys, errs)
    g.close()


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (3, 1e-12), (1, 1e-4), (2, 1e-4)])
def test_uniform_flow_is_steady(S, prec, tol):
    """A uniform state moving with a uniform velocity is steady: its residual
    is only rounding (the streamed stencil sums of equal values, and the
    second-derivative centre coefficient against its neighbours; binary64:
    ~1e-15, binary32: below 1e-4 of the field scales), and the state stays
    put."""
    n = (37, 20, 19)
    rho, u, p = 1.3, (0.2, -0.1, 0.05), 1.0 / (GAMMA * MACH**2) * 1.1
    E = p / (GAMMA - 1.0) + 0.5 * rho * sum(v * v for v in u)
    q = np.empty((5, n[2], n[1], n[0]))
    q[0] = rho
    for i in range(3):
        q[1 + i] = rho * u[i]
    q[4] = E
    g = S.Grid(n, prec, S.SBLI_FUSED)
    g.set_state(to_dev(q))
    r = g.rhs().cpu().numpy()
    scale = np.array([1.0, 1.0, 1.0, 1.0, E])
    assert max(float(np.max(np.abs(r[f]))) / scale[f] for f in range(5)) <= tol
    g.step_n(5, 1e-3)
    got = g.get_state().cpu().numpy()
    assert max(rel_fields(got, q)) <= (1e-14 if prec in (0, 3) else 1e-6)
    g.close()


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_host_buffers_equal_device_buffers(S, prec):
    """The state read and written through host memory (pageable and pinned,
    the path the end-to-end measurement takes) is bit for bit the state
    through device memory, for single grids and batch members."""
    n = (24, 20, 12)
    q = random_state(n, 606)
    g = S.Grid(n, prec, S.SBLI_FUSED)
    g.set_state(torch.from_numpy(q))  # pageable host
    a = g.get_state()
    g.set_state(to_dev(q))
    assert torch.equal(g.get_state(), a)
    g.step_n(2, 1e-3)
    dev = g.get_state()
    pinned = torch.empty(g.shape, dtype=torch.float64).pin_memory()
    g.get_state(pinned)
    pageable = torch.empty(g.shape, dtype=torch.float64)
    g.get_state(pageable)
    assert torch.equal(pinned, dev.cpu()) and torch.equal(pageable, dev.cpu())
    g.close()
    b = S.Batch([n, (16, 16, 16)], prec)  # batch members
    b.init_tgv([1.0, 1.0])
    b.set_state(0, torch.from_numpy(q))
    b.step_n(2, 1e-3)
    out = torch.empty(b.shape(0), dtype=torch.float64)
    b.get_state(0, out)
    assert torch.equal(out, b.get_state(0).cpu())
    b.close()


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_set_state_mid_run_equals_fresh_grid(S, prec):
    """After an odd number of steps the state sits in the other register of
    the rotation; setting a new state there and stepping on equals a fresh
    grid given the same state, bit for bit (for binary32 grids this checks
    that the binary32 copy of the state the first stage reads is rewritten
    wherever the state lives)."""
    n = (40, 24, 20)
    q1, q2 = random_state(n, 811), random_state(n, 812)
    g = S.Grid(n, prec, S.SBLI_FUSED)
    g.set_state(to_dev(q1))
    g.step_n(1, 1e-3)
    g.set_state(to_dev(q2))
    g.step_n(7, 1e-3)  # one captured 6-step graph plus one direct step
    h = S.Grid(n, prec, S.SBLI_FUSED)
    h.set_state(to_dev(q2))
    h.step_n(7, 1e-3)
    assert torch.equal(g.get_state(), h.get_state())
    g.init_tgv(0.9)  # likewise for the initial field
    g.step_n(3, 1e-3)
    h.init_tgv(0.9)
    h.step_n(3, 1e-3)
    assert torch.equal(g.get_state(), h.get_state())
    g.close()
    h.close()
