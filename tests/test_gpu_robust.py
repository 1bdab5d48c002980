"""Robustness of the stage kernels through the C ABI: grids stepping at the
same time on separate streams (their CTAs share SMs, TMEM-queue kernels
included) give the results they give alone; launch configurations changed
between steps keep the state on the same trajectory; odd grid sizes in every
precision match the oracle."""
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
    out = []
    mom = max(np.max(np.abs(b[1:4])), 1e-300)
    for f in range(5):
        den = mom if 1 <= f <= 3 else max(np.max(np.abs(b[f])), 1e-300)
        out.append(float(np.max(np.abs(a[f] - b[f])) / den))
    return out


def random_state(n, seed):
    e0 = 1.0 / (GAMMA * (GAMMA - 1.0) * MACH**2) + 0.5
    return workloads.smooth_state(n, seed, offsets=(1.0, 0.0, 0.0, 0.0, e0), amplitudes=(0.05, 0.5, 0.5, 0.5, 0.5))


# (n, precision, config or None)
CONCURRENT = [
    ((96, 64, 48), 1, (8, 16, 1, 1)),
    ((64, 96, 40), 2, (16, 8, 1, 1)),
    ((80, 48, 56), 2, (8, 12, 1, 1)),
    ((64, 64, 32), 0, None),
    ((48, 40, 36), 3, None),
]


def test_concurrent_grids_on_streams_equal_alone(S):
    dt, steps = 1e-3, 8
    states = [torch.from_numpy(random_state(n, 300 + i)).cuda() for i, (n, _, _) in enumerate(CONCURRENT)]
    torch.cuda.synchronize()

    def make(i, stream):
        n, prec, cfg = CONCURRENT[i]
        g = S.Grid(n, prec, S.SBLI_FUSED, stream=stream)
        if cfg:
            g.set_config(*cfg)
        g.set_state(states[i])
        return g

    alone = []
    for i in range(len(CONCURRENT)):
        st = torch.cuda.Stream()
        g = make(i, st)
        with torch.cuda.stream(st):
            g.step_n(steps, dt)
        alone.append(g.get_state())
        torch.cuda.synchronize()
        g.close()
    streams = [torch.cuda.Stream() for _ in CONCURRENT]
    grids = [make(i, streams[i]) for i in range(len(CONCURRENT))]
    torch.cuda.synchronize()
    for _ in range(steps):  # interleave single steps so the launches overlap on the device
        for g, st in zip(grids, streams):
            with torch.cuda.stream(st):
                g.step_n(1, dt)
    torch.cuda.synchronize()
    outs = [g.get_state() for g in grids]  # copied on each grid's stream
    torch.cuda.synchronize()
    for i, g in enumerate(grids):
        assert torch.equal(outs[i], alone[i]), CONCURRENT[i]
        g.close()


@pytest.mark.parametrize("precision", [1, 2])
def test_config_changes_between_steps(S, precision):
    """Switching tile height, planes per CTA and the z queue between steps
    (each switch rebuilds the captured graphs) leaves the state bitwise on the
    trajectory of a run that never switched."""
    n, dt = (72, 40, 36), 1e-3
    q = torch.from_numpy(random_state(n, 77)).cuda()
    ref = S.Grid(n, precision, S.SBLI_FUSED)
    ref.set_state(q)
    ref.step_n(9, dt)
    g = S.Grid(n, precision, S.SBLI_FUSED)
    g.set_state(q)
    for cfg, k in (((8, 8, 0, 1), 2), ((16, 5, 1, 1), 3), ((8, 36, 1, 1), 1), ((16, 12, 0, 1), 3)):
        g.set_config(*cfg)
        g.step_n(k, dt)
    assert torch.equal(g.get_state(), ref.get_state())


ODD = [(7, 13, 11), (33, 17, 9), (100, 5, 6), (65, 31, 19), (5, 5, 300), (700, 5, 5), (9, 260, 5)]


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (3, 1e-12), (1, 1e-5), (2, 1e-5)])
@pytest.mark.parametrize("n", ODD)
def test_odd_sizes_two_steps_match_oracle(S, orc, n, precision, tol):
    """Two steps on grids whose edges are not multiples of the tile sizes, in
    the configuration the autotuner picks, against the oracle."""
    q = random_state(n, 500 + sum(n))
    g = S.Grid(n, precision, S.SBLI_FUSED)
    if precision in (1, 2):
        g.autotune(2)
    g.set_state(torch.from_numpy(q).cuda())
    g.step_n(2, 1e-3)
    got = g.get_state().cpu().numpy()
    want = orc.step(orc.params(n), q, 1e-3, 2)
    errs = rel_fields(got, want)
    assert max(errs) <= tol, (n, precision, g.config(), errs)
