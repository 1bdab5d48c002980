"""The largest grids one GB300 holds.

1296^3 = 2.18e9 points (past 2^31; about 261 GB of workspace at 120 bytes per
point, of the 280 GB of HBM) is advanced one time step from the Taylor-Green
field of Sec. 4 in every precision, and sampled points (box corners, the
ragged last x tile, tile and z-chunk edges, points whose linear index exceeds
2^31, random points) are compared with the oracle.  The oracle cannot hold
the grid, so each sample is computed on a 25^3 window centred on it with the
grid's spacing: one step reaches 3 stages x 4 points = 12 points to each
side, so the window's centre sees exactly the full grid's neighbourhood (the
oracle pins check the window construction against full-grid steps).
The state is read back point by point (sbli_sample_state), never whole.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N = 1296          # 40.5 tiles of 32 in x: the last x tile is ragged
DT = 2e-4         # stable at this spacing (h = 4.85e-3)
W, HALF = 25, 12  # oracle window and its reach


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1709_09713_gb300 import build

    build.build()
    from paper_1709_09713_gb300 import sbli

    sbli.lib()
    return sbli


def test_sample_state_matches_get_state(S):
    """Bitwise the entries of the full read-out, NaN outside the grid, in
    every precision (binary64 and double-float state layouts)."""
    n = (37, 20, 11)
    P = n[0] * n[1] * n[2]
    idx = torch.tensor([0, 1, 36, 37, P - 1, 5 * 37 + 3 + 740 * 7, -1, P, 10 * P], dtype=torch.int64, device="cuda")
    for prec in (S.SBLI_FP64, S.SBLI_FP32, S.SBLI_FP32_DF, S.SBLI_DF64):
        g = S.Grid(n, prec)
        g.init_tgv(0.95)
        g.step_n(2, 1e-3)
        full = g.get_state().reshape(5, -1)
        got = g.sample_state(idx)
        torch.cuda.synchronize()
        inside = idx[:6]
        assert torch.equal(got[:, :6], full[:, inside]), prec
        assert torch.isnan(got[:, 6:]).all(), prec
        assert g.sample_state(idx[:0]).shape == (5, 0)
        g.close()


def sample_points():
    rng = np.random.default_rng(1296)
    pts = [(i, j, k) for i in (0, N - 1) for j in (0, N - 1) for k in (0, N - 1)]  # corners
    pts += [(1280, 600, 17), (1287, 1295, 640), (1295, 8, 1294)]                  # ragged last x tile
    pts += [(31, 7, 300), (32, 8, 301), (33, 9, 129), (63, 15, 128), (64, 16, 258)]  # tile / z-chunk edges
    pts += [(0, 0, 1279), (1000, 1200, 1280), (77, 1295, 1290), (1295, 1294, 1293)]  # linear index > 2^31
    pts += [tuple(int(v) for v in rng.integers(0, N, size=3)) for _ in range(32)]
    return pts


@pytest.fixture(scope="module")
def oracle_samples(orc):
    """Per sample: the oracle's initial value and its value after one step."""
    p = orc.params(N)
    pw = orc.window_params(p, (W, W, W))
    pts = sample_points()
    q0 = np.empty((5, len(pts)))
    q1 = np.empty((5, len(pts)))
    for m, (i, j, k) in enumerate(pts):
        win = orc.init_tgv_window(p, 1.0, (i - HALF, j - HALF, k - HALF), (W, W, W))
        q0[:, m] = win[:, HALF, HALF, HALF]
        q1[:, m] = orc.step(pw, win, DT, 1)[:, HALF, HALF, HALF]
    return pts, q0, q1


def rel(a, b):
    mom = max(np.max(np.abs(b[1:4])), 1e-300)
    return [float(np.max(np.abs(a[f] - b[f])) / (mom if 1 <= f <= 3 else max(np.max(np.abs(b[f])), 1e-300)))
            for f in range(5)]


# (precision, launch configuration or None for the default, state tol, increment tol)
CASES = [
    (0, None, 1e-12, 2e-9),
    (3, None, 1e-12, 2e-9),
    (2, (8, 129, 1, 1), 1e-5, None),  # 129 planes per CTA: the last z chunk is ragged
    (1, None, 1e-5, None),
]


@pytest.mark.parametrize("precision,cfg,tol,inc_tol", CASES)
def test_1296_cubed_one_step_sampled(S, oracle_samples, precision, cfg, tol, inc_tol):
    pts, q0, q1 = oracle_samples
    bytes_needed = S.sbli_workspace_bytes(N, N, N, precision, S.SBLI_FUSED)
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    if free < bytes_needed + (4 << 30):
        pytest.skip(f"{bytes_needed / 1e9:.0f} GB workspace, {free / 1e9:.0f} GB free")
    assert N**3 > 2**31
    idx = torch.tensor([i + N * (j + N * k) for (i, j, k) in pts], dtype=torch.int64, device="cuda")
    g = S.Grid(N, precision)
    try:
        if cfg:
            g.set_config(*cfg)
        g.init_tgv(1.0)
        s0 = g.sample_state(idx).cpu().numpy()
        g.step_n(1, DT)
        s1 = g.sample_state(idx).cpu().numpy()
        config = g.config()
    finally:
        g.close()
        del g
        torch.cuda.empty_cache()
    assert np.isfinite(s1).all()
    e0, e1 = rel(s0, q0), rel(s1, q1)
    print(f"1296^3 precision {precision} config {config}: state {max(e1):.2e}, "
          f"increment {max(rel(s1 - s0, q1 - q0)):.2e}")
    assert max(e0) <= 1e-14, e0  # the initial fields agree to rounding
    assert max(e1) <= tol, (config, e1)
    if inc_tol is not None:
        # the step's increment itself, not only the state it is added to
        ei = rel(s1 - s0, q1 - q0)
        assert max(ei) <= inc_tol, (config, ei)
