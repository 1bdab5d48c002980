"""Allocation-free kinetic energy / enstrophy entry point.

sbli_kinetic_energy_noalloc serves callers that cannot allocate device
memory, so cannot give the library a grid workspace: it takes only their
state pointer and an output pointer and keeps its partial sums in a static
device array.  These checks call it through the C ABI and compare it with the
workspace-based sbli_kinetic_energy on the same states, twice in a row (the
static array is shared by every call and keeps the previous call's sums).
"""
import gc

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


def _state(n, seed):
    e0 = 1.0 / (1.4 * 0.4 * 0.01) + 0.5
    q = workloads.smooth_state(n, seed, offsets=(1.0, 0.0, 0.0, 0.0, e0), amplitudes=(0.05, 0.5, 0.5, 0.5, 0.5))
    return torch.from_numpy(q).cuda()


def _existing(S, n, q):
    g = S.Grid(n, S.SBLI_FP64, S.SBLI_FUSED)
    g.set_state(q)
    out = g.kinetic_energy()
    g.close()
    return out


def _noalloc(S, n, q, L=1.0):
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    S.sbli_kinetic_energy_noalloc(q.data_ptr(), n[0], n[1], n[2], L, out.data_ptr(),
                                  torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("n", [(32, 32, 32), (40, 24, 20), (5, 6, 7)])
def test_noalloc_matches_workspace_entry_point_two_calls(S, n):
    qa, qb = _state(n, 101), _state(n, 202)
    ka, ea = _existing(S, n, qa)
    kb, eb = _existing(S, n, qb)
    first = _noalloc(S, n, qa)
    second = _noalloc(S, n, qb)
    assert first[0] == pytest.approx(ka, rel=1e-13) and first[1] == pytest.approx(ea, rel=1e-12)
    assert second[0] == pytest.approx(kb, rel=1e-13) and second[1] == pytest.approx(eb, rel=1e-12)
    # the shared array carries nothing from one call into the next
    again = _noalloc(S, n, qa)
    assert np.array_equal(again, first)


def test_noalloc_tgv_closed_form(S):
    """Same TGV state the workspace path produces: KE = 1/8 exactly."""
    n = (16, 16, 16)
    g = S.Grid(n, S.SBLI_FP64, S.SBLI_FUSED)
    g.init_tgv(1.0)
    q = g.get_state()
    ke, ens = g.kinetic_energy()
    out = _noalloc(S, n, q)
    assert out[0] == pytest.approx(0.125, rel=1e-13)
    assert out[0] == pytest.approx(ke, rel=1e-13) and out[1] == pytest.approx(ens, rel=1e-12)


def test_noalloc_rejects_grids_beyond_its_maximum(S):
    q = torch.zeros(16, dtype=torch.float64, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pytest.raises(S.SbliError) as e:
        S.sbli_kinetic_energy_noalloc(q.data_ptr(), 1024, 512, 512, 1.0, out.data_ptr())
    assert e.value.code == S.SBLI_EINVAL
    assert "maximum" in str(e.value)
    with pytest.raises(S.SbliError) as e:
        S.sbli_kinetic_energy_noalloc(q.data_ptr(), 4, 8, 8, 1.0, out.data_ptr())
    assert e.value.code == S.SBLI_EINVAL
    with pytest.raises(S.SbliError):
        S.sbli_kinetic_energy_noalloc(0, 8, 8, 8, 1.0, out.data_ptr())


def test_noalloc_domain_scale_and_side_stream(S):
    """L = 2 doubles every spacing h: the kinetic energy is unchanged and the
    enstrophy (squares of first derivatives) scales by exactly 1/4 in
    binary arithmetic; the result does not depend on the stream used."""
    n = (24, 20, 28)
    q = _state(n, 303)
    base = _noalloc(S, n, q, L=1.0)
    scaled = _noalloc(S, n, q, L=2.0)
    assert scaled[0] == pytest.approx(base[0], rel=1e-15)
    assert scaled[1] == pytest.approx(base[1] / 4.0, rel=1e-13)
    side = torch.cuda.Stream()
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    S.sbli_kinetic_energy_noalloc(q.data_ptr(), n[0], n[1], n[2], 1.0, out.data_ptr(), side.cuda_stream)
    side.synchronize()
    assert np.array_equal(out.cpu().numpy(), base)


def test_noalloc_limit_and_pointers_checked_before_launch(S):
    """One plane past 512^3 is refused, as are host pointers, with nothing
    launched (the output keeps its sentinel)."""
    q = torch.zeros(16, dtype=torch.float64, device="cuda")
    out = torch.full((2,), 7.0, dtype=torch.float64, device="cuda")
    with pytest.raises(S.SbliError) as e:
        S.sbli_kinetic_energy_noalloc(q.data_ptr(), 512, 512, 513, 1.0, out.data_ptr())
    assert e.value.code == S.SBLI_EINVAL
    host = np.zeros(5 * 8 * 8 * 8)
    with pytest.raises(S.SbliError) as e:
        S.sbli_kinetic_energy_noalloc(host.ctypes.data, 8, 8, 8, 1.0, out.data_ptr())
    assert e.value.code == S.SBLI_EINVAL
    hout = np.zeros(2)
    qd = _state((8, 8, 8), 5)
    with pytest.raises(S.SbliError) as e:
        S.sbli_kinetic_energy_noalloc(qd.data_ptr(), 8, 8, 8, 1.0, hout.ctypes.data)
    assert e.value.code == S.SBLI_EINVAL
    torch.cuda.synchronize()
    assert out.cpu().tolist() == [7.0, 7.0]


def test_noalloc_allocates_nothing(S):
    """After a first call (module and symbol set-up), further calls leave the
    device's free memory and torch's allocation count unchanged."""
    n = (32, 32, 32)
    q = _state(n, 404)
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    S.sbli_kinetic_energy_noalloc(q.data_ptr(), n[0], n[1], n[2], 1.0, out.data_ptr())
    torch.cuda.synchronize()
    gc.collect()  # tensors of earlier tests freed now, not during the loop below
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(5):
        S.sbli_kinetic_energy_noalloc(q.data_ptr(), n[0], n[1], n[2], 1.0, out.data_ptr())
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_allocated() == alloc0
