"""CPU-side checks of the C ABI: the library loads without a GPU, exports
every entry point the headers under include/ declare, and rejects invalid
arguments that need no device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def sbli():
    from paper_1709_09713_gb300 import build

    build.build()
    from paper_1709_09713_gb300 import sbli as S

    S.lib()
    return S


def declared_functions():
    inc = os.path.join(ROOT, "include")
    text = "".join(open(os.path.join(inc, f)).read() for f in sorted(os.listdir(inc)) if f.endswith(".h"))
    return sorted(set(re.findall(r"SBLI_API\s+(?:const\s+)?\w+\*?\s+\*?(sbli_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["sbli_create_grid", "sbli_init_tgv", "sbli_rhs", "sbli_rk_stage", "sbli_step_n",
                     "sbli_kinetic_energy", "sbli_destroy_grid", "sbli_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(sbli):
    lib = ctypes.CDLL(sbli.LIB_PATH)
    for name in declared_functions():
        assert hasattr(lib, name), name
    # the binding wraps every declared function with the same name
    for name in declared_functions():
        assert name in sbli.SIGNATURES, name
        assert callable(getattr(sbli, name))


def test_exports_only_the_abi(sbli):
    import subprocess

    out = subprocess.run(["nm", "-D", "--defined-only", sbli.LIB_PATH], capture_output=True, text=True).stdout
    syms = [line.split()[-1] for line in out.splitlines() if line.strip()]
    assert syms and all(s.startswith("sbli_") for s in syms), [s for s in syms if not s.startswith("sbli_")]


def test_version(sbli):
    assert sbli.sbli_abi_version() == 1


@pytest.mark.parametrize("n", [(4, 8, 8), (8, 4, 8), (8, 8, 4), (0, 8, 8), (-3, 8, 8)])
def test_rejects_grids_below_stencil_width(sbli, n):
    with pytest.raises(sbli.SbliError) as e:
        sbli.sbli_workspace_bytes(*n, sbli.SBLI_FP64, sbli.SBLI_FUSED)
    assert e.value.code == sbli.SBLI_EINVAL
    assert "5" in sbli.sbli_last_error()


@pytest.mark.parametrize("n", [(65536, 32768, 8), (2048, 2048, 1024), (1625, 1625, 1627)])
def test_rejects_grids_beyond_32_bit_offsets(sbli, n):
    """n0*n1 >= 2^31 or n0*n1*n2 >= 2^32 would overflow the stage kernels'
    32-bit point offsets; the largest grids that fit a GB300 (~1300^3 at 120
    bytes per point) stay below both."""
    with pytest.raises(sbli.SbliError) as e:
        sbli.sbli_workspace_bytes(*n, sbli.SBLI_FP64, sbli.SBLI_FUSED)
    assert e.value.code == sbli.SBLI_EINVAL
    assert "2^32" in sbli.sbli_last_error()


def test_accepts_the_largest_grids_that_fit(sbli):
    # 1296^3 (2.18e9 points, past 2^31) and 1625^3 (4.29e9, just below 2^32)
    for n in (1296, 1625):
        b = sbli.sbli_workspace_bytes(n, n, n, sbli.SBLI_FP64, sbli.SBLI_FUSED)
        assert b >= 3 * 5 * n**3 * 8


def test_rejects_unknown_modes(sbli):
    with pytest.raises(sbli.SbliError) as e:
        sbli.sbli_workspace_bytes(8, 8, 8, 7, sbli.SBLI_FUSED)
    assert e.value.code == sbli.SBLI_EINVAL
    with pytest.raises(sbli.SbliError) as e:
        sbli.sbli_workspace_bytes(8, 8, 8, sbli.SBLI_FP64, 7)
    assert e.value.code == sbli.SBLI_EINVAL
    with pytest.raises(sbli.SbliError) as e:
        sbli.sbli_workspace_bytes(8, 8, 8, sbli.SBLI_FP64, -1)
    assert e.value.code == sbli.SBLI_EINVAL


def test_workspace_sizes(sbli):
    P = 32**3
    f64 = sbli.sbli_workspace_bytes(32, 32, 32, sbli.SBLI_FP64, sbli.SBLI_FUSED)
    f32 = sbli.sbli_workspace_bytes(32, 32, 32, sbli.SBLI_FP32, sbli.SBLI_FUSED)
    bl = sbli.sbli_workspace_bytes(32, 32, 32, sbli.SBLI_FP64, sbli.SBLI_STORE_ALL)
    assert f64 >= 3 * 5 * P * 8 and f64 < 3 * 5 * P * 8 + (1 << 20)
    assert f32 >= 2 * 5 * P * 8 + 2 * 5 * P * 4
    assert bl >= f64 + 82 * P * 8
    # intermediate storage: primitives (u_i, p, T) and the 9 velocity gradients
    for v in (sbli.SBLI_RS, sbli.SBLI_SS):
        assert sbli.sbli_workspace_bytes(32, 32, 32, sbli.SBLI_FP64, v) == f64 + 14 * P * 8
    # minimal storage: the primitive arrays only, no derivative arrays
    for v in (sbli.SBLI_RA, sbli.SBLI_SN, sbli.SBLI_SN2):
        assert sbli.sbli_workspace_bytes(32, 32, 32, sbli.SBLI_FP64, v) == f64 + 5 * P * 8


def test_df64_uses_the_binary64_registers(sbli):
    f64 = sbli.sbli_workspace_bytes(24, 20, 16, sbli.SBLI_FP64, sbli.SBLI_FUSED)
    assert sbli.sbli_workspace_bytes(24, 20, 16, sbli.SBLI_DF64, sbli.SBLI_FUSED) == f64
    with pytest.raises(sbli.SbliError) as e:
        sbli.sbli_workspace_bytes(24, 20, 16, sbli.SBLI_DF64, sbli.SBLI_STORE_ALL)
    assert e.value.code == sbli.SBLI_EUNSUPPORTED


@pytest.mark.parametrize("precision", [1, 2, 3])
@pytest.mark.parametrize("variant", [2, 3, 4, 5, 6])
def test_comparison_variants_are_binary64_only(sbli, precision, variant):
    with pytest.raises(sbli.SbliError) as e:
        sbli.sbli_workspace_bytes(16, 16, 16, precision, variant)
    assert e.value.code == sbli.SBLI_EUNSUPPORTED


def test_null_arguments_are_errors(sbli):
    lib = sbli.lib()
    assert lib.sbli_workspace_bytes(8, 8, 8, 0, 0, None) == sbli.SBLI_EINVAL
    assert lib.sbli_create_grid(None, 8, 8, 8, 0, 0, None, None, 0, None) == sbli.SBLI_EINVAL
    assert lib.sbli_rk_stage(None, 0, 1e-3) == sbli.SBLI_EINVAL
    assert lib.sbli_sample_state(None, None, 1, None) == sbli.SBLI_EINVAL
    assert lib.sbli_destroy_grid(None) == sbli.SBLI_OK
    h = ctypes.c_void_p()
    prm = sbli.params()
    # null workspace is rejected before any device call
    assert lib.sbli_create_grid(ctypes.byref(h), 8, 8, 8, 0, 0, ctypes.byref(prm), None, 0, None) == sbli.SBLI_EINVAL
    bad = sbli.params(Re=-1.0)
    assert lib.sbli_create_grid(ctypes.byref(h), 8, 8, 8, 0, 0, ctypes.byref(bad), None, 0, None) == sbli.SBLI_EINVAL
    assert "param" in sbli.sbli_last_error()


def test_missing_library_fails_loudly(sbli, monkeypatch):
    """Without the compiled library every entry point raises: there is no
    CPU fallback behind the binding."""
    monkeypatch.setattr(sbli, "LIB_PATH", os.path.join(ROOT, "no-such-dir", "libsbli.so"))
    monkeypatch.setattr(sbli, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        sbli.lib()
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        sbli.sbli_workspace_bytes(16, 16, 16, sbli.SBLI_FP64, sbli.SBLI_FUSED)


def test_product_package_never_loads_the_oracle():
    """The oracle is test infrastructure: importing every module of the
    product package loads nothing from oracle/, and no CUDA source includes
    an oracle header."""
    import subprocess
    import sys

    code = ("import sys; import paper_1709_09713_gb300, paper_1709_09713_gb300.sbli, paper_1709_09713_gb300.build, "
            "paper_1709_09713_gb300.history, paper_1709_09713_gb300.workloads; "
            "bad = [m for m in sys.modules if m == 'oracle' or m.startswith('oracle.')]; print(bad); "
            "sys.exit(1 if bad else 0)")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    csrc = os.path.join(ROOT, "paper_1709_09713_gb300", "csrc")
    for f in os.listdir(csrc):
        text = open(os.path.join(csrc, f)).read()
        assert "sbli_oracle" not in text and "orc_" not in text, f


def test_batch_limits(sbli):
    """Batches take 1..64 members (the member table is a kernel parameter),
    every precision, and the single-grid size rules per member."""
    ok = sbli.sbli_batch_workspace_bytes([(16, 16, 16)] * 64, sbli.SBLI_FP32)
    assert ok >= 64 * 5 * 16**3 * 4
    assert sbli.sbli_batch_workspace_bytes([(16, 16, 16)] * 64, sbli.SBLI_FP32_DF) == ok
    for sizes, prec in (([(16, 16, 16)] * 65, sbli.SBLI_FP32), ([(16, 16, 16)], 7),
                        ([(16, 16, 16), (4, 16, 16)], sbli.SBLI_FP64), ([(2048, 2048, 1024)], sbli.SBLI_FP64)):
        with pytest.raises(sbli.SbliError) as e:
            sbli.sbli_batch_workspace_bytes(sizes, prec)
        assert e.value.code == sbli.SBLI_EINVAL
    lib = sbli.lib()
    assert lib.sbli_batch_workspace_bytes(0, None, 1, None) == sbli.SBLI_EINVAL


def test_probe_rejects_arguments_without_a_device(sbli):
    """The throughput probe checks its arguments before touching a device."""
    with pytest.raises(sbli.SbliError) as e:
        sbli.sbli_probe_fma_rate(sbli.SBLI_DF64, 10, 1)
    assert e.value.code == sbli.SBLI_EINVAL
    with pytest.raises(sbli.SbliError) as e:
        sbli.sbli_probe_fma_rate(sbli.SBLI_FP64, 0, 1)
    assert e.value.code == sbli.SBLI_EINVAL
    with pytest.raises(sbli.SbliError) as e:
        sbli.sbli_probe_fma_rate(sbli.SBLI_FP64, 10, 0)
    assert e.value.code == sbli.SBLI_EINVAL
