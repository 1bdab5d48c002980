"""The binary64 reciprocal of the stage kernels (a hardware approximation
refined by two Newton-Raphson steps) against CUDA's correctly rounded
reciprocal: within one unit in the last place on seeded inputs spanning the
density range of the kernels and a wide exponent range."""
import os
import shutil
import subprocess

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1709_09713_gb300", "csrc")


def test_binary64_reciprocal_within_one_ulp(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nvcc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    if not os.path.exists(nvcc):
        nvcc = shutil.which("nvcc")
    if not nvcc:
        pytest.skip("nvcc not found")
    exe = str(tmp_path / "recip_check")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "--expt-relaxed-constexpr",
                    "-I", CSRC, "-o", exe, os.path.join(HERE, "recip_check.cu")], check=True, capture_output=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split()
    worst, differ, n = (int(v) for v in out)
    assert n > 0
    assert worst <= 1, (worst, differ, n)
