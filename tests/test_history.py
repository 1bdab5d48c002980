"""Long-run Taylor-Green histories (the energy balance of the viscous decay).

CPU: the balance and summary arithmetic on a closed-form decay.  GPU: a short
well-resolved run (48^3, Re 100) whose kinetic-energy decay rate matches
(2/Re) x enstrophy to the O(M^2) compressible terms, and the binary32 paths
against the binary64 history over the same run.
"""
import math

import numpy as np
import pytest

from paper_1709_09713_gb300 import history


def test_energy_balance_of_a_closed_form_decay():
    """KE = K0 exp(-2 nu s t) with enstrophy = s KE gives -dKE/dt = 2 nu Omega
    exactly; central differences reproduce it to O(dt^2)."""
    Re, s, dt = 400.0, 3.0, 1e-3
    t = dt * np.arange(2001)
    ke = 0.125 * np.exp(-2.0 / Re * s * t)
    ens = s * ke
    tb, bal = history.energy_balance(t, ke, ens, Re)
    assert len(tb) == len(t) - 2
    assert np.max(np.abs(bal - 1.0)) < 1e-6
    out = history.summary(t, ke, ens, Re, samples=5)
    assert out["steps"] == 2000 and out["t_end"] == pytest.approx(2.0)
    assert out["t_enstrophy_peak"] == 0.0 and out["ke_end"] == pytest.approx(ke[-1])
    assert abs(out["balance_min"] - 1) < 1e-6 and abs(out["balance_max"] - 1) < 1e-6
    assert [h[0] for h in out["history"]] == pytest.approx([0.0, 0.5, 1.0, 1.5, 2.0])


@pytest.mark.gpu
def test_short_run_energy_balance_and_precisions():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1709_09713_gb300 import build, sbli

    build.build()
    sbli.lib()
    n, Re, dt, t_end = 48, 100.0, 1e-3, 1.0
    t, ke, ens = history.run_history(n, t_end, dt, sbli.SBLI_FP64, Re=Re, tune=False)
    assert len(t) == 1001 and np.all(np.diff(ke) < 0)
    tb, bal = history.energy_balance(t, ke, ens, Re)
    # dilatational dissipation and pressure work are O(M^2) = 1 % at M = 0.1
    assert np.all(np.abs(bal - 1.0) < 0.02), (bal.min(), bal.max())
    for precision in (sbli.SBLI_FP32, sbli.SBLI_FP32_DF, sbli.SBLI_DF64):
        _, k2, e2 = history.run_history(n, t_end, dt, precision, Re=Re, tune=False)
        tol = 1e-12 if precision == sbli.SBLI_DF64 else 1e-6
        assert np.max(np.abs(k2 - ke) / ke) <= tol, precision
        assert np.max(np.abs(e2 - ens) / ens) <= 10 * tol, precision
    assert math.isfinite(ke[-1])
