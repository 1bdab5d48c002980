"""Long-run Taylor-Green histories (Sec. 4): kinetic energy and enstrophy of
every step to a final time, with the energy balance of the viscous decay.

For a periodic box, the kinetic energy KE = <rho |u|^2 / 2> decays at the rate
-dKE/dt = (2 / Re) Omega + (4 / 3Re) <(div u)^2> - <p div u> (with mu = 1 in
reference units), Omega = <rho |omega|^2 / 2> the enstrophy as this library
reports it (up to the density weight, which is 1 + O(M^2)).  At low Mach
number the dilatational terms are small, so the ratio
    balance(t) = (-dKE/dt) / ((2 / Re) Omega)
stays near 1 while the grid resolves the dissipative scales; the time
derivative is the central difference of the per-step history.

    python -m paper_1709_09713_gb300.history --n 256 --t-end 20 --precision fp32df
prints one JSON line (sampled history, peak enstrophy and its time, the
energy-balance error) and, with --out, writes the full history as .npz.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

PRECISIONS = {"fp64": 0, "fp32": 1, "fp32df": 2}


def run_history(n: int, t_end: float, dt: float, precision: int = 0, Re: float = 1600.0, Mach: float = 0.1,
                chunk: int = 2000, tune: bool = True, stream=None):
    """Advance the Taylor-Green vortex from t = 0 to t_end (a whole number of
    steps of dt) and return (t, ke, enstrophy) of the state before every step
    and after the last one, as binary64 numpy arrays."""
    import torch

    from . import sbli as S

    steps = int(round(t_end / dt))
    g = S.Grid(n, precision, S.SBLI_FUSED, Re=Re, Mach=Mach, stream=stream)
    try:
        if tune and precision != S.SBLI_FP64:
            g.autotune(3)
        g.init_tgv()
        parts = []
        done = 0
        while done < steps:
            k = min(chunk, steps - done)
            parts.append(g.step_n_history(k, dt).cpu().numpy())
            done += k
        ke_end, ens_end = g.kinetic_energy()
        torch.cuda.synchronize()
    finally:
        g.close()
    h = np.concatenate(parts + [np.array([[ke_end, ens_end]])])
    t = dt * np.arange(steps + 1)
    return t, h[:, 0], h[:, 1]


def energy_balance(t, ke, ens, Re: float):
    """balance(t_i) = (-dKE/dt) / ((2 / Re) Omega) at the interior samples
    (central differences)."""
    dke = (ke[2:] - ke[:-2]) / (t[2:] - t[:-2])
    return t[1:-1], -dke / ((2.0 / Re) * ens[1:-1])


def summary(t, ke, ens, Re: float, samples: int = 21) -> dict:
    tb, bal = energy_balance(t, ke, ens, Re)
    i_peak = int(np.argmax(ens))
    eps = -(ke[2:] - ke[:-2]) / (t[2:] - t[:-2])
    pick = np.unique(np.linspace(0, len(t) - 1, samples).round().astype(int))
    return {
        "steps": len(t) - 1,
        "t_end": float(t[-1]),
        "ke0": float(ke[0]),
        "ke_end": float(ke[-1]),
        "enstrophy_peak": float(ens[i_peak]),
        "t_enstrophy_peak": float(t[i_peak]),
        "dissipation_peak": float(np.max(eps)),
        "t_dissipation_peak": float(tb[int(np.argmax(eps))]),
        "balance_min": float(np.min(bal)),
        "balance_max": float(np.max(bal)),
        "history": [[float(t[i]), float(ke[i]), float(ens[i])] for i in pick],
    }


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--t-end", type=float, default=20.0)
    ap.add_argument("--dt", type=float, default=1e-3)
    ap.add_argument("--precision", choices=sorted(PRECISIONS), default="fp32df")
    ap.add_argument("--re", type=float, default=1600.0)
    ap.add_argument("--mach", type=float, default=0.1)
    ap.add_argument("--out", default=None, help="write t, ke, enstrophy to this .npz")
    a = ap.parse_args(argv)
    t0 = time.time()
    t, ke, ens = run_history(a.n, a.t_end, a.dt, PRECISIONS[a.precision], a.re, a.mach)
    wall = time.time() - t0
    if a.out:
        np.savez(a.out, t=t, ke=ke, enstrophy=ens)
    s = summary(t, ke, ens, a.re)
    s.update({"n": a.n, "dt": a.dt, "precision": a.precision, "Re": a.re, "Mach": a.mach, "wall_s": round(wall, 1),
              "pt_stage_per_s": 3 * (len(t) - 1) * a.n**3 / wall if math.isfinite(wall) and wall > 0 else None})
    print(json.dumps(s))


if __name__ == "__main__":
    main()
