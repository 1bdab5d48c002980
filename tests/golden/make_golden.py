"""Writes tests/golden/tgv32_oracle.txt from the oracle alone.

The fixture is the 32^3 Taylor-Green case of Sec. 4 (Re 1600, M 0.1,
Pr 0.71, gamma 1.4, dt 1e-3): kinetic energy and enstrophy before each of
10 steps and the five conserved variables after 10 steps at fixed sample
points.  It pins the oracle against later changes of its own arithmetic
(each such change must name the passage that justifies it); the oracle's
agreement with the paper is pinned by test_oracle_pins.py.

    python tests/golden/make_golden.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402

N, DT, STEPS = 32, 1e-3, 10
SAMPLES = [(0, 0, 0), (5, 9, 13), (31, 0, 17), (16, 16, 16), (3, 30, 31), (24, 7, 2)]


def compute():
    p = oracle.params(N)
    q = oracle.init_tgv(p)
    hist = []
    for _ in range(STEPS):
        hist.append(oracle.ke_enstrophy(p, q))
        q = oracle.step(p, q, DT, 1)
    pts = [[float(q[f, k, j, i]) for f in range(5)] for (i, j, k) in SAMPLES]
    return hist, pts


def main():
    hist, pts = compute()
    with open(os.path.join(HERE, "tgv32_oracle.txt"), "w") as f:
        f.write("# Taylor-Green vortex (Sec. 4), 32^3, Re 1600, M 0.1, Pr 0.71, gamma 1.4, dt 1e-3\n")
        f.write("# written by tests/golden/make_golden.py from the oracle only\n")
        f.write("# step ke enstrophy (before the step)\n")
        for s, (ke, ens) in enumerate(hist):
            f.write(f"h {s} {ke!r} {ens!r}\n")
        f.write("# i j k rho rho_u0 rho_u1 rho_u2 rho_E after 10 steps\n")
        for (i, j, k), v in zip(SAMPLES, pts):
            f.write(f"q {i} {j} {k} " + " ".join(repr(x) for x in v) + "\n")


if __name__ == "__main__":
    main()
