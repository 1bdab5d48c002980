"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

Nothing here evaluates the Navier-Stokes method: the generators draw random
numbers (smooth periodic fields, ensemble parameters, request traces) and
return them.  Both the CUDA path and the CPU oracle receive the same arrays,
so neither side's arithmetic leaks into the other.

Recipes (the Taylor-Green vortex workload of §4 of arXiv:1709.09713 is the
base case; these generate the perturbed and mixed inputs around it):

* ``smooth_state``: five exactly periodic fields, each a sum of random Fourier
  modes with wavenumbers |k_i| <= kmax, added to the constant offsets the
  caller gives (density ~1, total energy large enough for positive pressure).
* ``ensemble``: per instance, grid edge N uniform over {32, 48, 64, 96, 128},
  Re ~ U[100, 1600], Mach ~ U[0.1, 0.4], velocity amplitude ~ U(0.9, 1.1),
  drawn in that order from one PCG64 stream.
* ``request_trace``: Poisson arrivals at a given mean rate, grid edge
  log-uniform on [32, 256] rounded to a multiple of 8, step count uniform on
  {50..2000}, precision flag FP64/FP32 with probability 1/2 each.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

ENSEMBLE_SIZES = (32, 48, 64, 96, 128)


def _grid_axes(n):
    n0, n1, n2 = n
    x = np.arange(n0) * (2.0 * math.pi / n0)
    y = np.arange(n1) * (2.0 * math.pi / n1)
    z = np.arange(n2) * (2.0 * math.pi / n2)
    return x, y, z


def smooth_field(n, rng: np.random.Generator, kmax: int = 3, modes: int = 6) -> np.ndarray:
    """One periodic field of shape (n2, n1, n0), values O(1), built from
    ``modes`` random plane waves cos(k.x + phase) with |k_i| <= kmax."""
    x, y, z = _grid_axes(n)
    out = np.zeros((len(z), len(y), len(x)))
    for _ in range(modes):
        k = rng.integers(-kmax, kmax + 1, size=3)
        if not k.any():
            k[0] = 1
        ph = rng.uniform(0.0, 2.0 * math.pi)
        amp = rng.uniform(0.3, 1.0) / modes
        out += amp * np.cos(k[0] * x[None, None, :] + k[1] * y[None, :, None] + k[2] * z[:, None, None] + ph)
    return out


def smooth_state(n, seed: int, offsets=(1.0, 0.0, 0.0, 0.0, 180.0), amplitudes=(0.05, 0.5, 0.5, 0.5, 0.5),
                 kmax: int = 3) -> np.ndarray:
    """Five smooth random periodic fields ``offsets[f] + amplitudes[f] * field_f``,
    shape (5, n2, n1, n0), float64.  ``n`` is an int (cube) or (n0, n1, n2)."""
    if isinstance(n, int):
        n = (n, n, n)
    rng = np.random.default_rng(seed)
    q = np.empty((5, n[2], n[1], n[0]))
    for f in range(5):
        q[f] = offsets[f] + amplitudes[f] * smooth_field(n, rng, kmax=kmax)
    return q


def perturbation(n, seed: int, scale: float, kmax: int = 4) -> np.ndarray:
    """A smooth random perturbation of all five fields, each scaled by ``scale``."""
    if isinstance(n, int):
        n = (n, n, n)
    rng = np.random.default_rng(seed)
    return np.stack([scale * smooth_field(n, rng, kmax=kmax) for _ in range(5)])


def separable_perturbation(n, seed: int, scale: float, modes: int = 2, kmax: int = 4) -> np.ndarray:
    """A smooth random perturbation of all five fields, cheap at large N: each
    field is ``scale`` times a sum of ``modes`` products a(x0) b(x1) c(x2) of
    random 1-D trigonometric polynomials (wavenumbers 1..kmax, random phases),
    shape (5, n2, n1, n0).  Breaks the Taylor-Green symmetries."""
    if isinstance(n, int):
        n = (n, n, n)
    rng = np.random.default_rng(seed)
    axes = _grid_axes(n)

    def series(x):
        out = np.zeros_like(x)
        for kw in range(1, kmax + 1):
            out += rng.uniform(-1.0, 1.0) / kw * np.cos(kw * x + rng.uniform(0.0, 2.0 * math.pi))
        return out

    q = np.zeros((5, n[2], n[1], n[0]))
    tmp = np.empty((n[2], n[1], n[0]))
    for f in range(5):
        for _ in range(modes):
            a, b, c = (series(x) for x in axes)
            np.multiply(((scale / modes) * c)[:, None, None], np.multiply.outer(b, a)[None, :, :], out=tmp)
            q[f] += tmp
    return q


@dataclass
class EnsembleMember:
    n: int
    Re: float
    Mach: float
    amplitude: float


def ensemble(count: int = 64, seed: int = 1709, sizes=ENSEMBLE_SIZES) -> list[EnsembleMember]:
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(count):
        n = int(sizes[int(rng.integers(0, len(sizes)))])
        Re = float(rng.uniform(100.0, 1600.0))
        M = float(rng.uniform(0.1, 0.4))
        A = float(rng.uniform(0.9, 1.1))
        out.append(EnsembleMember(n, Re, M, A))
    return out


@dataclass
class Request:
    arrival_s: float
    n: int
    steps: int
    precision: int  # 0 = FP64, 1 = FP32 storage
    Re: float
    Mach: float
    amplitude: float


def request_trace(count: int = 200, seed: int = 20, rate_hz: float = 20.0, nmin: int = 32, nmax: int = 256,
                  steps_lo: int = 50, steps_hi: int = 2000, Re: float = 1600.0, Mach: float = 0.1) -> list[Request]:
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for _ in range(count):
        t += float(rng.exponential(1.0 / rate_hz))
        n = math.exp(rng.uniform(math.log(nmin), math.log(nmax)))
        n = int(min(nmax, max(nmin, 8 * round(n / 8.0))))
        steps = int(rng.integers(steps_lo, steps_hi + 1))
        prec = int(rng.integers(0, 2))
        out.append(Request(t, n, steps, prec, Re, Mach, 1.0))
    return out
