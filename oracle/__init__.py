"""Plain FP64 CPU oracle for the compressible Navier-Stokes RHS + RK3 stage.

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and bench.py's
``cpu_baseline`` / ``--impl reference`` legs are the only callers.  The product
package never imports this module and this module never imports the product.

The arithmetic lives in ``sbli_oracle.c`` (compiled with ``-ffp-contract=off``);
this file only builds it with gcc and marshals numpy arrays through ctypes.
See the C file's header for the equations followed and the readings taken
where the paper (arXiv:1709.09713) is silent or garbled.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "lib")
_LIB_PATH = os.path.join(_LIBDIR, "liboracle.so")
_SOURCES = [os.path.join(_HERE, "sbli_oracle.c")]
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (OpenMP if the compiler has it)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    newest_src = max(os.path.getmtime(s) for s in _SOURCES + [os.path.join(_HERE, "sbli_oracle.h")])
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest_src:
        return _LIB_PATH
    base = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fno-fast-math",
            "-fPIC", "-shared", "-o", _LIB_PATH + ".tmp"] + _SOURCES + ["-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


class Params(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int * 3),
        ("Re", ctypes.c_double),
        ("Mach", ctypes.c_double),
        ("Pr", ctypes.c_double),
        ("gamma", ctypes.c_double),
        ("L", ctypes.c_double),
        ("energy_form", ctypes.c_int),
    ]


RHS_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double))
_DP = ctypes.POINTER(ctypes.c_double)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            override = os.environ.get("ORACLE_LIB")
            lib = ctypes.CDLL(override if override else build())
            P = ctypes.POINTER(Params)
            sig = {
                "orc_h": (ctypes.c_double, [P, ctypes.c_int]),
                "orc_d1": (None, [P, _DP, ctypes.c_int, _DP]),
                "orc_d2": (None, [P, _DP, ctypes.c_int, _DP]),
                "orc_mixed": (None, [P, _DP, ctypes.c_int, ctypes.c_int, _DP]),
                "orc_primitives": (None, [P, _DP, _DP, _DP, _DP]),
                "orc_rhs": (None, [P, _DP, _DP]),
                "orc_rhs_point": (None, [P, _DP, ctypes.c_int, ctypes.c_int, ctypes.c_int, _DP]),
                "orc_lsrk3_step": (None, [ctypes.c_size_t, _DP, ctypes.c_double, RHS_FN, ctypes.c_void_p, _DP]),
                "orc_stage": (None, [P, ctypes.c_int, ctypes.c_double, _DP, _DP, _DP]),
                "orc_stage_point": (None, [P, ctypes.c_int, ctypes.c_double, _DP, _DP, ctypes.c_int,
                                           ctypes.c_int, ctypes.c_int, _DP, _DP]),
                "orc_step": (None, [P, _DP, ctypes.c_double, ctypes.c_int]),
                "orc_rk_coefficients": (None, [_DP, _DP]),
                "orc_init_tgv": (None, [P, ctypes.c_double, _DP]),
                "orc_init_tgv_window": (None, [P, ctypes.c_double, ctypes.POINTER(ctypes.c_int),
                                               ctypes.POINTER(ctypes.c_int), _DP]),
                "orc_ke_enstrophy": (None, [P, _DP, _DP, _DP]),
                "orc_set_threads": (None, [ctypes.c_int]),
                "orc_get_threads": (ctypes.c_int, []),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
            _lib.orc_set_threads(int(os.environ.get("ORACLE_THREADS", os.cpu_count() or 1)))
    return _lib


def params(n, Re=1600.0, Mach=0.1, Pr=0.71, gamma=1.4, L=1.0, energy_form=0) -> Params:
    if isinstance(n, int):
        n = (n, n, n)
    p = Params()
    p.n[0], p.n[1], p.n[2] = (int(v) for v in n)
    p.Re, p.Mach, p.Pr, p.gamma, p.L = float(Re), float(Mach), float(Pr), float(gamma), float(L)
    p.energy_form = int(energy_form)
    return p


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_DP)


def _npts(p: Params) -> int:
    return p.n[0] * p.n[1] * p.n[2]


def shape(p: Params, fields: int = 1):
    """numpy shape of a field (z, y, x) so that x0 is the fastest index."""
    s = (p.n[2], p.n[1], p.n[0])
    return s if fields == 1 else (fields,) + s


def set_threads(n: int) -> None:
    _load().orc_set_threads(int(n))


def get_threads() -> int:
    return int(_load().orc_get_threads())


def h(p: Params, axis: int) -> float:
    return float(_load().orc_h(ctypes.byref(p), axis))


def d1(p: Params, f: np.ndarray, axis: int) -> np.ndarray:
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.empty_like(f)
    _load().orc_d1(ctypes.byref(p), _ptr(f), axis, _ptr(out))
    return out


def d2(p: Params, f: np.ndarray, axis: int) -> np.ndarray:
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.empty_like(f)
    _load().orc_d2(ctypes.byref(p), _ptr(f), axis, _ptr(out))
    return out


def mixed(p: Params, f: np.ndarray, a: int, b: int) -> np.ndarray:
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.empty_like(f)
    _load().orc_mixed(ctypes.byref(p), _ptr(f), a, b, _ptr(out))
    return out


def primitives(p: Params, q: np.ndarray):
    q = np.ascontiguousarray(q, dtype=np.float64)
    u = np.empty(shape(p, 3))
    pr = np.empty(shape(p))
    T = np.empty(shape(p))
    _load().orc_primitives(ctypes.byref(p), _ptr(q), _ptr(u), _ptr(pr), _ptr(T))
    return u, pr, T


def rhs(p: Params, q: np.ndarray) -> np.ndarray:
    q = np.ascontiguousarray(q, dtype=np.float64)
    r = np.empty_like(q)
    _load().orc_rhs(ctypes.byref(p), _ptr(q), _ptr(r))
    return r


def rhs_point(p: Params, q: np.ndarray, i: int, j: int, k: int) -> np.ndarray:
    q = np.ascontiguousarray(q, dtype=np.float64)
    r = np.empty(5)
    _load().orc_rhs_point(ctypes.byref(p), _ptr(q), i, j, k, _ptr(r))
    return r


def lsrk3_step(q: np.ndarray, dt: float, f) -> np.ndarray:
    """One step of the oracle's low-storage RK3 on a generic RHS ``f(q) -> r``."""
    q = np.array(q, dtype=np.float64, copy=True).ravel()
    n = q.size
    work = np.empty(2 * n)

    def cb(_ctx, qp, rp):
        qa = np.ctypeslib.as_array(qp, shape=(n,))
        ra = np.ctypeslib.as_array(rp, shape=(n,))
        ra[:] = f(qa.copy())

    fn = RHS_FN(cb)
    _load().orc_lsrk3_step(n, _ptr(q), float(dt), fn, None, _ptr(work))
    return q


def stage(p: Params, k: int, dt: float, q_in: np.ndarray, acc: np.ndarray):
    """Returns (q_out, acc_out) of stage k (0..2) in two-register form."""
    q_in = np.ascontiguousarray(q_in, dtype=np.float64)
    acc = np.array(acc, dtype=np.float64, copy=True)
    q_out = np.empty_like(q_in)
    _load().orc_stage(ctypes.byref(p), int(k), float(dt), _ptr(q_in), _ptr(acc), _ptr(q_out))
    return q_out, acc


def stage_point(p: Params, k: int, dt: float, q_in: np.ndarray, acc_in: np.ndarray, i: int, j: int, kk: int):
    q_in = np.ascontiguousarray(q_in, dtype=np.float64)
    acc_in = np.ascontiguousarray(acc_in, dtype=np.float64)
    qo = np.empty(5)
    ao = np.empty(5)
    _load().orc_stage_point(ctypes.byref(p), int(k), float(dt), _ptr(q_in), _ptr(acc_in), i, j, kk, _ptr(qo), _ptr(ao))
    return qo, ao


def step(p: Params, q: np.ndarray, dt: float, nsteps: int = 1) -> np.ndarray:
    q = np.array(q, dtype=np.float64, copy=True)
    _load().orc_step(ctypes.byref(p), _ptr(q), float(dt), int(nsteps))
    return q


def rk_coefficients():
    a = np.empty(3)
    b = np.empty(3)
    _load().orc_rk_coefficients(_ptr(a), _ptr(b))
    return a, b


def init_tgv(p: Params, A: float = 1.0) -> np.ndarray:
    q = np.empty(shape(p, 5))
    _load().orc_init_tgv(ctypes.byref(p), float(A), _ptr(q))
    return q


def init_tgv_window(p: Params, A: float, origin, width) -> np.ndarray:
    """The TGV field of grid ``p`` on a window: shape (5, w2, w1, w0), first
    point the global point ``origin`` (wrapped periodically)."""
    o = (ctypes.c_int * 3)(*(int(v) for v in origin))
    w = (ctypes.c_int * 3)(*(int(v) for v in width))
    q = np.empty((5, int(width[2]), int(width[1]), int(width[0])))
    _load().orc_init_tgv_window(ctypes.byref(p), float(A), o, w, _ptr(q))
    return q


def window_params(p: Params, width) -> Params:
    """Params of a window grid with the same spacing h as ``p`` along each
    axis (n = width, L scaled by width/n; the stencils see only h)."""
    if p.n[0] != p.n[1] or p.n[1] != p.n[2] or width[0] != width[1] or width[1] != width[2]:
        raise ValueError("window params need a cubic grid and a cubic window (one L for all axes)")
    return params(tuple(int(v) for v in width), Re=p.Re, Mach=p.Mach, Pr=p.Pr, gamma=p.gamma,
                  L=p.L * width[0] / p.n[0], energy_form=p.energy_form)


def ke_enstrophy(p: Params, q: np.ndarray):
    q = np.ascontiguousarray(q, dtype=np.float64)
    ke = ctypes.c_double()
    ens = ctypes.c_double()
    _load().orc_ke_enstrophy(ctypes.byref(p), _ptr(q), ctypes.byref(ke), ctypes.byref(ens))
    return ke.value, ens.value


INF = math.inf
