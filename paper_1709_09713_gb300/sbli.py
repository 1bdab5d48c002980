"""Thin ctypes binding of the C ABI in include/sbli.h.

Every ``sbli_*`` function here has the same name and arguments as the C
entry point and only marshals arguments; all arithmetic runs in
``lib/libsbli.so``.  PyTorch supplies device memory (the workspace) and the
CUDA stream.  ``Grid`` is a small convenience owner of one handle and its
workspace tensor.  There is no CPU fallback: if the library is missing,
``lib()`` raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libsbli.so")

SBLI_OK, SBLI_EINVAL, SBLI_ENOMEM, SBLI_ECUDA, SBLI_ETIMEOUT, SBLI_EUNSUPPORTED = range(6)
SBLI_FP64, SBLI_FP32, SBLI_FP32_DF, SBLI_DF64 = 0, 1, 2, 3
SBLI_FUSED, SBLI_STORE_ALL, SBLI_RS, SBLI_SS, SBLI_RA, SBLI_SN, SBLI_SN2 = range(7)
# the paper's algorithm names (§2.3-2.5) of each variant; "fused" is the tiled product kernel
VARIANT_NAMES = {SBLI_FUSED: "fused", SBLI_STORE_ALL: "BL", SBLI_RS: "RS", SBLI_SS: "SS", SBLI_RA: "RA",
                 SBLI_SN: "SN", SBLI_SN2: "SN2"}

# Every entry point the header declares, with its ctypes signature.
_c_int, _c_double, _c_size_t, _vp = ctypes.c_int, ctypes.c_double, ctypes.c_size_t, ctypes.c_void_p
_DP = ctypes.POINTER(ctypes.c_double)


class Params(ctypes.Structure):
    _fields_ = [("Re", _c_double), ("Mach", _c_double), ("Pr", _c_double), ("gamma", _c_double), ("L", _c_double)]


class Request(ctypes.Structure):
    _fields_ = [("n0", _c_int), ("n1", _c_int), ("n2", _c_int), ("precision", _c_int), ("steps", _c_int),
                ("dt", _c_double), ("params", Params), ("amplitude", _c_double), ("result", _vp),
                ("result_is_host", _c_int)]


class Result(ctypes.Structure):
    _fields_ = [("id", ctypes.c_longlong), ("ke", _c_double), ("enstrophy", _c_double), ("t_submit", _c_double),
                ("t_admit", _c_double), ("t_done", _c_double), ("steps", _c_int), ("precision", _c_int),
                ("points", ctypes.c_longlong)]


class ServerStatus(ctypes.Structure):
    _fields_ = [("pending", _c_int), ("active", _c_int), ("completed_unpolled", _c_int), ("free_bytes", _c_size_t),
                ("largest_free_block", _c_size_t), ("arena_bytes", _c_size_t), ("ticks", ctypes.c_longlong),
                ("now", _c_double)]


SIGNATURES = {
    "sbli_abi_version": (_c_int, []),
    "sbli_workspace_bytes": (_c_int, [_c_int, _c_int, _c_int, _c_int, _c_int, ctypes.POINTER(_c_size_t)]),
    "sbli_create_grid": (_c_int, [ctypes.POINTER(_vp), _c_int, _c_int, _c_int, _c_int, _c_int,
                                  ctypes.POINTER(Params), _vp, _c_size_t, _vp]),
    "sbli_destroy_grid": (_c_int, [_vp]),
    "sbli_init_tgv": (_c_int, [_vp, _c_double]),
    "sbli_set_state": (_c_int, [_vp, _vp, _c_int]),
    "sbli_get_state": (_c_int, [_vp, _vp, _c_int]),
    "sbli_sample_state": (_c_int, [_vp, _vp, _c_int, _vp]),
    "sbli_get_stage": (_c_int, [_vp, _vp, _vp, _c_int]),
    "sbli_rhs": (_c_int, [_vp, _vp]),
    "sbli_rk_stage": (_c_int, [_vp, _c_int, _c_double]),
    "sbli_step_n": (_c_int, [_vp, _c_int, _c_double]),
    "sbli_step_n_history": (_c_int, [_vp, _c_int, _c_double, _vp]),
    "sbli_kinetic_energy": (_c_int, [_vp, _DP, _DP]),
    "sbli_kinetic_energy_async": (_c_int, [_vp, _vp]),
    "sbli_kinetic_energy_noalloc": (_c_int, [_vp, _c_int, _c_int, _c_int, _c_double, _vp, _vp]),
    "sbli_get_config": (_c_int, [_vp, ctypes.POINTER(_c_int), ctypes.POINTER(_c_int), ctypes.POINTER(_c_int),
                                 ctypes.POINTER(_c_int)]),
    "sbli_set_config": (_c_int, [_vp, _c_int, _c_int, _c_int, _c_int]),
    "sbli_autotune": (_c_int, [_vp, _c_int, ctypes.POINTER(_c_int), ctypes.POINTER(_c_int), ctypes.POINTER(_c_int),
                               ctypes.POINTER(_c_int), ctypes.POINTER(ctypes.c_float)]),
    "sbli_stage_count": (_c_int, [_vp, ctypes.POINTER(ctypes.c_longlong)]),
    "sbli_batch_workspace_bytes": (_c_int, [_c_int, _vp, _c_int, ctypes.POINTER(_c_size_t)]),
    "sbli_batch_create": (_c_int, [ctypes.POINTER(_vp), _c_int, _vp, _vp, _c_int, _vp, _c_size_t, _vp]),
    "sbli_batch_destroy": (_c_int, [_vp]),
    "sbli_batch_count": (_c_int, [_vp, ctypes.POINTER(_c_int)]),
    "sbli_batch_work_items": (_c_int, [_vp, ctypes.POINTER(ctypes.c_longlong)]),
    "sbli_batch_init_tgv": (_c_int, [_vp, _vp]),
    "sbli_batch_set_state": (_c_int, [_vp, _c_int, _vp, _c_int]),
    "sbli_batch_get_state": (_c_int, [_vp, _c_int, _vp, _c_int]),
    "sbli_batch_step_n": (_c_int, [_vp, _c_int, _c_double]),
    "sbli_batch_step_n_history": (_c_int, [_vp, _c_int, _c_double, _vp]),
    "sbli_batch_kinetic_energy": (_c_int, [_vp, _vp, _vp]),
    "sbli_batch_get_schedule": (_c_int, [_vp, ctypes.POINTER(_c_int), _vp]),
    "sbli_batch_set_schedule": (_c_int, [_vp, _c_int, _vp]),
    "sbli_batch_autotune": (_c_int, [_vp, _c_int, ctypes.POINTER(_c_int), ctypes.POINTER(ctypes.c_float)]),
    "sbli_server_create": (_c_int, [ctypes.POINTER(_vp), _vp, _c_size_t, _c_int, _c_int, _vp, _vp]),
    "sbli_server_destroy": (_c_int, [_vp]),
    "sbli_server_request_bytes": (_c_int, [ctypes.POINTER(Request), ctypes.POINTER(_c_size_t)]),
    "sbli_server_submit": (_c_int, [_vp, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_longlong)]),
    "sbli_server_tick": (_c_int, [_vp, ctypes.POINTER(_c_int)]),
    "sbli_server_poll": (_c_int, [_vp, ctypes.POINTER(Result), _c_int, ctypes.POINTER(_c_int)]),
    "sbli_server_stats": (_c_int, [_vp, ctypes.POINTER(ServerStatus)]),
    "sbli_last_error": (ctypes.c_char_p, []),
    "sbli_probe_fma_rate": (_c_int, [_c_int, ctypes.c_longlong, _vp, _vp, _DP, ctypes.POINTER(ctypes.c_float)]),
}

_lock = threading.Lock()
_lib = None


class SbliError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"sbli error {code}: {msg}")
        self.code = code


def lib() -> ctypes.CDLL:
    """Load libsbli.so (built by ``build.build()``); raises if it is missing."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() (there is no CPU fallback)")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(rc: int) -> None:
    if rc != SBLI_OK:
        raise SbliError(rc, lib().sbli_last_error().decode())


def params(Re=1600.0, Mach=0.1, Pr=0.71, gamma=1.4, L=1.0) -> Params:
    return Params(float(Re), float(Mach), float(Pr), float(gamma), float(L))


# ---- same-name wrappers of the C entry points (status codes become exceptions)

def sbli_abi_version() -> int:
    return lib().sbli_abi_version()


def sbli_workspace_bytes(n0: int, n1: int, n2: int, precision: int, variant: int) -> int:
    out = _c_size_t()
    _check(lib().sbli_workspace_bytes(n0, n1, n2, precision, variant, ctypes.byref(out)))
    return out.value


def sbli_create_grid(n0, n1, n2, precision, variant, prm: Params, workspace_ptr: int, workspace_bytes: int,
                     stream: int) -> int:
    h = _vp()
    _check(lib().sbli_create_grid(ctypes.byref(h), n0, n1, n2, precision, variant, ctypes.byref(prm),
                                  _vp(workspace_ptr), workspace_bytes, _vp(stream)))
    return h.value


def sbli_destroy_grid(h: int) -> None:
    _check(lib().sbli_destroy_grid(_vp(h)))


def sbli_init_tgv(h: int, amplitude: float = 1.0) -> None:
    _check(lib().sbli_init_tgv(_vp(h), float(amplitude)))


def sbli_set_state(h: int, q_ptr: int, q_is_host: bool) -> None:
    _check(lib().sbli_set_state(_vp(h), _vp(q_ptr), int(bool(q_is_host))))


def sbli_get_state(h: int, q_ptr: int, q_is_host: bool) -> None:
    _check(lib().sbli_get_state(_vp(h), _vp(q_ptr), int(bool(q_is_host))))


def sbli_sample_state(h: int, idx_ptr: int, count: int, out_ptr: int) -> None:
    _check(lib().sbli_sample_state(_vp(h), _vp(idx_ptr), int(count), _vp(out_ptr)))


def sbli_get_stage(h: int, q_stage_ptr: int, q_acc_ptr: int, q_is_host: bool) -> None:
    _check(lib().sbli_get_stage(_vp(h), _vp(q_stage_ptr), _vp(q_acc_ptr), int(bool(q_is_host))))


def sbli_rhs(h: int, r_ptr: int) -> None:
    _check(lib().sbli_rhs(_vp(h), _vp(r_ptr)))


def sbli_rk_stage(h: int, stage: int, dt: float) -> None:
    _check(lib().sbli_rk_stage(_vp(h), int(stage), float(dt)))


def sbli_step_n(h: int, nsteps: int, dt: float) -> None:
    _check(lib().sbli_step_n(_vp(h), int(nsteps), float(dt)))


def sbli_step_n_history(h: int, nsteps: int, dt: float, hist_ptr: int) -> None:
    _check(lib().sbli_step_n_history(_vp(h), int(nsteps), float(dt), _vp(hist_ptr)))


def sbli_kinetic_energy(h: int) -> tuple[float, float]:
    ke, ens = _c_double(), _c_double()
    _check(lib().sbli_kinetic_energy(_vp(h), ctypes.byref(ke), ctypes.byref(ens)))
    return ke.value, ens.value


def sbli_kinetic_energy_async(h: int, out_ptr: int) -> None:
    _check(lib().sbli_kinetic_energy_async(_vp(h), _vp(out_ptr)))


def sbli_kinetic_energy_noalloc(q_ptr: int, n0: int, n1: int, n2: int, L: float, out_ptr: int,
                                stream: int = 0) -> None:
    """Allocation-free KE/enstrophy of a plain device state (no grid, no workspace)."""
    _check(lib().sbli_kinetic_energy_noalloc(_vp(q_ptr), n0, n1, n2, float(L), _vp(out_ptr), _vp(stream)))


def sbli_probe_fma_rate(precision: int, iters: int, sink_ptr: int, stream: int = 0) -> tuple[float, float]:
    """FMA throughput of the current device (include/sbli_probe.h): (flop/s, kernel ms)."""
    rate, ms = _c_double(), ctypes.c_float()
    _check(lib().sbli_probe_fma_rate(int(precision), int(iters), _vp(sink_ptr), _vp(stream), ctypes.byref(rate),
                                     ctypes.byref(ms)))
    return rate.value, ms.value


def sbli_get_config(h: int) -> tuple[int, int, int, int]:
    ty, zc, zq, px = _c_int(), _c_int(), _c_int(), _c_int()
    _check(lib().sbli_get_config(_vp(h), ctypes.byref(ty), ctypes.byref(zc), ctypes.byref(zq), ctypes.byref(px)))
    return ty.value, zc.value, zq.value, px.value


def sbli_set_config(h: int, tile_y: int, planes_per_cta: int, z_queue: int = 0, columns_per_thread: int = 1) -> None:
    _check(lib().sbli_set_config(_vp(h), int(tile_y), int(planes_per_cta), int(z_queue), int(columns_per_thread)))


def sbli_autotune(h: int, reps: int = 3) -> tuple[int, int, int, int, float]:
    ty, zc, zq, px, ms = _c_int(), _c_int(), _c_int(), _c_int(), ctypes.c_float()
    _check(lib().sbli_autotune(_vp(h), int(reps), ctypes.byref(ty), ctypes.byref(zc), ctypes.byref(zq),
                               ctypes.byref(px), ctypes.byref(ms)))
    return ty.value, zc.value, zq.value, px.value, ms.value


def sbli_stage_count(h: int) -> int:
    v = ctypes.c_longlong()
    _check(lib().sbli_stage_count(_vp(h), ctypes.byref(v)))
    return v.value


def _ints(vals):
    return (ctypes.c_int * len(vals))(*[int(v) for v in vals])


def _doubles(vals):
    return (ctypes.c_double * len(vals))(*[float(v) for v in vals])


def sbli_batch_workspace_bytes(sizes, precision: int) -> int:
    flat = [v for n in sizes for v in n]
    out = _c_size_t()
    _check(lib().sbli_batch_workspace_bytes(len(sizes), ctypes.cast(_ints(flat), _vp), precision, ctypes.byref(out)))
    return out.value


def sbli_batch_create(sizes, prms, precision: int, workspace_ptr: int, workspace_bytes: int, stream: int) -> int:
    flat = [v for n in sizes for v in n]
    parr = (Params * len(prms))(*prms)
    h = _vp()
    _check(lib().sbli_batch_create(ctypes.byref(h), len(sizes), ctypes.cast(_ints(flat), _vp), ctypes.cast(parr, _vp),
                                   precision, _vp(workspace_ptr), workspace_bytes, _vp(stream)))
    return h.value


def sbli_batch_destroy(h: int) -> None:
    _check(lib().sbli_batch_destroy(_vp(h)))


def sbli_batch_count(h: int) -> int:
    v = _c_int()
    _check(lib().sbli_batch_count(_vp(h), ctypes.byref(v)))
    return v.value


def sbli_batch_work_items(h: int) -> int:
    v = ctypes.c_longlong()
    _check(lib().sbli_batch_work_items(_vp(h), ctypes.byref(v)))
    return v.value


def sbli_batch_get_schedule(h: int, count: int) -> tuple[int, list[int]]:
    """(z_queue, planes per work item of each member)."""
    zq = _c_int()
    zc = (ctypes.c_int * count)()
    _check(lib().sbli_batch_get_schedule(_vp(h), ctypes.byref(zq), ctypes.cast(zc, _vp)))
    return zq.value, list(zc)


def sbli_batch_set_schedule(h: int, z_queue: int, planes_per_item=None) -> None:
    arr = _ints(planes_per_item) if planes_per_item is not None else None
    _check(lib().sbli_batch_set_schedule(_vp(h), int(z_queue), ctypes.cast(arr, _vp) if arr is not None else None))


def sbli_batch_autotune(h: int, reps: int = 3) -> tuple[int, float]:
    """Tune the batch schedule; returns (z_queue, best stage ms)."""
    zq, ms = _c_int(), ctypes.c_float()
    _check(lib().sbli_batch_autotune(_vp(h), int(reps), ctypes.byref(zq), ctypes.byref(ms)))
    return zq.value, ms.value


def sbli_batch_init_tgv(h: int, amplitudes) -> None:
    _check(lib().sbli_batch_init_tgv(_vp(h), ctypes.cast(_doubles(amplitudes), _vp)))


def sbli_batch_set_state(h: int, member: int, q_ptr: int, q_is_host: bool) -> None:
    _check(lib().sbli_batch_set_state(_vp(h), member, _vp(q_ptr), int(bool(q_is_host))))


def sbli_batch_get_state(h: int, member: int, q_ptr: int, q_is_host: bool) -> None:
    _check(lib().sbli_batch_get_state(_vp(h), member, _vp(q_ptr), int(bool(q_is_host))))


def sbli_batch_step_n(h: int, nsteps: int, dt: float) -> None:
    _check(lib().sbli_batch_step_n(_vp(h), int(nsteps), float(dt)))


def sbli_batch_step_n_history(h: int, nsteps: int, dt: float, hist_ptr: int) -> None:
    _check(lib().sbli_batch_step_n_history(_vp(h), int(nsteps), float(dt), _vp(hist_ptr)))


def sbli_batch_kinetic_energy(h: int, count: int):
    ke = (ctypes.c_double * count)()
    ens = (ctypes.c_double * count)()
    _check(lib().sbli_batch_kinetic_energy(_vp(h), ctypes.cast(ke, _vp), ctypes.cast(ens, _vp)))
    return list(ke), list(ens)


class Batch:
    """An ensemble of grids advanced together (workspace tensor + handle)."""

    def __init__(self, sizes, precision=SBLI_FP32, Re=None, Mach=None, Pr=0.71, gamma=1.4, L=1.0, stream=None):
        import torch

        self.sizes = [(n, n, n) if isinstance(n, int) else tuple(int(v) for v in n) for n in sizes]
        count = len(self.sizes)
        Re = Re if Re is not None else [1600.0] * count
        Mach = Mach if Mach is not None else [0.1] * count
        self.prms = [params(Re[i], Mach[i], Pr, gamma, L) for i in range(count)]
        self.precision = precision
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.bytes = sbli_batch_workspace_bytes(self.sizes, precision)
        self.workspace = torch.empty(self.bytes + 256, dtype=torch.uint8, device=self.device)
        aligned = (self.workspace.data_ptr() + 255) // 256 * 256
        self.handle = sbli_batch_create(self.sizes, self.prms, precision, aligned, self.bytes, self.stream.cuda_stream)

    def close(self):
        if getattr(self, "handle", None):
            sbli_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __len__(self):
        return len(self.sizes)

    def shape(self, m):
        n = self.sizes[m]
        return (5, n[2], n[1], n[0])

    def init_tgv(self, amplitudes=None):
        sbli_batch_init_tgv(self.handle, amplitudes if amplitudes is not None else [1.0] * len(self))

    def set_state(self, m, q):
        sbli_batch_set_state(self.handle, m, q.data_ptr(), not q.is_cuda)

    def get_state(self, m, out=None):
        import torch

        if out is None:
            out = torch.empty(self.shape(m), dtype=torch.float64, device=self.device)
        sbli_batch_get_state(self.handle, m, out.data_ptr(), not out.is_cuda)
        return out

    def step_n(self, nsteps, dt):
        sbli_batch_step_n(self.handle, nsteps, dt)

    def step_n_history(self, nsteps, dt):
        import torch

        hist = torch.empty((max(nsteps, 1), len(self), 2), dtype=torch.float64, device=self.device)
        sbli_batch_step_n_history(self.handle, nsteps, dt, hist.data_ptr())
        return hist[:nsteps]

    def kinetic_energy(self):
        return sbli_batch_kinetic_energy(self.handle, len(self))

    def work_items(self):
        return sbli_batch_work_items(self.handle)

    def schedule(self):
        return sbli_batch_get_schedule(self.handle, len(self))

    def set_schedule(self, z_queue, planes_per_item=None):
        sbli_batch_set_schedule(self.handle, z_queue, planes_per_item)

    def autotune(self, reps=3):
        return sbli_batch_autotune(self.handle, reps)


def request(n, precision=SBLI_FP64, steps=10, dt=1e-3, Re=1600.0, Mach=0.1, Pr=0.71, gamma=1.4, L=1.0,
            amplitude=1.0, result=None) -> Request:
    """A solve request; ``result`` is an optional float64 tensor (5, n2, n1, n0)."""
    n = (n, n, n) if isinstance(n, int) else tuple(int(v) for v in n)
    r = Request()
    r.n0, r.n1, r.n2 = n
    r.precision, r.steps, r.dt = int(precision), int(steps), float(dt)
    r.params = params(Re, Mach, Pr, gamma, L)
    r.amplitude = float(amplitude)
    r.result = _vp(result.data_ptr()) if result is not None else None
    r.result_is_host = 0 if result is None or result.is_cuda else 1
    return r


def sbli_server_create(arena_ptr: int, arena_bytes: int, max_slots: int, backfill: bool, stream64: int,
                       stream32: int) -> int:
    h = _vp()
    _check(lib().sbli_server_create(ctypes.byref(h), _vp(arena_ptr), arena_bytes, int(max_slots), int(bool(backfill)),
                                    _vp(stream64), _vp(stream32)))
    return h.value


def sbli_server_destroy(h: int) -> None:
    _check(lib().sbli_server_destroy(_vp(h)))


def sbli_server_request_bytes(r: Request) -> int:
    out = _c_size_t()
    _check(lib().sbli_server_request_bytes(ctypes.byref(r), ctypes.byref(out)))
    return out.value


def sbli_server_submit(h: int, r: Request) -> int:
    rid = ctypes.c_longlong()
    _check(lib().sbli_server_submit(_vp(h), ctypes.byref(r), ctypes.byref(rid)))
    return rid.value


def sbli_server_tick(h: int) -> int:
    n = _c_int()
    _check(lib().sbli_server_tick(_vp(h), ctypes.byref(n)))
    return n.value


def sbli_server_poll(h: int, max_results: int = 256) -> list:
    arr = (Result * max_results)()
    n = _c_int()
    _check(lib().sbli_server_poll(_vp(h), arr, max_results, ctypes.byref(n)))
    return [arr[i] for i in range(n.value)]


def sbli_server_stats(h: int) -> ServerStatus:
    st = ServerStatus()
    _check(lib().sbli_server_stats(_vp(h), ctypes.byref(st)))
    return st


class Server:
    """Continuous-batching request loop over a device arena tensor."""

    def __init__(self, arena_bytes: int, max_slots: int = 64, backfill: bool = True):
        import torch

        self.device = torch.device("cuda", torch.cuda.current_device())
        self.s64 = torch.cuda.Stream()
        self.s32 = torch.cuda.Stream()
        self.arena = torch.empty(arena_bytes + 256, dtype=torch.uint8, device=self.device)
        aligned = (self.arena.data_ptr() + 255) // 256 * 256
        self.handle = sbli_server_create(aligned, arena_bytes, max_slots, backfill, self.s64.cuda_stream,
                                         self.s32.cuda_stream)

    def close(self):
        if getattr(self, "handle", None):
            sbli_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, r: Request) -> int:
        return sbli_server_submit(self.handle, r)

    def tick(self) -> int:
        return sbli_server_tick(self.handle)

    def poll(self) -> list:
        return sbli_server_poll(self.handle)

    def stats(self) -> ServerStatus:
        return sbli_server_stats(self.handle)


def sbli_last_error() -> str:
    return lib().sbli_last_error().decode()


# ---- convenience owner (torch tensors for memory and stream)

class Grid:
    """One grid: a workspace tensor on the current CUDA device plus a handle.

    ``n`` is an int (cube) or (n0, n1, n2).  State tensors exchanged with the
    library have shape (5, n2, n1, n0), float64, x0 fastest.
    """

    def __init__(self, n, precision=SBLI_FP64, variant=SBLI_FUSED, Re=1600.0, Mach=0.1, Pr=0.71, gamma=1.4, L=1.0,
                 stream=None, device=None):
        import torch

        self.n = (n, n, n) if isinstance(n, int) else tuple(int(v) for v in n)
        self.precision, self.variant = precision, variant
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.prm = params(Re, Mach, Pr, gamma, L)
        self.bytes = sbli_workspace_bytes(*self.n, precision, variant)
        self.workspace = torch.empty(self.bytes + 256, dtype=torch.uint8, device=self.device)
        base = self.workspace.data_ptr()
        aligned = (base + 255) // 256 * 256
        self.handle = sbli_create_grid(*self.n, precision, variant, self.prm, aligned, self.bytes,
                                       self.stream.cuda_stream)

    @property
    def shape(self):
        return (5, self.n[2], self.n[1], self.n[0])

    def close(self):
        if getattr(self, "handle", None):
            sbli_destroy_grid(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_tgv(self, amplitude=1.0):
        sbli_init_tgv(self.handle, amplitude)

    def set_state(self, q):
        import torch

        assert q.dtype == torch.float64 and q.is_contiguous() and tuple(q.shape) == self.shape
        sbli_set_state(self.handle, q.data_ptr(), not q.is_cuda)

    def get_state(self, out=None):
        import torch

        if out is None:
            out = torch.empty(self.shape, dtype=torch.float64, device=self.device)
        assert out.dtype == torch.float64 and out.is_contiguous() and tuple(out.shape) == self.shape
        sbli_get_state(self.handle, out.data_ptr(), not out.is_cuda)
        return out

    def sample_state(self, idx):
        """Plain conserved variables at linear point indices ``idx`` (int64
        device tensor, i0 + n0*(i1 + n1*i2)) as a (5, len(idx)) binary64
        device tensor; NaN where an index is outside the grid."""
        import torch

        assert idx.dtype == torch.int64 and idx.is_cuda and idx.dim() == 1
        idx = idx.contiguous()
        out = torch.empty((5, idx.numel()), dtype=torch.float64, device=self.device)
        sbli_sample_state(self.handle, idx.data_ptr(), idx.numel(), out.data_ptr())
        return out

    def rhs(self, out=None):
        import torch

        if out is None:
            out = torch.empty(self.shape, dtype=torch.float64, device=self.device)
        sbli_rhs(self.handle, out.data_ptr())
        return out

    def get_stage(self):
        """(Q_k, Q_acc) between stages, as plain binary64 device tensors."""
        import torch

        qs = torch.empty(self.shape, dtype=torch.float64, device=self.device)
        qa = torch.empty(self.shape, dtype=torch.float64, device=self.device)
        sbli_get_stage(self.handle, qs.data_ptr(), qa.data_ptr(), False)
        return qs, qa

    def rk_stage(self, stage, dt):
        sbli_rk_stage(self.handle, stage, dt)

    def step_n(self, nsteps, dt):
        sbli_step_n(self.handle, nsteps, dt)

    def step_n_history(self, nsteps, dt):
        import torch

        hist = torch.empty((max(nsteps, 1), 2), dtype=torch.float64, device=self.device)
        sbli_step_n_history(self.handle, nsteps, dt, hist.data_ptr())
        return hist[:nsteps]

    def kinetic_energy(self):
        return sbli_kinetic_energy(self.handle)

    def config(self):
        return sbli_get_config(self.handle)

    def set_config(self, tile_y, planes_per_cta, z_queue=0, columns_per_thread=1):
        sbli_set_config(self.handle, tile_y, planes_per_cta, z_queue, columns_per_thread)

    def autotune(self, reps=3):
        return sbli_autotune(self.handle, reps)

    def stage_count(self):
        return sbli_stage_count(self.handle)
