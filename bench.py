#!/usr/bin/env python3
"""Benchmark of the fused Navier-Stokes RHS + RK3 stage on GB300.

Main workload: Taylor-Green vortex 512^3, binary64, Re 1600, M 0.1,
dt 5e-4 (the 512^3 single-solve workload; the paper's case of section 4 of
arXiv:1709.09713 on a 512^3 grid), fused on-the-fly kernel.  One bench step is
one time step = 3 fused stages over the whole grid; the metric is point-stage
updates per second.

The JSON line carries:
  value        device-resident throughput over exactly --steps steps (CUDA
               events on the grid's stream; barrier + synchronize on both
               sides; max over ranks);
  e2e          the same metric through the public C ABI with host buffers:
               every e2e step copies the initial state from pinned host
               memory, runs --solve-steps time steps, copies the state back
               (mean of --e2e-reps steps after one untimed);
  roofline     the fused stage kernel against its binding roofline: the FP64
               pipe for binary64, whose peak is measured in the same run by
               the library's FMA-throughput probe (clocks sampled meanwhile);
               HBM for the binary32 paths;
  legs         binary32 storage at 512^3 (both accumulators, 200 steps, HBM
               roofline), double-float arithmetic at 512^3, the paper's
               algorithm classes (store-all BL ... SN2) at 256^3, the 64-member
               ensemble and the serving traces;
  energy       NVML total-energy delta per point-stage over the timed region;
  cpu_baseline the CPU oracle (unchanged) on a bounded sample of the workload.
``--impl reference`` times only the CPU oracle (the reference arm).
Multi-GPU (torchrun): independent replicas, one grid per rank (weak scaling).
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0

# Algorithmic HBM bytes per point-stage of the fused kernel, averaged over
# the three stages of a step (minimum traffic of the two-register scheme):
#   binary64: 50 values per point-step / 3 * 8 B = 133.3 B
#   binary32 stage fields + binary64 accumulator: 320 B / 3 = 106.7 B
ALG_BYTES = {"fp64": 400.0 / 3.0, "fp32": 320.0 / 3.0, "fp32df": 320.0 / 3.0, "df64": 400.0 / 3.0}

# Counters of the stage kernels taken with ncu (profiles/), per point-stage,
# each valid for the kernel sources whose hash is given (KERNEL_SOURCES under
# paper_1709_09713_gb300/csrc); bench.py reports a counter as stale (null)
# once the sources differ.
#   fp64 flop_per_pt: binary64 flop executed (2 DFMA + DADD + DMUL), mean of
#        the three stages of a 256^3 step; traffic_per_pt: DRAM read + write
#        bytes per point of one launch, same capture (2.2499e9 per launch at
#        256^3; scaled by points to other grids);
#   df64 inst_per_pt: thread instructions (smsp__inst_executed x 32 / points),
#        mean of the three stages of a 256^3 step, per z-queue mode.
KERNEL_SOURCES = ["fused_stage.cuh", "fused_fp64.cu", "fused_df64.cu", "dfloat.cuh", "fpconv.cuh", "f32x2.cuh",
                  "sbli_internal.cuh"]
KERNEL_COUNTS = {
    "fp64": {"flop_per_pt": 568.44, "traffic_per_pt": 2.2499e9 / 256**3, "sources": "651ecf03b0a6",
             "profile": "profiles/fused_stage_fp64_256.md"},
    "df64": {"inst_per_pt": {0: 3727.1, 1: 3693.1}, "sources": "651ecf03b0a6",
             "profile": "profiles/fused_stage_df64_256.md"},
}


def kernel_sources_hash() -> str:
    import hashlib

    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1709_09713_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:12]


def kernel_count(precision: str, key: str):
    """A counter of KERNEL_COUNTS if it was taken on the current sources, else None."""
    c = KERNEL_COUNTS.get(precision)
    if not c or key not in c or c["sources"] != kernel_sources_hash():
        return None
    return c[key]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32", "fp32df", "df64"],
                    help="main line precision: binary64 (default), binary32 storage with a binary64 or "
                         "double-float accumulator, or binary64 storage with double-float arithmetic")
    ap.add_argument("--variant", default="fused", choices=["fused", "store_all"])
    ap.add_argument("--alg-steps", type=int, default=24,
                    help="steps per algorithm class in the comparison leg (>= ~1 s each for NVML energy)")
    ap.add_argument("--dt", type=float, default=None,
                    help="time step (default 5e-4 for n >= 512, the linear stability limit there, else 1e-3)")
    ap.add_argument("--solve-steps", type=int, default=10, help="time steps per e2e solve")
    ap.add_argument("--e2e-reps", type=int, default=3, help="timed e2e solves (mean), after one untimed")
    ap.add_argument("--no-legs", action="store_true", help="skip the FP32 512^3 and store-all legs")
    ap.add_argument("--leg-steps", type=int, default=200, help="time steps of the 512^3 binary32 legs")
    ap.add_argument("--df64-leg-steps", type=int, default=40)
    ap.add_argument("--ens-steps", type=int, default=40)
    ap.add_argument("--serve-requests", type=int, default=24)
    ap.add_argument("--serve-requests-low", type=int, default=10)
    ap.add_argument("--serve-rate-low", type=float, default=1.0)
    ap.add_argument("--serve-nmax", type=int, default=256)
    ap.add_argument("--serve-steps-hi", type=int, default=2000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-planes", type=int, default=8,
                    help="the oracle's bounded sample: a periodic n x n x planes slab of the workload's planes")
    ap.add_argument("--cpu-sample-steps", type=int, default=2)
    ap.add_argument("--profile", choices=["stage", "algorithms", "ensemble"], default=None,
                    help="untimed runs for ncu: 'stage' = --steps steps of one grid (--n, --profile-precision, "
                         "--profile-variant) stage by stage; 'algorithms' = stage 0 of every binary64 "
                         "algorithm class at --n; 'ensemble' = --steps steps of the first --profile-members "
                         "members of the seeded ensemble (--profile-precision)")
    ap.add_argument("--probe", action="store_true",
                    help="only measure the FMA peaks (binary64, binary32) with the library's probe, clocks sampled")
    ap.add_argument("--profile-members", type=int, default=16)
    ap.add_argument("--profile-precision", default="fp64", choices=sorted(PRECISIONS))
    ap.add_argument("--profile-variant", default="fused", choices=sorted(VARIANTS))
    ap.add_argument("--profile-config", default=None, help="tile_y,planes_per_cta,z_queue (default: the grid's)")
    args = ap.parse_args()
    if args.dt is None:
        args.dt = 5e-4 if args.n >= 512 else 1e-3
    return args


def run_profile(args):
    """Work for profiler captures: no timing, prints "ok"."""
    import torch

    from paper_1709_09713_gb300 import build as B
    from paper_1709_09713_gb300 import sbli as S

    if not os.path.exists(S.LIB_PATH):
        B.build()
    S.lib()
    if args.profile == "stage":
        g = S.Grid(args.n, PRECISIONS[args.profile_precision], VARIANTS[args.profile_variant])
        if args.profile_config:
            g.set_config(*(int(x) for x in args.profile_config.split(",")))
        g.init_tgv(1.0)
        for _ in range(args.steps):
            for k in range(3):
                g.rk_stage(k, args.dt)
        torch.cuda.synchronize()
        g.close()
    elif args.profile == "ensemble":
        from paper_1709_09713_gb300 import workloads

        members = workloads.ensemble(64, seed=1709)[: args.profile_members]
        b = S.Batch([m.n for m in members], PRECISIONS[args.profile_precision], Re=[m.Re for m in members],
                    Mach=[m.Mach for m in members])
        b.init_tgv([m.amplitude for m in members])
        b.step_n(args.steps, args.dt)
        torch.cuda.synchronize()
        b.close()
    else:
        for name in ("store_all", "RS", "SS", "RA", "SN", "SN2", "fused"):
            g = S.Grid(args.n, S.SBLI_FP64, VARIANTS[name])
            g.init_tgv(1.0)
            g.rk_stage(0, args.dt)
            torch.cuda.synchronize()
            g.close()
            del g
            torch.cuda.empty_cache()
    print("ok")


# ------------------------------------------------------------ clocks, NVML

class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons, power = [], None, set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
                power.append(float(parts[3]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm), "power_w_median": statistics.median(power) if power else None}


class Nvml:
    """Total-energy counter of one GPU through libnvidia-ml (ctypes)."""

    def __init__(self, index: int):
        self.ok = False
        try:
            self.lib = ctypes.CDLL("libnvidia-ml.so.1")
            if self.lib.nvmlInit_v2() != 0:
                return
            self.dev = ctypes.c_void_p()
            if self.lib.nvmlDeviceGetHandleByIndex_v2(index, ctypes.byref(self.dev)) != 0:
                return
            self.ok = self.energy_mj() is not None
        except OSError:
            pass

    def energy_mj(self):
        v = ctypes.c_ulonglong()
        if self.lib.nvmlDeviceGetTotalEnergyConsumption(self.dev, ctypes.byref(v)) != 0:
            return None
        return v.value


# --------------------------------------------------------------- helpers

def measured_peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": FALLBACK_HBM_GBS}, "fallback"


def dist_env():
    return int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0"))


def dist_max(x: float) -> float:
    """Maximum of x over all ranks (identity without a process group).  Works
    with nccl (CUDA tensor) and gloo (CPU tensor)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_barrier() -> None:
    import torch.distributed as dist

    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def weak_scaling_value(units_per_rank: float, seconds_this_rank: float) -> tuple[float, float]:
    """Whole-job throughput of independent replicas: all ranks' units over the
    slowest rank's time.  Returns (value, max_seconds)."""
    import torch.distributed as dist

    ws = dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1
    t = dist_max(seconds_this_rank)
    return units_per_rank * ws / t, t


def oracle_slab_sample(n: int, planes: int, steps: int, threads: int):
    """The CPU oracle, unchanged, on a bounded sample of the n^3 workload: the
    Taylor-Green vortex on a periodic n x n x `planes` slab (same points per
    x2 plane and the same arithmetic per point as the full grid; `planes`/n
    of its points), `steps` time steps on `threads` host threads.  Returns
    (pt-stage/s, seconds, threads used)."""
    import oracle

    oracle.build()
    oracle.set_threads(threads)
    p = oracle.params((n, n, planes))
    q = oracle.init_tgv(p)
    t0 = time.perf_counter()
    oracle.step(p, q, 1e-3, steps)
    el = time.perf_counter() - t0
    return n * n * planes * 3 * steps / el, el, oracle.get_threads()


def cpu_baseline(n: int, planes: int, steps: int):
    """The oracle on all host cores, plus one time step of a narrower slab on one core."""
    v, el, cores = oracle_slab_sample(n, planes, steps, os.cpu_count() or 1)
    rows = max(5, n // 4)
    v1, el1, _ = oracle_slab_sample_rows(n, rows, planes)
    return {"value": v, "unit": "pt-stage/s", "cores": cores, "kind": "oracle",
            "sample": f"TGV {n} x {n} x {planes} periodic slab (the {n}^3 workload's planes), FP64, {steps} time "
                      f"steps ({3 * steps} stages) in {el:.2f} s",
            "single_thread": {"value": v1, "unit": "pt-stage/s", "cores": 1,
                              "sample": f"TGV {n} x {rows} x {planes} periodic slab, FP64, 1 time step in {el1:.2f} s"}}


def oracle_slab_sample_rows(n: int, rows: int, planes: int):
    """One time step of an n x rows x planes slab on one host thread."""
    import oracle

    oracle.build()
    cores = oracle.get_threads()
    oracle.set_threads(1)
    p = oracle.params((n, rows, planes))
    q = oracle.init_tgv(p)
    t0 = time.perf_counter()
    oracle.step(p, q, 1e-3, 1)
    el = time.perf_counter() - t0
    oracle.set_threads(cores)
    return n * rows * planes * 3 / el, el, 1


def probe_peak(S, precision, seconds, gpu_index):
    """FMA throughput of this GPU (the library's probe), run for about
    `seconds` with nvidia-smi clocks sampled meanwhile."""
    import torch

    sink = torch.zeros(1, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    rate, ms = S.sbli_probe_fma_rate(precision, 2000, sink.data_ptr())
    iters = max(2000, int(2000 * seconds * 1e3 / max(ms, 1e-3)))
    clocks = ClockSampler(gpu_index)
    clocks.start()
    time.sleep(0.3)
    rate, ms = S.sbli_probe_fma_rate(precision, iters, sink.data_ptr())
    clk = clocks.stop()
    return {"flop_per_s": rate, "ms": ms, "iters": iters, "clocks": clk}


def time_steps(S, g, stream, steps, dt, ws):
    """CUDA-event time of exactly `steps` steps on the grid's stream, max over ranks."""
    import torch

    dist_barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    g.step_n(steps, dt)
    e1.record(stream)
    e1.synchronize()
    torch.cuda.synchronize()
    dist_barrier()
    return dist_max(e0.elapsed_time(e1))


def energy_per_pt_stage(g, stream, points, stage_ms, dt, nvml, seconds=1.0):
    """NVML total-energy delta per point-stage over about `seconds` of
    further steps (long enough for the counter's resolution), or None."""
    import torch

    if nvml is None or not nvml.ok:
        return None
    steps = max(1, int(seconds * 1e3 / (3.0 * stage_ms)))
    torch.cuda.synchronize()
    e0 = nvml.energy_mj()
    g.step_n(steps, dt)
    stream.synchronize()
    e1 = nvml.energy_mj()
    if e0 is None or e1 is None or e1 <= e0:
        return None
    return {"j_per_pt_stage": (e1 - e0) / 1e3 / (3.0 * points * steps), "steps": steps,
            "source": "nvmlDeviceGetTotalEnergyConsumption delta over further steps after the timed ones"}


def ensemble_leg(S, steps, warmup, dt, ws, count=64, seed=1709, nvml=None, precision=None, tune=True):
    """64 Taylor-Green members, N uniform over {32,48,64,96,128}, Re ~ U[100,1600],
    M ~ U[0.1,0.4], amplitude ~ U(0.9,1.1); binary32 stages with a binary64
    accumulator (or, precision SBLI_FP32_DF, a double-float one); one
    persistent launch per stage, graph-captured steps, schedule (z-queue mode,
    planes per work item per size class) picked by the batch autotuner."""
    import torch

    from paper_1709_09713_gb300 import workloads

    members = workloads.ensemble(count, seed=seed)
    prec = S.SBLI_FP32 if precision is None else precision
    stream = torch.cuda.Stream()
    b = S.Batch([m.n for m in members], prec, Re=[m.Re for m in members], Mach=[m.Mach for m in members],
                stream=stream)
    with torch.cuda.stream(stream):
        b.init_tgv([m.amplitude for m in members])
    default_items = b.work_items()
    zq, tuned_ms = b.autotune(3) if tune else (b.schedule()[0], None)
    zq, zc = b.schedule()
    by_n = {}
    for m, z in zip(members, zc):
        by_n.setdefault(str(m.n), z)
    with torch.cuda.stream(stream):
        b.step_n(max(warmup, 6), dt)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.step_n(steps, dt)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    pts = sum(m.n**3 for m in members)
    items = b.work_items()
    energy = energy_per_pt_stage(b, stream, pts, ms / (3 * steps), dt, nvml)
    b.close()
    del b
    torch.cuda.empty_cache()
    acc = "f64 accumulator" if prec == S.SBLI_FP32 else "double-float accumulator"
    peaks, kind = measured_peaks()
    ach = ALG_BYTES["fp32"] * pts / (ms / (3 * steps) / 1e3) / 1e9
    return {"workload": f"ensemble of {count} TGV grids (N in {{32,48,64,96,128}}, Re U[100,1600], M U[0.1,0.4]), "
                        f"fp32 + {acc}, persistent launch per stage", "value": 3.0 * pts * steps * ws / (ms / 1e3),
            "unit": "pt-stage/s", "steps": steps, "points": pts, "work_items_per_stage": items,
            "stage_ms": ms / (3 * steps), "launches_per_stage": 1, "energy": energy,
            "schedule": {"autotuned": bool(tune), "z_queue": zq, "planes_per_item_by_n": by_n,
                         "work_items_default_schedule": default_items, "tuned_stage0_ms": tuned_ms},
            "hbm": {"achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": ach / peaks["hbm_gbs"],
                    "peak_source": kind, "bytes_per_pt_stage": ALG_BYTES["fp32"]}}


def serving_leg(S, count, rate_hz, nmin, nmax, steps_lo, steps_hi, seed=20, arena_gb=200.0, fp64_as=0):
    """Poisson arrivals of TGV solve requests (grid edge log-uniform, step
    count uniform, FP64/FP32 flag 50/50) replayed in wall-clock time against
    the continuous-batching server; latency = completion - arrival.
    fp64_as: the precision FP64-flagged requests run in (SBLI_FP64, or
    SBLI_DF64: the same 1e-12 bar in double-float arithmetic)."""
    import torch

    from paper_1709_09713_gb300 import workloads

    trace = workloads.request_trace(count, seed=seed, rate_hz=rate_hz, nmin=nmin, nmax=nmax, steps_lo=steps_lo,
                                    steps_hi=steps_hi)
    free, _ = torch.cuda.mem_get_info()
    arena = int(min(arena_gb * 2**30, free * 0.8))
    srv = S.Server(arena, max_slots=64, backfill=True)
    t0 = time.perf_counter()
    nxt, res, arrival = 0, {}, {}
    while len(res) < count:
        now = time.perf_counter() - t0
        while nxt < count and trace[nxt].arrival_s <= now:
            q = trace[nxt]
            prec = fp64_as if q.precision == S.SBLI_FP64 else q.precision
            rid = srv.submit(S.request(q.n, prec, q.steps, 1e-3, Re=q.Re, Mach=q.Mach, amplitude=q.amplitude))
            arrival[rid] = q.arrival_s
            nxt += 1
        st = srv.stats()
        if st.active == 0 and st.pending == 0 and nxt < count:
            time.sleep(max(0.0, min(0.01, trace[nxt].arrival_s - now)))
            continue
        srv.tick()
        for r in srv.poll():
            res[r.id] = (r, time.perf_counter() - t0)
    wall = time.perf_counter() - t0
    srv.close()
    del srv
    torch.cuda.empty_cache()
    lat = sorted(done_t - arrival[rid] for rid, (r, done_t) in res.items())
    work = sum(3.0 * r.points * r.steps for r, _ in res.values())

    def pct(v, p):
        return v[min(len(v) - 1, int(round(p / 100.0 * (len(v) - 1))))] if v else None

    def lane_lat(f64_lane):
        v = sorted(done_t - arrival[rid] for rid, (r, done_t) in res.items()
                   if (r.precision in (S.SBLI_FP64, S.SBLI_DF64)) == f64_lane)
        return {"requests": len(v), "p50_latency_s": pct(v, 50), "p99_latency_s": pct(v, 99)}

    f64 = "fp64" if fp64_as == S.SBLI_FP64 else "fp64 (double-float arithmetic)"
    return {"workload": f"serving: {count} Poisson requests at {rate_hz} req/s, N log-uniform [{nmin},{nmax}], "
                        f"steps U{{{steps_lo}..{steps_hi}}}, {f64}/fp32 50/50, dt 1e-3",
            "value": work / wall, "unit": "pt-stage/s", "requests": count, "wall_s": wall,
            "p50_latency_s": pct(lat, 50), "p99_latency_s": pct(lat, 99), "max_latency_s": lat[-1],
            "by_lane": {"fp64_lane": lane_lat(True), "fp32_lane": lane_lat(False)},
            "offered_pt_stage_per_s": sum(3.0 * q.n**3 * q.steps for q in trace) / max(trace[-1].arrival_s, 1e-9)}


PRECISIONS = {"fp64": 0, "fp32": 1, "fp32df": 2, "df64": 3}
VARIANTS = {"fused": 0, "store_all": 1, "RS": 2, "SS": 3, "RA": 4, "SN": 5, "SN2": 6}


def leg(S, n, precision, variant, steps, warmup, dt, ws, tune=False, clock_ghz=None, nvml=None):
    """Throughput of one extra configuration (no e2e, no clocks)."""
    import torch

    stream = torch.cuda.Stream()
    prec = PRECISIONS[precision]
    var = S.SBLI_FUSED if variant == "fused" else S.SBLI_STORE_ALL
    g = S.Grid(n, prec, var, stream=stream)
    with torch.cuda.stream(stream):
        g.init_tgv(1.0)
    cfg = list(g.autotune(3)[:4]) if tune else (list(g.config()) if var == S.SBLI_FUSED else None)
    with torch.cuda.stream(stream):
        g.step_n(warmup, dt)
    ms = time_steps(S, g, stream, steps, dt, ws)
    P = n**3
    stage_ms = ms / (3 * steps)
    energy = energy_per_pt_stage(g, stream, P, stage_ms, dt, nvml)
    g.close()
    del g
    torch.cuda.empty_cache()
    out = {"workload": f"TGV {n}^3 {precision} {variant}, dt {dt}", "value": 3.0 * P * steps * ws / (ms / 1e3),
           "unit": "pt-stage/s", "steps": steps, "stage_ms": stage_ms, "config": cfg,
           "config_fields": "tile_y, planes_per_cta, z_queue, columns_per_thread", "autotuned": bool(tune),
           "energy": energy}
    if variant == "fused":
        peaks, kind = measured_peaks()
        ach = ALG_BYTES[precision] * P / (stage_ms / 1e3) / 1e9
        out["hbm"] = {"achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": ach / peaks["hbm_gbs"],
                      "peak_source": kind, "bytes_per_pt_stage": ALG_BYTES[precision]}
        if precision == "fp32":
            # the last stage also writes the binary32 copy of the new state and
            # stage 0 reads it: 360 B per point-step moved against the 320 B minimum
            out["hbm"]["bytes_moved_per_pt_stage"] = 120.0
            out["hbm"]["frac_of_bytes_moved"] = 120.0 * P / (stage_ms / 1e3) / 1e9 / peaks["hbm_gbs"]
        inst = kernel_count("df64", "inst_per_pt") if precision == "df64" else None
        inst = inst.get(cfg[2]) if inst and cfg else None  # the count of the z-queue mode in use
        if inst and clock_ghz:
            sms = torch.cuda.get_device_properties(0).multi_processor_count
            peak = sms * 4 * 32 * clock_ghz * 1e9
            rate = inst * P / (stage_ms / 1e3)
            out["issue"] = {"achieved": rate, "peak": peak, "unit": "thread-instr/s", "frac": rate / peak,
                            "note": f"{inst:.0f} instructions per pt-stage ({KERNEL_COUNTS['df64']['profile']}); "
                                    f"peak = {sms} SMs x 4 sub-partitions x 32 lanes x {clock_ghz:.3f} GHz"}
    return out


def algorithms_leg(S, n, steps, warmup, dt, ws, nvml):
    """The paper's algorithm classes (section 2.3) on the binary64 Taylor-Green
    vortex: the tiled fused kernel, store-all (BL), intermediate storage (RS,
    SS) and one-thread-per-point minimal storage (RA, SN, SN2).  Throughput,
    joules per pt-stage (NVML energy over each timed region), and speed-up and
    energy saving relative to BL as the paper tabulates them."""
    import torch

    rows = []
    for var in (S.SBLI_STORE_ALL, S.SBLI_RS, S.SBLI_SS, S.SBLI_RA, S.SBLI_SN, S.SBLI_SN2, S.SBLI_FUSED):
        stream = torch.cuda.Stream()
        g = S.Grid(n, S.SBLI_FP64, var, stream=stream)
        with torch.cuda.stream(stream):
            g.init_tgv(1.0)
            g.step_n(warmup, dt)
        stream.synchronize()
        e0 = nvml.energy_mj() if nvml.ok else None
        ms = time_steps(S, g, stream, steps, dt, ws)
        e1 = nvml.energy_mj() if nvml.ok else None
        g.close()
        del g
        torch.cuda.empty_cache()
        pts = 3.0 * n**3 * steps
        row = {"algorithm": S.VARIANT_NAMES[var], "value": pts * ws / (ms / 1e3), "stage_ms": ms / (3 * steps)}
        if e0 is not None and e1 is not None and e1 > e0:  # the counter may not advance over a short region
            row["j_per_pt_stage"] = (e1 - e0) / 1e3 / pts
        rows.append(row)
    bl = rows[0]
    for r in rows:
        r["speedup_vs_bl"] = bl["stage_ms"] / r["stage_ms"]
        if "j_per_pt_stage" in r and "j_per_pt_stage" in bl:
            r["energy_saving_vs_bl"] = bl["j_per_pt_stage"] / r["j_per_pt_stage"]
    return {"workload": f"TGV {n}^3 fp64, Re 1600, M 0.1, dt {dt}: the paper's algorithm classes",
            "unit": "pt-stage/s", "steps": steps, "rows": rows}


# ------------------------------------------------------------- our arm

def workload_name(args) -> str:
    return (f"TGV {args.n}^3 {args.precision} {args.variant}, Re 1600, M 0.1, Pr 0.71, gamma 1.4, "
            f"dt {args.dt:g}")


def run_ours(args):
    import torch

    from paper_1709_09713_gb300 import build as B
    from paper_1709_09713_gb300 import sbli as S

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    if not os.path.exists(S.LIB_PATH):
        B.build()
    S.lib()
    prec = PRECISIONS[args.precision]
    var = S.SBLI_FUSED if args.variant == "fused" else S.SBLI_STORE_ALL
    n, dt, P = args.n, args.dt, args.n**3

    # the binary64 FMA peak of this GPU, measured now (the ALU roofline's denominator)
    fp64_probe = probe_peak(S, S.SBLI_FP64, 1.0, local)

    stream = torch.cuda.Stream()
    g = S.Grid(n, prec, var, stream=stream)
    with torch.cuda.stream(stream):
        g.init_tgv(1.0)
        g.step_n(args.warmup, dt)
    stream.synchronize()
    cfg = list(g.config()) if var == S.SBLI_FUSED else None

    nvml = Nvml(torch.cuda.current_device())
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    e_before = nvml.energy_mj() if nvml.ok else None
    ms = time_steps(S, g, stream, args.steps, dt, ws)
    e_after = nvml.energy_mj() if nvml.ok else None
    clk = clocks.stop()
    value = 3.0 * P * args.steps * ws / (ms / 1e3)
    stage_ms = ms / (3 * args.steps)  # one fused launch per stage

    # e2e: initial state from pinned host memory, --solve-steps steps, state back
    q_host = torch.empty(g.shape, dtype=torch.float64, pin_memory=True)
    r_host = torch.empty(g.shape, dtype=torch.float64, pin_memory=True)
    g.init_tgv(1.0)
    g.get_state(q_host)
    e2e_t = []
    for rep in range(1 + args.e2e_reps):  # the first, untimed, touches the pinned buffers and graphs once
        dist_barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S.sbli_set_state(g.handle, q_host.data_ptr(), True)
        S.sbli_step_n(g.handle, args.solve_steps, dt)
        S.sbli_get_state(g.handle, r_host.data_ptr(), True)
        torch.cuda.synchronize()
        if rep > 0:
            e2e_t.append(time.perf_counter() - t0)
    t_e2e = dist_max(sum(e2e_t) / len(e2e_t))
    state_bytes = 5 * P * 8
    g.close()
    del g, q_host, r_host
    torch.cuda.empty_cache()

    peaks, kind = measured_peaks()
    src = kernel_sources_hash()
    if prec in (S.SBLI_FP64, S.SBLI_DF64) and var == S.SBLI_FUSED:
        hbm_frac = ALG_BYTES[args.precision] * P / (stage_ms / 1e3) / 1e9 / peaks["hbm_gbs"]
    if prec == S.SBLI_FP64 and var == S.SBLI_FUSED:
        flop = kernel_count("fp64", "flop_per_pt")
        tpp = kernel_count("fp64", "traffic_per_pt")
        peak_tf = fp64_probe["flop_per_s"] / 1e12
        ach = flop * P / (stage_ms / 1e3) / 1e12 if flop else None
        roof = {"bound": "alu", "achieved": ach, "peak": peak_tf, "unit": "TFLOP/s",
                "frac": ach / peak_tf if ach else None, "traffic": tpp * P if tpp else None,
                "note": f"binary64 FMA pipe; {flop} flop per pt-stage executed ({KERNEL_COUNTS['fp64']['profile']}, "
                        f"kernel sources {KERNEL_COUNTS['fp64']['sources']}, current {src}); peak measured in this "
                        f"run by sbli_probe_fma_rate (independent DFMA chains on every SM, "
                        f"{fp64_probe['ms']:.0f} ms, median SM clock {fp64_probe['clocks'].get('sm_mhz')} MHz); "
                        f"traffic = DRAM bytes per point of one 256^3 launch (ncu) x points",
                "peak_source": "measured (probe, this run)", "hbm_frac": hbm_frac,
                "hbm_peak_gbs": peaks["hbm_gbs"]}
    elif prec == S.SBLI_DF64 and var == S.SBLI_FUSED:
        inst = kernel_count("df64", "inst_per_pt")
        inst = inst.get(cfg[2]) if inst and cfg else None
        clock_ghz = (clk.get("sm_mhz") or 2070.0) / 1e3
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        peak = sms * 4 * 32 * clock_ghz * 1e9
        ach = inst * P / (stage_ms / 1e3) if inst else None
        roof = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "thread-instr/s",
                "frac": ach / peak if ach else None, "traffic": None,
                "note": f"binary32 issue: {inst} instructions per pt-stage (ncu); peak = {sms} SMs x "
                        f"4 sub-partitions x 32 lanes x {clock_ghz:.3f} GHz", "hbm_frac": hbm_frac}
    else:
        ach = ALG_BYTES[args.precision] * P / (stage_ms / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": ach / peaks["hbm_gbs"], "traffic": None, "peak_source": kind}

    line = {
        "metric": "pt-stage updates/s",
        "value": value,
        "unit": "pt-stage/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"fp64": "f64", "fp32": "f32 (f64 accumulator)", "fp32df": "f32 (f32-pair accumulator)",
                  "df64": "f32 pairs (double-float), f64 storage"}[args.precision],
        "data": "synthetic (Taylor-Green vortex initial field of section 4)",
        "config": {"workload": workload_name(args), "grid": [n, n, n],
                   "l2": f"inputs larger than L2 ({state_bytes / 2**20:.0f} MiB state register)",
                   "parallelism": f"independent replicas x{ws}", "launch_config": cfg,
                   "launch_config_fields": "tile_y, planes_per_cta, z_queue, columns_per_thread"},
        "e2e": {"value": 3.0 * P * args.solve_steps * ws / t_e2e, "unit": "pt-stage/s",
                "h2d_bytes_per_step": state_bytes, "d2h_bytes_per_step": state_bytes,
                "note": f"each e2e step = H2D state + {args.solve_steps} time steps + D2H state; mean of "
                        f"{args.e2e_reps} after one untimed"},
        "roofline": roof,
        "fp64_peak_probe": {"tflops": fp64_probe["flop_per_s"] / 1e12, "ms": fp64_probe["ms"],
                            "clocks": fp64_probe["clocks"]},
        "clocks": clk,
        "gpu_launches": 3 * args.steps,
        "stage_ms": stage_ms,
    }
    if e_before is not None and e_after is not None:
        joules = (e_after - e_before) / 1e3
        line["energy"] = {"joules": joules, "j_per_pt_stage": joules / (3.0 * P * args.steps),
                          "source": "nvmlDeviceGetTotalEnergyConsumption delta over the timed region"}
    if not args.no_legs:
        cg = (clk.get("sm_mhz") or 2070.0) / 1e3
        line["legs"] = [leg(S, 512, "fp32", "fused", args.leg_steps, 2, 5e-4, ws, tune=True, nvml=nvml),
                        leg(S, 512, "fp32df", "fused", args.leg_steps, 2, 5e-4, ws, tune=True, nvml=nvml),
                        leg(S, 512, "df64", "fused", args.df64_leg_steps, 2, 5e-4, ws, tune=True, clock_ghz=cg,
                            nvml=nvml),
                        leg(S, 256, "df64", "fused", 3 * args.df64_leg_steps, 2, 1e-3, ws, tune=True, clock_ghz=cg,
                            nvml=nvml),
                        algorithms_leg(S, 256, args.alg_steps, 1, 1e-3, ws, nvml),
                        ensemble_leg(S, args.ens_steps, 6, 1e-3, ws, nvml=nvml),
                        ensemble_leg(S, args.ens_steps, 6, 1e-3, ws, nvml=nvml, precision=S.SBLI_FP32_DF),
                        # the serving distribution: N log-uniform [32,256], steps U{50..2000}, FP64/FP32 50/50
                        serving_leg(S, args.serve_requests, 20.0, 32, args.serve_nmax, 50, args.serve_steps_hi),
                        serving_leg(S, args.serve_requests, 20.0, 32, args.serve_nmax, 50, args.serve_steps_hi,
                                    fp64_as=S.SBLI_DF64),
                        # below saturation: latency close to each request's own service time
                        serving_leg(S, args.serve_requests_low, args.serve_rate_low, 32, args.serve_nmax, 50,
                                    args.serve_steps_hi, fp64_as=S.SBLI_DF64)]
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(n, args.cpu_sample_planes, args.cpu_sample_steps)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def run_reference(args):
    """The reference arm: the CPU oracle as it stands, on the host cores, on a
    bounded sample of the main line's workload (an n x n x planes periodic
    slab of its grid's planes per step)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle

    oracle.build()
    oracle.set_threads(os.cpu_count() or 1)
    n, planes = args.n, args.cpu_sample_planes
    p = oracle.params((n, n, planes))
    q = oracle.init_tgv(p)
    q = oracle.step(p, q, args.dt, args.warmup)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        q = oracle.step(p, q, args.dt, 1)
    el = time.perf_counter() - t0
    pts = n * n * planes
    value = 3.0 * pts * args.steps / el
    sample = (f"each step: one time step of the Taylor-Green vortex on a periodic {n} x {n} x {planes} slab "
              f"(the {n}^3 workload's points per x2 plane and arithmetic per point, {planes}/{n} of its points) "
              f"on the CPU oracle")
    line = {
        "impl": "reference", "metric": "pt-stage updates/s", "value": value, "unit": "pt-stage/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (Taylor-Green vortex of section 4)",
        "config": {"workload": workload_name(args), "grid": [n, n, n], "sample": sample},
        "cpu_baseline": {"value": value, "unit": "pt-stage/s", "cores": oracle.get_threads(), "kind": "oracle",
                         "sample": f"TGV {n} x {n} x {planes} slab, {args.steps} time steps after {args.warmup} "
                                   f"warm-up steps"},
        "e2e": {"value": value, "unit": "pt-stage/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_probe(args):
    """The binary64 and binary32 FMA peaks of this GPU, three times each."""
    import torch

    from paper_1709_09713_gb300 import build as B
    from paper_1709_09713_gb300 import sbli as S

    torch.cuda.set_device(0)
    if not os.path.exists(S.LIB_PATH):
        B.build()
    S.lib()
    out = {"fp64": [], "fp32": []}
    for name, prec in (("fp64", S.SBLI_FP64), ("fp32", S.SBLI_FP32)):
        for _ in range(3):
            r = probe_peak(S, prec, 1.0, 0)
            out[name].append({"tflops": r["flop_per_s"] / 1e12, "ms": r["ms"], "sm_mhz": r["clocks"].get("sm_mhz"),
                              "reasons": r["clocks"].get("reasons")})
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.probe:
        run_probe(args)
    elif args.profile:
        run_profile(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
