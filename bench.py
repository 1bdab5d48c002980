#!/usr/bin/env python3
"""Benchmark of the fused Navier-Stokes RHS + RK3 stage on GB300.

Workload (default): Taylor-Green vortex 256^3, binary64, Re 1600, M 0.1,
dt 1e-3 (§4 of arXiv:1709.09713 at the paper's grid size).  One bench step is
one time step = 3 fused stages over the whole grid; the metric is
point-stage updates per second (grid points x stages / s).

Legs printed in the one JSON line:
  value      device-resident throughput over exactly --steps steps (CUDA
             events on the grid's stream, barrier + synchronize on both sides,
             max over ranks);
  e2e        the same metric through the public C ABI with host buffers:
             every e2e step copies the initial state from pinned host memory,
             runs --solve-steps time steps and copies the final state back;
  roofline   the dominant kernel against its binding roofline;
  cpu_baseline  the CPU oracle (as it stands) on a bounded sample.
``--impl reference`` times only the CPU oracle (the reference arm).
Multi-GPU (torchrun): independent replicas, one grid per rank (weak scaling).
"""
from __future__ import annotations

import argparse
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

# Algorithmic HBM bytes per point-stage of the fused kernel (minimum traffic,
# averaged over the three stages of a step):
#   binary64: 50 values per point-step / 3 stages * 8 B = 133.3 B
#   binary32 stage fields + binary64 accumulator: 320 B / 3 = 106.7 B
ALG_BYTES = {0: 400.0 / 3.0, 1: 320.0 / 3.0}
# binary64 FLOPs per point-stage executed by the fused kernel (DADD + DMUL +
# 2 DFMA counted by ncu on the 256^3 stage; see profiles/).
FUSED_FP64_FLOPS_PER_PT = None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32"])
    ap.add_argument("--variant", default="fused", choices=["fused", "store_all"])
    ap.add_argument("--dt", type=float, default=1e-3)
    ap.add_argument("--solve-steps", type=int, default=10, help="time steps per e2e solve")
    ap.add_argument("--e2e-reps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-n", type=int, default=64)
    ap.add_argument("--cpu-sample-steps", type=int, default=2)
    return ap.parse_args()


# ----------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms."""

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
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
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
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------- helpers

def measured_peaks():
    try:
        with open(PEAKS_FILE) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": FALLBACK_HBM_GBS}, "fallback"


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cpu_baseline(n: int, steps: int, dt: float):
    """Time the CPU oracle (unchanged) on an n^3 TGV for `steps` time steps."""
    import oracle

    oracle.build()
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    p = oracle.params(n)
    q = oracle.init_tgv(p)
    t0 = time.perf_counter()
    oracle.step(p, q, dt, steps)
    el = time.perf_counter() - t0
    pts = n**3 * 3 * steps
    return {"value": pts / el, "unit": "pt-stage/s", "cores": oracle.get_threads(), "kind": "oracle",
            "sample": f"TGV {n}^3 FP64, {steps} time steps ({3 * steps} stages), {el:.2f} s"}


# ------------------------------------------------------------- our arm

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
    prec = S.SBLI_FP64 if args.precision == "fp64" else S.SBLI_FP32
    var = S.SBLI_FUSED if args.variant == "fused" else S.SBLI_STORE_ALL
    n, dt = args.n, args.dt
    stream = torch.cuda.Stream()
    g = S.Grid(n, prec, var, stream=stream)
    P = n**3

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    # warm-up (also builds the step graphs)
    with torch.cuda.stream(stream):
        g.init_tgv(1.0)
        for _ in range(args.warmup):
            g.step_n(1, dt)
    stream.synchronize()

    # device-resident timed region: exactly K steps
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    g.step_n(args.steps, dt)
    e1.record(stream)
    e1.synchronize()
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    ms_max = ms
    if ws > 1:
        t = torch.tensor([ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms_max = float(t.item())
    pt_stages = 3.0 * P * args.steps * ws
    value = pt_stages / (ms_max / 1e3)

    # per-launch duration of the dominant kernel: one stage = one launch
    stage_ms = ms / (3 * args.steps)

    # e2e through the C ABI with host buffers
    q_host = torch.empty(g.shape, dtype=torch.float64).pin_memory()
    r_host = torch.empty(g.shape, dtype=torch.float64).pin_memory()
    g.init_tgv(1.0)
    g.get_state(q_host)
    e2e_times = []
    for _ in range(args.e2e_reps):
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S.sbli_set_state(g.handle, q_host.data_ptr(), True)
        S.sbli_step_n(g.handle, args.solve_steps, dt)
        S.sbli_get_state(g.handle, r_host.data_ptr(), True)
        torch.cuda.synchronize()
        e2e_times.append(time.perf_counter() - t0)
    e2e_t = min(e2e_times)
    if ws > 1:
        t = torch.tensor([e2e_t], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e_t = float(t.item())
    e2e_value = 3.0 * P * args.solve_steps * ws / e2e_t
    state_bytes = 5 * P * 8

    peaks, kind = measured_peaks()
    if prec == S.SBLI_FP32 and var == S.SBLI_FUSED:
        alg = ALG_BYTES[1] * P
        achieved = alg / (stage_ms / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": None, "peak_source": kind}
    else:
        alg = ALG_BYTES[0] * P
        achieved = alg / (stage_ms / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": None, "peak_source": kind}

    line = {
        "metric": "pt-stage updates/s",
        "value": value,
        "unit": "pt-stage/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64" if prec == S.SBLI_FP64 else "f32 (f64 accumulator)",
        "data": "synthetic (Taylor-Green vortex initial field, section 4)",
        "config": {"workload": f"TGV {n}^3 {args.precision} {args.variant}, Re 1600, M 0.1, dt {dt}",
                   "grid": [n, n, n], "l2": "inputs larger than L2 (state register "
                   f"{state_bytes / 2**20:.0f} MiB > 129 MB)", "parallelism": f"replicas x{ws}"},
        "e2e": {"value": e2e_value, "unit": "pt-stage/s", "h2d_bytes_per_step": state_bytes,
                "d2h_bytes_per_step": state_bytes, "solve_steps": args.solve_steps},
        "roofline": roof,
        "clocks": clk,
        "gpu_launches": 3 * args.steps,
        "stage_ms": stage_ms,
    }
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.cpu_sample_n, args.cpu_sample_steps, dt)
    g.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    per_step = []
    import oracle

    oracle.build()
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    n = args.cpu_sample_n
    p = oracle.params(n)
    q = oracle.init_tgv(p)
    for _ in range(args.warmup):
        q = oracle.step(p, q, args.dt, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        q = oracle.step(p, q, args.dt, 1)
    el = time.perf_counter() - t0
    value = 3.0 * n**3 * args.steps / el
    line = {
        "impl": "reference", "metric": "pt-stage updates/s", "value": value, "unit": "pt-stage/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (Taylor-Green vortex, section 4)",
        "config": {"workload": f"TGV {args.n}^3 {args.precision} {args.variant}, Re 1600, M 0.1, dt {args.dt}",
                   "sample": f"CPU oracle on the {n}^3 TGV (bounded sample of the workload)"},
        "cpu_baseline": {"value": value, "unit": "pt-stage/s", "cores": oracle.get_threads(), "kind": "oracle",
                         "sample": f"TGV {n}^3, {args.steps} time steps"},
        "e2e": {"value": value, "unit": "pt-stage/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
