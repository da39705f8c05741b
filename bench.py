"""Benchmark of the polarized lattice-Boltzmann RT step on one B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision P] [--impl ours|reference]

Workload: the 2048 x 2048 (x, z) lattice with n = 64 directions (8 zenith x 8
azimuth, a 256 x 256 scattering contraction per site), two-layer cloud medium
(seed 1), top beam, vacuum sides.  Metric: site-direction updates per second
(one update = one (site, direction) Stokes vector advanced one step).  Prints
one JSON line.  The state (4.3 GB per buffer) is far larger than L2, so no
flush is needed between timed steps.

--impl reference times the FP64 CPU oracle on the host cores on a bounded
crop of the same workload (the oracle is the reference arm: the paper ships no
code and reports no timing).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)

from paper_2609_23057_b300 import workloads as W  # noqa: E402

METRIC = "site-direction updates/s (2048x2048 lattice, n=64)"
UNIT = "sdu/s"


def _peaks():
    try:
        with open(os.path.join(HERE, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2032.0}, "fallback"


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(rows)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cpu_baseline(steps: int, seconds: float = 12.0):
    """Oracle (FP64, OpenMP) on the 256 x 256 crop of the workload's medium:
    runs single steps until `seconds` have passed; returns sdu/s."""
    import oracle
    sys.path.insert(0, os.path.join(HERE, "tests"))
    from _util import oracle_problem
    w = W.precision_crop(steps=1)
    P = oracle_problem(oracle, w)
    S = P.zero_state()
    S = P.step(S)                       # warm-up (page-in, thread pool)
    t0 = time.perf_counter()
    k = 0
    while True:
        S = P.step(S)
        k += 1
        if time.perf_counter() - t0 >= seconds or k >= max(steps, 1000):
            break
    dt = time.perf_counter() - t0
    sdu = w.sites * w.n * k
    return {"value": sdu / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"FP64 oracle, {k} steps of the 256x256 crop [896,1152)^2 of the same "
                      f"medium (n=64), {dt:.1f} s"}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    per_step = []
    import oracle
    sys.path.insert(0, os.path.join(HERE, "tests"))
    from _util import oracle_problem
    w = W.precision_crop(steps=1)
    P = oracle_problem(oracle, w)
    S = P.zero_state()
    for _ in range(args.warmup):
        S = P.step(S)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        t = time.perf_counter()
        S = P.step(S)
        per_step.append(time.perf_counter() - t)
    dt = time.perf_counter() - t0
    sdu = w.sites * w.n * args.steps
    value = sdu / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "lattice2048_n64 (oracle on the 256x256 crop, same medium)",
                   "nx": 2048, "nz": 2048, "n_dirs": 64, "sample_sites": w.sites},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(),
                         "kind": "oracle", "sample": f"{args.steps} steps of the 256x256 crop"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    from paper_2609_23057_b300 import solver as SV

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = W.precision(seed=1, steps=args.steps)
    s = SV.solver_for(w, args.precision)
    stream = torch.cuda.current_stream(dev)
    n, sites = w.n, w.sites
    sdu_per_step = sites * n

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)

    # warm-up (also brings the state away from zero)
    s.step(args.warmup)
    barrier()

    sampler = ClockSampler(local)
    sampler.start()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    barrier()
    ev[0].record(stream)
    for k in range(args.steps):
        s.step(1)
        ev[k + 1].record(stream)
    barrier()
    clocks = sampler.stop()
    per_launch = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    total_ms = ev[0].elapsed_time(ev[-1])
    t_max = total_ms
    if ws > 1:
        import torch.distributed as dist
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_max = float(t.item())
    value = ws * sdu_per_step * args.steps / (t_max * 1e-3)

    # end to end through the public API with host buffers: each step uploads
    # the state from pinned host memory, advances one step and reads the top
    # radiance back to the host.
    e2e_steps = max(1, min(args.steps, 3))
    host_state = torch.empty((w.nz, w.nx, n, 4), dtype=torch.float32, pin_memory=True)
    s.get_state(out=host_state)
    host_top = torch.empty((w.nx, n, 4), dtype=torch.float32, pin_memory=True)
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        s.set_state(host_state)
        s.step(1)
        s.radiance_out("top", out=host_top)
    barrier()
    e2e_dt = time.perf_counter() - t0
    e2e = {"value": ws * sdu_per_step * e2e_steps / e2e_dt, "unit": UNIT,
           "h2d_bytes_per_step": host_state.numel() * 4, "d2h_bytes_per_step": host_top.numel() * 4}

    peaks, src = _peaks()
    bytes_per_sdu = 32.0 + 16.0 / n
    avg_launch_s = statistics.mean(per_launch) * 1e-3
    if args.precision == "fp32":
        flops = 32.0 * n * sdu_per_step
        smax = float(peaks.get("sm_max_mhz", 2032.0))
        peak = 148 * 128 * 2 * smax * 1e6 / 1e12
        roof = {"bound": "alu", "achieved": flops / avg_launch_s / 1e12, "peak": peak,
                "unit": "TFLOP/s", "frac": flops / avg_launch_s / 1e12 / peak, "traffic": None,
                "peak_source": f"148 SMs x 128 FP32 lanes x 2 x {smax:.0f} MHz"}
    else:
        gbs = bytes_per_sdu * sdu_per_step / avg_launch_s / 1e9
        peak = float(peaks["hbm_gbs"])
        roof = {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                "traffic": None, "peak_source": f"{src} hbm_gbs"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32", "bf16": "bf16 operands, f32 accumulate + f32 state",
                      "bf16x3": "bf16 hi+lo operands, f32 accumulate + f32 state"}[args.precision],
            "data": "synthetic",
            "config": {"workload": w.name, "nx": w.nx, "nz": w.nz, "n_dirs": n,
                       "precision": args.precision, "sites": sites, "phase_classes": 2,
                       "l2": "inputs larger than L2 (4.3 GB state per buffer)",
                       "parallelism": f"replicas{ws}" if ws > 1 else "single"},
            "roofline": roof,
            "e2e": e2e,
            "gpu_launches": args.steps,
            "clocks": clocks,
        }
        if ws == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(args.steps)
        print(json.dumps(line), flush=True)
    s.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp32", "bf16", "bf16x3"], default="fp32")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
