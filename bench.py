#!/usr/bin/env python3
"""Benchmark of the HWENO hot path: 2D Euler cell-updates per second per RK stage.

Workload: 2D Euler (gamma = 1.4) four-quadrant Riemann data on [0,1]^2, 2048 x 2048
cells, transmissive boundaries, KXRCF troubled-cell modification, CFL 0.6.
One bench step = one whole pass of the hot path: the CFL wave-speed reduction
(hweno_max_dt) and one SSP-RK3 step (hweno_step: three stages of reconstruct,
indicator + modification, troubled re-reconstruction, fluxes + quadrature +
update).  value = cells * 3 stages * steps / device time, FP64 (the scheme as
specified); the FP32-bulk form is timed beside it and reported under "forms"
with its relative L1 difference to FP64.

Multi-GPU (torchrun): each rank advances its own independently seeded problem
(weak scaling, no data-path collective); the timing barrier and the max over
ranks use torch.distributed.

--impl reference times the CPU FP64 oracle (the reference arm of this build)
on a bounded window of the same workload.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N = 2048
CFL = 0.6
WORKLOAD = "2d_euler_four_quadrant_2048x2048"
METRIC = "2D Euler cell-updates/s (per RK stage)"
UNIT = "cell-updates/s"
# Algorithmic work of one reconstruction of one variable in one cell, as the kernel
# evaluates it (mirror-parity form): split + smoothness indicators + point values
# (counted by the table generator, D2_FLOP_SBV in hweno_parity.h) plus beta_1 and the
# nonlinear weights (112 flop, a division counted as one).  Per cell add the 44 flop
# of the KXRCF face-velocity partials and norm (Euler).


def _rec_flop_per_cell(nvar=4):
    import re
    with open(os.path.join(ROOT, "paper_2201_12193_gb300", "csrc", "hweno_parity.h")) as f:
        sbv = int(re.search(r"D2_FLOP_SBV = (\d+);", f.read()).group(1))
    return nvar * (sbv + 112) + 44
# algorithmic HBM bytes per cell-stage: read U^(k) (12 doubles), read U^n for stages 2-3, write U^(k+1)
ALGO_BYTES_PER_CELL_STAGE = 12 * 8 * (1 + 2.0 / 3.0 + 1)
FP64_PEAK_NOMINAL = 1.25e12   # GB300 FP64 FLOP/s (nominal)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N, help=argparse.SUPPRESS)
    ap.add_argument("--no-forms", action="store_true", help="skip the FP32-bulk form")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32"],
                    help="form of the main measurement (fp64 = the scheme as specified)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched form")
    ap.add_argument("--no-cpu", action="store_true")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples (200 ms) while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.index)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ distributed plumbing

def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if os.environ.get("HWENO_BENCH_GLOO") is None else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ oracle timing (CPU)

def oracle_window(p, half):
    """A (2*half)^2 window of the problem around its centre (four-quadrant split)."""
    import oracle
    c = p.nx // 2
    sub = np.ascontiguousarray(p.m[:, :, c - half:c + half, c - half:c + half])
    cfg = oracle.make_cfg(2, 2 * half, 2 * half, dx=p.dx, dy=p.dy, eq="euler", gamma=p.gamma,
                          bc=("transmissive",) * 4)
    return oracle, cfg, sub


def time_oracle(p, half, steps):
    """The oracle as it stands (single thread) on `steps` SSP-RK3 steps of a window."""
    oracle, cfg, m = oracle_window(p, half)
    oracle.build()
    t0 = time.perf_counter()
    for _ in range(steps):
        m, _, rc = oracle.step(cfg, m, oracle.max_dt(cfg, m, CFL))
        if rc != 0:
            raise RuntimeError("oracle step failed")
    dt = time.perf_counter() - t0
    cells = (2 * half) ** 2
    return cells * 3 * steps / dt, dt, f"{2 * half}x{2 * half} centre window of the {p.nx}x{p.ny} workload, " \
                                       f"{steps} SSP-RK3 step(s) ({cells * 3 * steps} cell-updates)"


# ------------------------------------------------------------------ our arm

def run_solver(torch, hweno, p, precision, steps, warmup, world, profile=False, clocks=None):
    s = hweno.Solver.from_problem(p, precision=precision)
    s.set_stream(torch.cuda.current_stream())
    s.set_moments(torch.from_numpy(p.m).cuda())
    for _ in range(warmup):
        s.step(s.max_dt(CFL))
    s.sync()
    if profile:
        s.profile(True)
    barrier(world)
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
        time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        s.step(s.max_dt(CFL))
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop() if clocks else None
    barrier(world)
    prof = s.profile_read() if profile else None
    s.profile(False)
    out = torch.empty(s.shape, dtype=torch.float64, device="cuda")
    s.get_moments(out)
    s.sync()
    return s, ms, prof, clk, out


def run_batched(torch, hweno, args, world, rank):
    """The batched form: 256 independent problems (sizes seeded uniformly in
    {64,128,256,512}^2; four-quadrant on [0,1]^2 and isentropic vortices on periodic
    [0,10]^2), one persistent launch per RK stage replayed from a CUDA graph, the
    update tile picked by the autotuner; FP32 bulk, and FP64 for the L1 comparison."""
    from paper_2201_12193_gb300 import autotune, workloads as W
    probs = W.batch_problems(256, seed=rank, npts=2)
    # Four-quadrant seeds whose solution leaves the physical set (the scheme has no
    # positivity limiter) are rejected and redrawn, and logged in the bench line.
    rejected = []
    for attempt in range(8):
        bad = set()
        for prec in ("fp32", "fp64"):
            s = hweno.BatchSolver(probs, precision=prec)
            for k, p in enumerate(probs):
                s.set_moments(k, torch.from_numpy(p.m).cuda())
            try:
                for _ in range(args.warmup + args.steps):
                    s.step()
                s.sync()
            except hweno.HwenoError:
                bad |= set(s.failed_problems())
            s.close()
        if not bad:
            break
        for k in sorted(bad):
            rejected.append({"problem": k, "seed": probs[k].seed, "n": probs[k].nx})
            new_seed = probs[k].seed + 7919 * (attempt + 1)
            probs[k] = W.four_quadrant_2d(probs[k].nx, seed=new_seed) if k % 2 == 0 else \
                W.vortex_2d(probs[k].nx, seed=new_seed, npts=2)
    cells = sum(p.nx * p.ny for p in probs)
    variant, tune_ms = autotune.tune_batch(probs, precision="fp32", steps=2)
    out = {}
    finals = {}
    for prec in ("fp32", "fp64"):
        s = hweno.BatchSolver(probs, precision=prec, stream=torch.cuda.current_stream())
        s.set_tile(variant)
        for k, p in enumerate(probs):
            s.set_moments(k, torch.from_numpy(p.m).cuda())
        steps = args.steps if prec == "fp32" else max(2, args.steps // 3)
        for _ in range(args.warmup):
            s.step()
        s.sync()
        barrier(world)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            s.step()
        e1.record()
        torch.cuda.synchronize()
        ms = max_over_ranks(e0.elapsed_time(e1), world)
        s.sync()
        graph = s.uses_graph()
        # the same number of steps for both precisions before comparing
        for _ in range(args.steps - steps if prec == "fp64" else 0):
            s.step()
        s.sync()
        finals[prec] = [s.get_moments(k) for k in range(0, len(probs), 8)]
        s.close()
        out[f"batched_{prec}"] = {"value": cells * 3 * steps * world / (ms * 1e-3), "ms_per_step": ms / steps,
                                  "problems": len(probs), "cells": cells, "graph": graph,
                                  "tile": autotune.VARIANTS[variant], "launches_per_step": 3}
    num = sum(float(np.abs(a - b).sum()) for a, b in zip(finals["fp32"], finals["fp64"]))
    den = sum(float(np.abs(b).sum()) for b in finals["fp64"])
    out["batched_fp32"]["rel_l1_vs_fp64_after_steps"] = num / den
    out["batched_fp32"]["tune_ms_per_step"] = {autotune.VARIANTS[int(k)]: v for k, v in tune_ms.items()}
    out["batched_fp32"]["rejected_seeds"] = rejected
    return out


def run_ours(args, world, rank, local):
    import torch

    from paper_2201_12193_gb300 import build, hweno, workloads as W
    torch.cuda.set_device(local)
    build.build()
    p = W.four_quadrant_2d(args.n, seed=rank)
    cells = p.nx * p.ny
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    smi_index = vis.split(",")[local] if vis and vis.split(",")[local].strip().isdigit() else local
    clocks = ClockSampler(smi_index)

    s64, ms, prof, clk, out64 = run_solver(torch, hweno, p, args.precision, args.steps, args.warmup, world,
                                           profile=True, clocks=clocks)
    ms = max_over_ranks(ms, world)
    value = cells * 3 * args.steps * world / (ms * 1e-3)
    ms_step = ms / args.steps

    # roofline of the dominant kernel (largest share of device time)
    kind, (kms, kn) = max(prof.items(), key=lambda kv: kv[1][0])
    total_kernel_ms = sum(v[0] for v in prof.values())
    flop = _rec_flop_per_cell(s64.nvar) * cells * kn if kind == "reconstruct" else None
    roof = None
    if flop:
        achieved = flop / (kms * 1e-3)
        roof = {"bound": "alu", "kernel": f"rec2d<double,4> ({kind})", "achieved": achieved / 1e12,
                "peak": FP64_PEAK_NOMINAL / 1e12, "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_NOMINAL,
                "peak_source": "GB300 nominal FP64 1.25 TFLOP/s (recipe table); FMA probe measured 1.05",
                "traffic": None, "launches": kn, "avg_ms": kms / kn, "share": kms / total_kernel_ms}
    kernels = {k: {"ms": v[0], "launches": v[1], "share": v[0] / total_kernel_ms} for k, v in prof.items()}
    hbm = {"algorithmic_GBps": ALGO_BYTES_PER_CELL_STAGE * cells * 3 * args.steps / (ms * 1e-3) / 1e9,
           "peak_GBps": 6796.2}
    hbm["frac"] = hbm["algorithmic_GBps"] / hbm["peak_GBps"]
    launches = sum(v[1] for v in prof.values()) + 2 * args.steps     # + wave-speed reduction kernels
    s64.close()

    forms = {}
    if not args.no_forms:
        s32, ms32, prof32, _, out32 = run_solver(torch, hweno, p, "fp32", args.steps, args.warmup, world,
                                                 profile=True)
        ms32 = max_over_ranks(ms32, world)
        a = out32.cpu().numpy()
        b = out64.cpu().numpy()
        forms["fp32bulk"] = {"value": cells * 3 * args.steps * world / (ms32 * 1e-3), "ms_per_step": ms32 / args.steps,
                             "dtype": "f32 (state and RK accumulation f64)",
                             "rel_l1_vs_fp64_after_steps": float(np.abs(a - b).sum() / np.abs(b).sum()),
                             "steps_compared": args.warmup + args.steps,
                             "kernels": {k: {"ms": v[0], "launches": v[1]} for k, v in prof32.items()}}
        s32.close()

    if not args.no_forms and not args.no_batch:
        forms.update(run_batched(torch, hweno, args, world, rank))

    e2e = None
    if not args.no_e2e:
        # through the public API with host buffers: H2D of the state, the step, D2H of the state
        s = hweno.Solver.from_problem(p, precision="fp64")
        host = torch.from_numpy(p.m.copy()).pin_memory()
        res = torch.empty_like(host).pin_memory()
        s.set_moments(host.numpy())
        s.step(s.max_dt(CFL))
        s.get_moments(res.numpy())
        k = max(2, min(args.steps, 4))
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(k):
            s.set_moments(host.numpy())
            s.step(s.max_dt(CFL))
            s.get_moments(res.numpy())
        t = max_over_ranks(time.perf_counter() - t0, world)
        e2e = {"value": cells * 3 * k * world / t, "unit": UNIT, "steps": k,
               "h2d_bytes_per_step": int(host.numel() * 8), "d2h_bytes_per_step": int(res.numel() * 8)}
        s.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        v, secs, sample = time_oracle(p, 128, 1)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample, "seconds": secs}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": WORKLOAD, "nx": p.nx, "ny": p.ny, "precision": "fp64", "indicator": "kxrcf",
                           "cfl": CFL, "seed_per_rank": "rank", "parallelism": f"replicas x{world}",
                           "l2": "inputs larger than L2 (state 403 MB, point values 2.1 GB per stage)"},
                "roofline": roof, "hbm": hbm, "kernels": kernels, "forms": forms, "e2e": e2e, "cpu_baseline": cpu,
                "gpu_launches": launches * 1, "clocks": clk}
        print(json.dumps(line))


# ------------------------------------------------------------------ reference arm (the oracle)

def run_reference(args, world, rank):
    if rank != 0:
        return
    from paper_2201_12193_gb300 import workloads as W
    p = W.four_quadrant_2d(args.n, seed=0)
    half = 64
    oracle, cfg, m = oracle_window(p, half)
    oracle.build()
    for _ in range(args.warmup):
        m, _, _ = oracle.step(cfg, m, oracle.max_dt(cfg, m, CFL))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        m, _, rc = oracle.step(cfg, m, oracle.max_dt(cfg, m, CFL))
        if rc != 0:
            raise RuntimeError("oracle step failed")
    secs = time.perf_counter() - t0
    cells = (2 * half) ** 2
    value = cells * 3 * args.steps / secs
    sample = f"{2 * half}x{2 * half} centre window of the {p.nx}x{p.ny} workload per step"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "nx": p.nx, "ny": p.ny, "precision": "fp64", "indicator": "kxrcf",
                       "cfl": CFL, "sample": sample},
            "cpu_baseline": {"kind": "oracle", "cores": 1, "sample": sample, "value": value, "unit": UNIT},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    args = parse()
    world, rank, local = dist_init()
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
