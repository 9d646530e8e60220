#!/usr/bin/env python3
"""Benchmark of the HWENO hot path: 2D Euler cell-updates per second per RK stage.

Workload: 2D Euler (gamma = 1.4) four-quadrant Riemann data on [0,1]^2, 2048 x 2048
cells, transmissive boundaries, KXRCF troubled-cell modification, CFL 0.6.
One bench step = one whole pass of the hot path: the CFL wave-speed reduction
(hweno_max_dt) and one SSP-RK3 step (hweno_step: three stages of reconstruct,
indicator + modification, troubled re-reconstruction, fluxes + quadrature +
update).  value = cells * 3 stages * steps / device time, FP64 (the scheme as
specified).  Under "forms": the FP32-bulk and double-float forms (relative L1
difference to FP64), the 1D Shu-Osher problem run whole (device-driven against
the host loop; FP32-bulk and double-float beside FP64 with the N = 4000 vs 8000
resolution gap), the batched form (256 problems of uneven size, one persistent
launch per stage, CUDA graph), and the learned-indicator form on 4096^2 blast
data against the plain scheme on the same data (throughputs, network roofline,
recall / miss / false-alarm rates against KXRCF, L1 drift).  --full-run adds the
2048^2 problem run whole to t = 0.25 in FP64 and FP32-bulk.

Multi-GPU (torchrun): the 2048^2 grid is split into one row slab per rank; the
4-row halos travel between neighbouring ranks (NCCL point to point) before
every Runge-Kutta stage and the CFL wave speeds are max-reduced (strong
scaling); the timing barrier and the max over ranks use torch.distributed.

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
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-indicator form")
    ap.add_argument("--no-1d", action="store_true", help="skip the 1D Shu-Osher full run")
    ap.add_argument("--no-fused", action="store_true", help="skip the fused-stage forms")
    ap.add_argument("--dmr", action="store_true",
                    help="also run Example 3.9 (double Mach reflection) at 1600 x 400 to t = 0.2")
    ap.add_argument("--step", action="store_true",
                    help="also run Example 3.10 (forward-facing step) at 600 x 200 to t = 4")
    ap.add_argument("--full-run", action="store_true",
                    help="also run the 2048^2 four-quadrant problem to t = 0.25 in FP64 and FP32-bulk")
    ap.add_argument("--learned-n", type=int, default=4096, help=argparse.SUPPRESS)
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
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate(cells_per_rank, stages, steps, world, ms_max):
    """Whole-job throughput: the cell-updates all ranks did over the slowest
    rank's time (weak scaling: every rank advances its own problem)."""
    return cells_per_rank * stages * steps * world / (ms_max * 1e-3)


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


def _oracle_worker(args):
    """One pool worker: the oracle on its own window, one SSP-RK3 step (spawned)."""
    n, seed, half, start = args
    import time as _t
    from paper_2201_12193_gb300 import workloads as W
    p = W.four_quadrant_2d(n, seed=seed)
    oracle, cfg, m = oracle_window(p, half)
    oracle.build()
    while _t.time() < start:          # all workers start together
        _t.sleep(0.001)
    t0 = _t.perf_counter()
    m, _, rc = oracle.step(cfg, m, oracle.max_dt(cfg, m, CFL))
    return (2 * half) ** 2 * 3, _t.perf_counter() - t0, rc


def time_oracle_all_cores(n, half):
    """The oracle as it stands, one process per host core (spawned pool), each
    on the same-size window for one step; value = all cell-updates over the
    slowest worker's time."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(int, range(cores))    # workers up before the clock starts
        start = time.time() + 3.0
        res = pool.map(_oracle_worker, [(n, 0, half, start)] * cores)
    if any(r[2] != 0 for r in res):
        raise RuntimeError("oracle step failed")
    work = sum(r[0] for r in res)
    slow = max(r[1] for r in res)
    return work / slow, cores, slow


# ------------------------------------------------------------------ our arm

def run_solver(torch, hweno, p, precision, steps, warmup, world, profile=False, clocks=None, fused=False):
    s = hweno.Solver.from_problem(p, precision=precision)
    if fused:
        s.set_fused(True)
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
    for prec in ("fp32", "fp64", "df64"):
        s = hweno.BatchSolver(probs, precision=prec, stream=torch.cuda.current_stream())
        s.set_tile(variant)
        for k, p in enumerate(probs):
            s.set_moments(k, torch.from_numpy(p.m).cuda())
        steps = args.steps if prec != "fp64" else max(2, args.steps // 3)
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
        out[f"batched_{prec}"] = {"value": aggregate(cells, 3, steps, world, ms), "ms_per_step": ms / steps,
                                  "problems": len(probs), "cells": cells, "graph": graph,
                                  "tile": autotune.VARIANTS[variant], "launches_per_step": 3}
    den = sum(float(np.abs(b).sum()) for b in finals["fp64"])
    for prec in ("fp32", "df64"):
        num = sum(float(np.abs(a - b).sum()) for a, b in zip(finals[prec], finals["fp64"]))
        out[f"batched_{prec}"]["rel_l1_vs_fp64_after_steps"] = num / den
    out["batched_fp32"]["tune_ms_per_step"] = {autotune.VARIANTS[int(k)]: v for k, v in tune_ms.items()}
    out["batched_fp32"]["rejected_seeds"] = rejected
    return out


MLP_FLOP_PER_CELL = 2 * (108 * 64 + 64 * 64 + 64)    # 11,072 multiply-adds per cell


KERNEL_SOURCES = ("hweno_2d_kernels.cuh", "hweno_device.cuh", "hweno_parity.h", "hweno_internal.h", "hweno_fused.cuh",
                  "df64.cuh")
# FP32-bulk update kernel, bytes per cell and launch that its inputs and outputs
# fix: point values 4 x 16 x 4 B, U^(k) 96 B, U^n 96 B in two stages of three
# (64 B on average), U^(k+1) 96 B and its float copy 48 B
UPD32_BYTES_PER_CELL = 256 + 96 + 64 + 96 + 48


# the fused 1D stage kernel's sources (its ncu figures: profiles/dram_traffic_1d.json)
KERNEL_SOURCES_1D = ("hweno_fused1d.cuh", "hweno_1d.cu", "hweno_device.cuh", "hweno_parity.h", "df64.cuh")
# fused 1D stage, bytes per cell and launch: U^(k) 48 B, U^n 48 B in two stages
# of three (32 B on average), U^(k+1) 48 B, the troubled mask 1 B and the
# previous stage's mask 1 B in two of three
FUSED1D_BYTES_PER_CELL = 48 + 32 + 48 + 1 + 2.0 / 3.0


def source_hash(sources=KERNEL_SOURCES):
    """SHA-256 of kernel sources (a committed ncu figure holds only for them)."""
    import hashlib
    h = hashlib.sha256()
    for f in sources:
        with open(os.path.join(ROOT, "paper_2201_12193_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def traffic_per_cell(kernel, table="dram_traffic.json", sources=KERNEL_SOURCES):
    """DRAM bytes per cell of one launch of `kernel` from the committed ncu
    figures (profiles/<table>), or None when the kernel sources changed since
    that capture."""
    try:
        with open(os.path.join(ROOT, "profiles", table)) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    k = d.get("kernels", {}).get(kernel)
    if not k or d.get("source_sha256") != source_hash(sources):
        return None
    return float(k["bytes_per_cell"])


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


HBM_FALLBACK_GBPS = 6800.0


def hbm_peak():
    """(GB/s, source): the measured copy bandwidth, else the recipe's fallback."""
    v = _peaks().get("hbm_gbs")
    return (float(v), "MEASURED_PEAKS.json hbm_gbs (of measured)") if v else \
        (HBM_FALLBACK_GBPS, "recipe fallback 6.8 TB/s (of fallback)")


def alu_peaks(hweno):
    """FP64 and FP32 FMA throughput measured on this device now (hweno_alu_probe,
    best of 3 launches), and the nominal FP64 figure derived from the unit
    counts: 2 FP64 FMA per clock per SM x 152 SMs x 2070 MHz x 2 flop."""
    f64 = max(hweno.alu_probe("fp64") for _ in range(3))
    f32 = max(hweno.alu_probe("fp32") for _ in range(3))
    return {"fp64_tflops": f64 / 1e12, "fp32_tflops": f32 / 1e12,
            "fp64_nominal_tflops": 2 * 2 * 152 * 2.07e9 / 1e12,
            "how": "hweno_alu_probe: 8 independent FMA chains per thread, 4 x 256 threads per SM, "
                   "CUDA events, best of 3 (of measured)"}


def run_shu_osher(torch, hweno, world):
    """The 1D Shu-Osher problem (N = 4000, transmissive, to t = 1.8, CFL 0.6): a
    latency-bound run of ~5,800 small steps (192 KB of state) on the fused 1D
    stage (the 1D default: one launch per Runge-Kutta stage).  FP64 timed whole,
    device-driven (hweno_advance: dt formed on the device, graph replays of 12
    steps) against the host-driven loop (hweno_max_dt + hweno_step) and against
    the four-launch pipeline (the same states bit for bit); the FP32-bulk
    and double-float forms run device-driven to the same time, each with the
    relative L1 difference of its final state to the FP64 run's (all moments, and
    cell averages alone) and the troubled cells per stage.  For scale, the same
    difference between the FP64 runs at N = 4000 and N = 8000 (cell averages of
    the fine run summed in pairs): the scheme's own resolution error."""
    from paper_2201_12193_gb300 import workloads as W
    p = W.shu_osher_1d(4000)
    out = {}
    finals = {}
    for mode, prec, nx in (("advance", "fp64", 4000), ("host_loop", "fp64", 4000), ("advance_pipeline", "fp64", 4000),
                           ("advance_fp32", "fp32", 4000), ("advance_df64", "df64", 4000),
                           ("advance_n8000", "fp64", 8000)):
        q = p if nx == 4000 else W.shu_osher_1d(nx)
        s = hweno.Solver.from_problem(q, precision=prec)
        if mode == "advance_pipeline":
            s.set_fused(False)     # the four-launch stage (the fused stage is the 1D default)
        s.set_stream(torch.cuda.current_stream())
        s.set_moments(torch.from_numpy(q.m).cuda())
        s.run(0.01) if mode == "host_loop" else s.advance(0.01)      # warm-up (graph capture)
        s.set_moments(torch.from_numpy(q.m).cuda())
        s.sync()
        s.rerecon_count()
        barrier(world)
        t0 = time.perf_counter()
        if mode == "host_loop":
            n = s.run(1.8, CFL)
        else:
            _, n = s.advance(1.8, CFL)
        secs = max_over_ranks(time.perf_counter() - t0, world)
        finals[mode] = s.get_moments()
        out[mode] = {"value": aggregate(q.nx, 3, n, world, secs * 1e3), "steps": n, "seconds": secs,
                     "us_per_step": secs * 1e6 / n, "troubled_per_stage": s.rerecon_count() / (3.0 * n)}
        s.close()
    ref = finals["advance"]

    def rel(a, b):
        return float(np.abs(a - b).sum() / np.abs(b).sum())
    for mode in ("advance_fp32", "advance_df64"):
        out[mode]["rel_l1_to_fp64"] = rel(finals[mode], ref)
        out[mode]["rel_l1_averages_to_fp64"] = rel(finals[mode][:, 0], ref[:, 0])
    fine = finals["advance_n8000"][:, 0, 0]
    coarse = 0.5 * (fine[:, 0::2] + fine[:, 1::2])
    same = bool(np.array_equal(finals["advance"], finals["host_loop"]))
    same_pipe = bool(np.array_equal(finals["advance"], finals["advance_pipeline"]))
    return {"shu_osher_1d_full_run": {"workload": "1d_euler_shu_osher_4000_to_t1.8", "dtype": "f64",
                                      "value": out["advance"]["value"], "unit": UNIT, "device_driven": out["advance"],
                                      "host_driven": out["host_loop"], "identical_states": same,
                                      "stage": "fused (one launch per Runge-Kutta stage)",
                                      "pipeline": out["advance_pipeline"],
                                      "identical_states_fused_vs_pipeline": same_pipe,
                                      "fp32bulk": out["advance_fp32"], "df64": out["advance_df64"],
                                      "resolution_gap_averages_n4000_vs_n8000": rel(ref[:, 0, 0], coarse),
                                      "n8000_troubled_per_stage": out["advance_n8000"]["troubled_per_stage"]}}


def run_shu_osher_long(torch, hweno, world, hbm_gbps, hbm_src, nx=1 << 24):
    """Shu-Osher data on 2^24 cells (transmissive, CFL 0.6, 805 MB of state per
    copy, far above L2) in the FP32-bulk form: the fused 1D stage kernel (one
    launch per Runge-Kutta stage) against HBM.  Its algorithmic bytes per cell
    and launch are the stage's inputs and outputs (FUSED1D_BYTES_PER_CELL); the
    duration is the CUDA-event time of its launches on the solver's stream."""
    from paper_2201_12193_gb300 import workloads as W
    p = W.shu_osher_1d(nx)
    s = hweno.Solver.from_problem(p, precision="fp32")
    s.set_stream(torch.cuda.current_stream())
    s.set_moments(torch.from_numpy(p.m).cuda())
    del p
    dt = s.max_dt(CFL)
    for _ in range(3):
        s.step(dt)
    s.sync()
    s.profile(True)
    s.profile_read()
    s.rerecon_count()
    steps = 5
    barrier(world)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        s.step(dt)
    e1.record()
    torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1), world)
    prof = s.profile_read()
    rer = s.rerecon_count()
    s.close()
    f_ms, f_n = prof["fused_stage"]
    out = {"workload": f"1d_euler_shu_osher_{nx}", "dtype": "f32 (state and RK accumulation f64)",
           "value": aggregate(nx, 3, steps, world, ms), "unit": UNIT, "ms_per_step": ms / steps,
           "rerecon_cells_per_stage": rer / (3.0 * steps),
           "kernels": {k: {"ms": v[0], "launches": v[1]} for k, v in prof.items() if v[1]}}
    if f_n:
        gbs = FUSED1D_BYTES_PER_CELL * nx * f_n / (f_ms * 1e-3) / 1e9
        t = traffic_per_cell("fused1d_fp32", "dram_traffic_1d.json", KERNEL_SOURCES_1D)
        out["roofline_fused_stage"] = {
            "bound": "hbm", "achieved": gbs, "peak": hbm_gbps, "unit": "GB/s", "frac": gbs / hbm_gbps,
            "peak_source": hbm_src, "bytes_per_cell": FUSED1D_BYTES_PER_CELL, "avg_ms": f_ms / f_n,
            "traffic": t * nx if t else None,
            "note": "the FP64 pipe, not HBM, binds: ncu shows it 72 % busy (the Runge-Kutta combination and "
                    "the flux differences of the average equation stay in FP64)"}
    return {"shu_osher_1d_long_fp32": out}


def run_four_quadrant_full(torch, hweno, world, rank):
    """The four-quadrant problem (2048^2, seeded quadrant states) run whole to
    t = 0.25, device-driven, in FP64 and FP32-bulk: steps, time,
    cell-updates/s and the relative L1 difference of each final state to the
    FP64 run's.  A seed whose FP64 run leaves the physical set is redrawn and
    listed.  Not part of the default run (about a quarter of an hour)."""
    from paper_2201_12193_gb300 import workloads as W
    rejected = []
    seed = rank
    out, finals, reached = {}, {}, {}

    def run(p, prec):
        s = hweno.Solver.from_problem(p, precision=prec)
        try:
            s.set_stream(torch.cuda.current_stream())
            s.set_moments(torch.from_numpy(p.m).cuda())
            s.sync()
            t0 = time.perf_counter()
            try:
                t, n = s.advance(0.25, CFL)
            except hweno.HwenoError:
                try:
                    reached[prec] = s.time()     # the start of the 12-step replay that failed
                except hweno.HwenoError:
                    pass
                raise
            secs = time.perf_counter() - t0
            finals[prec] = s.get_moments()
            out[prec] = {"value": aggregate(p.nx * p.ny, 3, n, 1, secs * 1e3), "steps": n, "seconds": secs,
                         "t": t, "troubled_fraction_last_stage": float(s.troubled_mask()[-1].mean())}
        finally:
            s.close()

    while True:
        p = W.four_quadrant_2d(N, seed=seed)
        try:
            run(p, "fp64")
            break
        except hweno.HwenoError as e:
            if e.status != hweno.ENONPHYSICAL or len(rejected) >= 8:
                raise
            rejected.append(seed)
            seed += 1000
    for prec in ("fp32",):
        try:
            run(p, prec)
        except hweno.HwenoError as e:
            out[prec] = {"failed": str(e), "t_reached": reached.get(prec)}
            continue
        out[prec]["rel_l1_to_fp64"] = float(np.abs(finals[prec] - finals["fp64"]).sum()
                                            / np.abs(finals["fp64"]).sum())
    return {"four_quadrant_2048_to_t0.25": {"workload": "2d_euler_four_quadrant_2048x2048_to_t0.25", "seed": seed,
                                            "rejected_seeds": rejected, "unit": UNIT, **out}}


def run_learned(torch, hweno, args, world, rank):
    """The learned-indicator form on its own workload: 2D Euler blast data
    (8 seeded circles, p in U[5,100] inside, 0.1 outside, rho = 1, at rest),
    4096^2, FP64, CFL 0.6, against the plain KXRCF scheme on the same data and
    the same dt sequence.  Reports both throughputs, the network pass's tensor
    roofline, and the judge: recall / false-negative / false-positive rates of
    the learned decisions against KXRCF on identical stage inputs, the share of
    cell decisions the network took, the troubled re-reconstruction work, and
    the relative L1 drift of the final state from the plain scheme's."""
    from paper_2201_12193_gb300 import learn, workloads as W
    n = args.learned_n
    t0 = time.time()
    p = W.blast_2d(n, seed=rank, ncircles=8)
    gen_s = time.time() - t0
    params = learn.load_params()
    cells = p.nx * p.ny
    steps, warm = args.steps, args.warmup
    res = {}
    dts = []
    finals = {}
    for mode in ("kxrcf", "mlp"):
        s = hweno.Solver.from_problem(p, indicator=mode)
        if mode == "mlp":
            s.set_mlp(params, 0.9)
        s.set_positivity_check(False)          # the scheme's transient p < 0 averages carry on
        s.set_stream(torch.cuda.current_stream())
        s.set_moments(torch.from_numpy(p.m).cuda())
        for k in range(warm):
            dt = s.max_dt(CFL)
            if mode == "kxrcf":
                dts.append(dt)
            s.step(dts[k])
        s.sync()
        s.rerecon_count()
        if mode == "mlp":
            s.mlp_fallbacks()
        s.profile(True)
        barrier(world)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for k in range(warm, warm + steps):
            dt = s.max_dt(CFL)                 # the same reduction in both runs
            if mode == "kxrcf":
                dts.append(dt)
            s.step(dts[k])                      # the plain run's dt sequence in both
        e1.record()
        torch.cuda.synchronize()
        ms = max_over_ranks(e0.elapsed_time(e1), world)
        prof = s.profile_read()
        s.profile(False)
        rer = s.rerecon_count()
        fb = s.mlp_fallbacks() if mode == "mlp" else None
        out = torch.empty(s.shape, dtype=torch.float64, device="cuda")
        s.get_moments(out)
        finals[mode] = out
        res[mode] = {"value": aggregate(cells, 3, steps, world, ms), "ms_per_step": ms / steps,
                     "rerecon_cells_per_stage": rer / (3 * steps), "prof": prof, "fallbacks": fb}
        s.close()
    a, b = finals["mlp"], finals["kxrcf"]
    drift = float((a - b).abs().sum() / b.abs().sum())
    del finals, a, b
    # judge on identical stage inputs: the initial state and the final plain state
    judge = {"tp": 0, "fp": 0, "fn": 0, "tn": 0}
    kx = hweno.Solver.from_problem(p)
    ml = hweno.Solver.from_problem(p, indicator="mlp")
    ml.set_mlp(params, 0.9)
    U = torch.from_numpy(p.m).cuda()
    Um, L = torch.empty_like(U), torch.empty_like(U)
    mk = torch.empty((p.ny, p.nx), dtype=torch.uint8, device="cuda")
    mm = torch.empty_like(mk)
    kx.set_positivity_check(False)
    kx.set_moments(U)
    for k, dt in enumerate(dts):
        if k in (0, len(dts) // 2, len(dts) - 1):
            kx.get_moments(U)
            kx.rhs(U, Um, L, mk)
            ml.rhs(U, Um, L, mm)
            x, y = mm.bool(), mk.bool()
            judge["tp"] += int((x & y).sum()); judge["fp"] += int((x & ~y).sum())
            judge["fn"] += int((~x & y).sum()); judge["tn"] += int((~x & ~y).sum())
        kx.step(dt)
    kx.close()
    ml.close()
    del U, Um, L
    torch.cuda.empty_cache()
    pos = max(judge["tp"] + judge["fn"], 1)
    lp = res["mlp"]["prof"]
    net_ms, net_n = lp["learned_indicator"]
    tot = sum(v[0] for v in lp.values())
    pk = _peaks()
    peak = pk.get("bf16_tflops_sustained")
    achieved = MLP_FLOP_PER_CELL * cells * net_n / (net_ms * 1e-3) / 1e12 if net_n else None
    roof = {"bound": "tensor", "kernel": "mlpre2d (features + 108-64-64-1 BF16 mma.sync, FP32 accumulate)",
            "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": (achieved / peak) if (achieved and peak) else None,
            "peak_source": "MEASURED_PEAKS bf16_tflops_sustained (of measured)" if peak else None,
            "avg_ms": net_ms / max(net_n, 1), "launches": net_n, "share": net_ms / tot if tot else None,
            "flop_per_cell": MLP_FLOP_PER_CELL}
    return {"learned_fp64": {
        "workload": f"2d_euler_blast_{n}x{n}", "value": res["mlp"]["value"], "ms_per_step": res["mlp"]["ms_per_step"],
        "plain_kxrcf_value": res["kxrcf"]["value"], "plain_kxrcf_ms_per_step": res["kxrcf"]["ms_per_step"],
        "speedup_vs_plain": res["kxrcf"]["ms_per_step"] / res["mlp"]["ms_per_step"], "steps": steps, "warmup": warm,
        "dtype": "f64 (network bf16 in, f32 accumulate)", "conf": 0.9,
        "recall": judge["tp"] / pos, "false_negative_rate": judge["fn"] / pos,
        "false_positive_rate": judge["fp"] / max(judge["fp"] + judge["tn"], 1),
        "decided_by_network": 1.0 - res["mlp"]["fallbacks"] / (cells * 3 * steps),
        "rerecon_cells_per_stage": {"mlp": res["mlp"]["rerecon_cells_per_stage"],
                                    "kxrcf": res["kxrcf"]["rerecon_cells_per_stage"]},
        "rel_l1_drift_vs_kxrcf": drift, "steps_compared": warm + steps,
        "kernels_ms": {"mlp": {k: v[0] for k, v in lp.items()},
                       "kxrcf": {k: v[0] for k, v in res["kxrcf"]["prof"].items()}},
        "roofline_network": roof, "input_generation_s": gen_s}}


def run_fused_forms(torch, hweno, args, p, world, out64, peaks, hbm_gbps, hbm_src):
    """The fused stage kernel (one launch per Runge-Kutta stage, point values in
    shared memory) on the headline workload in FP32 bulk, double-float and
    FP64: throughput, the HBM roofline of its algorithmic bytes, the ALU rate
    of the reconstruction it performs once per cell (the recomputed halo not
    counted), and the relative L1 distance of its state to the FP64 pipeline's
    after the same steps."""
    cells = p.nx * p.ny
    b = out64.cpu().numpy()
    out = {}
    for prec in ("fp32", "df64", "fp64"):
        s, ms, prof, _, o = run_solver(torch, hweno, p, prec, args.steps, args.warmup, world, profile=True,
                                       fused=True)
        ms = max_over_ranks(ms, world)
        a = o.cpu().numpy()
        fz_ms, fz_n = prof["fused_stage"]
        gbs = ALGO_BYTES_PER_CELL_STAGE * cells * fz_n / (fz_ms * 1e-3) / 1e9
        flops = _rec_flop_per_cell(4) * cells * fz_n / (fz_ms * 1e-3)
        pk = peaks["fp32_tflops"] if prec == "fp32" else peaks["fp64_tflops"]
        out[f"fused_{prec}"] = {
            "value": aggregate(cells, 3, args.steps, world, ms), "ms_per_step": ms / args.steps,
            "launches_per_step": fz_n / args.steps,
            "dtype": {"fp32": "f32 (state and RK accumulation f64)", "df64": "f32x2 double-float",
                      "fp64": "f64"}[prec],
            "rel_l1_vs_fp64_pipeline_after_steps": float(np.abs(a - b).sum() / np.abs(b).sum()),
            "steps_compared": args.warmup + args.steps,
            "roofline_hbm": {"bound": "hbm", "achieved": gbs, "peak": hbm_gbps, "unit": "GB/s",
                             "frac": gbs / hbm_gbps, "peak_source": hbm_src,
                             "bytes_per_cell_stage": ALGO_BYTES_PER_CELL_STAGE,
                             "traffic": (traffic_per_cell(f"fused2d_{prec}") or 0) * cells or None},
            "roofline_alu": {"bound": "alu", "achieved": flops / 1e12, "peak": pk, "unit": "TFLOP/s",
                             "frac": flops / 1e12 / pk,
                             "note": "reconstruction flop per cell once (FP64-equivalent count for double-float) "
                                     "against the measured FMA rate of the precision that executes it"}}
        s.close()
    return out


def run_double_mach(torch, hweno):
    """Example 3.9 (double Mach reflection) at the paper's 1600 x 400 to
    t = 0.2, FP64, KXRCF, CFL 0.6, device-driven: with the modified first
    moments used inside L only, and written back into the state (where the
    run stops at a p < 0 cell average next to the start of the wall)."""
    import math
    from paper_2201_12193_gb300 import workloads as W
    p = W.double_mach_2d(400)
    out = {}
    for name, persist in (("L_only", False), ("persist", True)):
        s = hweno.Solver.from_problem(p)
        s.set_persistence(persist)
        s.set_stream(torch.cuda.current_stream())
        s.set_moments(torch.from_numpy(p.m).cuda())
        t0 = time.perf_counter()
        reached, steps, err = 0.0, 0, None
        while reached < p.t_end - 1e-14:
            try:
                t, n = s.advance(min(0.01, p.t_end - reached), CFL)
            except hweno.HwenoError as e:
                err = str(e)[:160]
                break
            reached += t
            steps += n
        secs = time.perf_counter() - t0
        r = {"t_reached": reached, "steps": steps, "seconds": secs, "failed": err,
             "value": p.nx * p.ny * 3 * steps / secs if secs else None}
        if err is None:
            m = s.get_moments()
            rho = m[0, 0]
            pr = 0.4 * (m[3, 0] - 0.5 * (m[1, 0] ** 2 + m[2, 0] ** 2) / rho)
            xc = (np.arange(p.nx) + 0.5) * p.dx
            xs = 1.0 / 6.0 + (1.0 + 20.0 * p.t_end) / math.sqrt(3.0)
            r.update({"min_rho": float(rho.min()), "min_p": float(pr.min()), "max_rho": float(rho.max()),
                      "top_row_shock_x": float(xc[np.argmax(rho[-1] < 0.5 * (8.0 + 1.4))]), "exact_trace_x": xs,
                      "troubled_fraction_last_stage": float(s.troubled_mask()[-1].mean())})
        out[name] = r
        s.close()
    return {"double_mach_1600x400_to_t0.2": {"workload": "2d_euler_double_mach_reflection_1600x400", "unit": UNIT,
                                             **out}}


def run_forward_step(torch, hweno):
    """Example 3.10 (Mach 3 flow over a forward-facing step) at the paper's
    600 x 200, FP64, KXRCF, CFL 0.6, host-driven steps with the positivity
    check on, until t = 4 or the first refused step (the component-wise
    reconstruction does not pass the step's corner: the run stops about
    twenty steps in): steps, time reached, the refusal, throughput over the
    steps taken and extreme values of the fluid cells."""
    from paper_2201_12193_gb300 import workloads as W
    p = W.forward_step_2d(200)
    s = hweno.Solver.from_problem(p)
    s.set_stream(torch.cuda.current_stream())
    s.set_moments(torch.from_numpy(p.m).cuda())
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    t, n, err = 0.0, 0, None
    try:
        while t < p.t_end and n < 100000:
            dt = min(s.max_dt(CFL), p.t_end - t)
            s.step(dt)
            t += dt
            n += 1
    except hweno.HwenoError as e:
        err = str(e)[:160]
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    m = s.get_moments()
    i0, j1 = p.meta["solid"]
    fluid = np.ones((p.ny, p.nx), bool)
    fluid[:j1, i0:] = False
    rho = m[0, 0]
    pr = 0.4 * (m[3, 0] - 0.5 * (m[1, 0] ** 2 + m[2, 0] ** 2) / rho)
    jp, ip = np.unravel_index(np.argmin(np.where(fluid, pr, np.inf)), pr.shape)
    out = {"workload": "2d_euler_forward_step_600x200", "t_end": p.t_end, "t_reached": t, "steps": n,
           "refused": err, "seconds": secs, "unit": UNIT,
           "value": int(fluid.sum()) * 3 * n / secs if n else None,
           "min_rho": float(rho[fluid].min()), "max_rho": float(rho[fluid].max()), "min_p": float(pr[fluid].min()),
           "min_p_cell": [int(ip), int(jp)], "corner_cell": [int(i0), int(j1)]}
    s.close()
    return {"forward_step_600x200": out}


def run_decomposed(args, world, rank, local):
    """N > 1: the headline problem split into N row slabs, one per rank, with the
    4-row halo exchange before every stage over NCCL and the CFL wave speeds
    max-reduced (decomp.DistSlab); strong scaling of the same 2048^2 grid."""
    import torch

    from paper_2201_12193_gb300 import build, decomp, hweno, workloads as W
    torch.cuda.set_device(local)
    build.build()
    p = W.four_quadrant_2d(args.n, seed=0)
    d = decomp.DistSlab(p, rank, world)
    lay = d.lay
    rows = np.arange(lay["r0"] - lay["lo"], lay["r1"] + lay["hi"]) % p.ny
    local_m = np.ascontiguousarray(p.m[:, :, rows, :])
    d.set_moments(torch.from_numpy(local_m).cuda())
    for _ in range(args.warmup):
        d.step(d.max_dt(CFL))
    d.solver.sync()
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    smi_index = vis.split(",")[local] if vis and vis.split(",")[local].strip().isdigit() else local
    clocks = ClockSampler(smi_index)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        d.step(d.max_dt(CFL))
    e1.record()
    torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1), world)
    clk = clocks.stop()
    cells = p.nx * p.ny
    value = cells * 3 * args.steps / (ms * 1e-3)
    # end to end: each rank's slab from pinned host memory, the step, the owned rows back
    host = torch.from_numpy(local_m.copy()).pin_memory()
    res = torch.empty_like(host).pin_memory()
    k = max(2, min(args.steps, 4))
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(k):
        d.solver.set_moments(host.numpy())
        d.step(d.max_dt(CFL))
        d.solver.get_moments(res.numpy())
    t = max_over_ranks(time.perf_counter() - t0, world)
    d.close()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "strong", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": WORKLOAD, "nx": p.nx, "ny": p.ny, "precision": "fp64", "indicator": "kxrcf",
                           "cfl": CFL, "parallelism": f"row slabs x{world} (4-row halo exchange per stage, NCCL)",
                           "l2": "inputs larger than L2"},
                "roofline": None, "e2e": {"value": cells * 3 * k / t, "unit": UNIT, "steps": k,
                                          "h2d_bytes_per_step": int(host.numel() * 8),
                                          "d2h_bytes_per_step": int(res.numel() * 8)},
                "gpu_launches": None, "clocks": clk}
        print(json.dumps(line))


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

    peaks = alu_peaks(hweno)                    # before the timed region, not inside it
    hbm_gbps, hbm_src = hbm_peak()
    s64, ms, prof, clk, out64 = run_solver(torch, hweno, p, args.precision, args.steps, args.warmup, world,
                                           profile=True, clocks=clocks)
    ms = max_over_ranks(ms, world)
    value = aggregate(cells, 3, args.steps, world, ms)
    ms_step = ms / args.steps

    # roofline of the dominant kernel (largest share of device time)
    kind, (kms, kn) = max(prof.items(), key=lambda kv: kv[1][0])
    total_kernel_ms = sum(v[0] for v in prof.values())
    flop = _rec_flop_per_cell(s64.nvar) * cells * kn if kind == "reconstruct" else None
    roof = None
    if flop:
        achieved = flop / (kms * 1e-3)
        pk = peaks["fp64_tflops"] * 1e12 if args.precision == "fp64" else peaks["fp32_tflops"] * 1e12
        roof = {"bound": "alu", "kernel": f"rec2d<{'double' if args.precision == 'fp64' else 'float'},4> ({kind})",
                "achieved": achieved / 1e12, "peak": pk / 1e12, "unit": "TFLOP/s", "frac": achieved / pk,
                "peak_source": f"{args.precision.upper()} FMA throughput measured in this run by hweno_alu_probe "
                               f"(of measured); nominal FP64 from unit counts {peaks['fp64_nominal_tflops']:.3f}",
                "frac_of_nominal_fp64": achieved / (peaks["fp64_nominal_tflops"] * 1e12),
                "flop_per_cell": _rec_flop_per_cell(s64.nvar), "traffic": None, "launches": kn, "avg_ms": kms / kn,
                "share": kms / total_kernel_ms}
        bpc = traffic_per_cell(f"rec2d_{args.precision}") if args.precision == "fp64" else None
        if bpc:
            roof["traffic"] = bpc * cells
            roof["traffic_unit"] = "bytes per launch (ncu dram read+write per cell x cells, profiles/dram_traffic.json)"
    kernels = {k: {"ms": v[0], "launches": v[1], "share": v[0] / total_kernel_ms} for k, v in prof.items()}
    hbm = {"algorithmic_GBps": ALGO_BYTES_PER_CELL_STAGE * cells * 3 * args.steps / (ms * 1e-3) / 1e9,
           "peak_GBps": hbm_gbps, "peak_source": hbm_src}
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
        forms["fp32bulk"] = {"value": aggregate(cells, 3, args.steps, world, ms32), "ms_per_step": ms32 / args.steps,
                             "dtype": "f32 (state and RK accumulation f64)",
                             "rel_l1_vs_fp64_after_steps": float(np.abs(a - b).sum() / np.abs(b).sum()),
                             "steps_compared": args.warmup + args.steps,
                             "kernels": {k: {"ms": v[0], "launches": v[1]} for k, v in prof32.items()}}
        rk_ms, rk_n = prof32["reconstruct"]
        up_ms, up_n = prof32["update"]
        if rk_n:
            ach = _rec_flop_per_cell(4) * cells * rk_n / (rk_ms * 1e-3) / 1e12
            t = traffic_per_cell("rec2d_fp32")
            forms["fp32bulk"]["roofline_reconstruct"] = {
                "bound": "alu", "achieved": ach, "peak": peaks["fp32_tflops"], "unit": "TFLOP/s",
                "frac": ach / peaks["fp32_tflops"], "peak_source": "FP32 FMA throughput measured in this run (of measured)",
                "flop_per_cell": _rec_flop_per_cell(4), "avg_ms": rk_ms / rk_n,
                "traffic": t * cells if t else None}
        if up_n:
            gbs = UPD32_BYTES_PER_CELL * cells * up_n / (up_ms * 1e-3) / 1e9
            t = traffic_per_cell("update2d_fp32")
            forms["fp32bulk"]["roofline_update"] = {
                "bound": "hbm", "achieved": gbs, "peak": hbm_gbps, "unit": "GB/s", "frac": gbs / hbm_gbps,
                "peak_source": hbm_src, "bytes_per_cell": UPD32_BYTES_PER_CELL, "avg_ms": up_ms / up_n,
                "traffic": t * cells if t else None}
        s32.close()
        sx, msx, profx, _, outx = run_solver(torch, hweno, p, "df64", args.steps, args.warmup, world, profile=True)
        msx = max_over_ranks(msx, world)
        a = outx.cpu().numpy()
        forms["df64"] = {"value": aggregate(cells, 3, args.steps, world, msx), "ms_per_step": msx / args.steps,
                         "dtype": "f32x2 double-float (48-bit significand; state and RK accumulation f64)",
                         "rel_l1_vs_fp64_after_steps": float(np.abs(a - b).sum() / np.abs(b).sum()),
                         "steps_compared": args.warmup + args.steps,
                         "kernels": {k: {"ms": v[0], "launches": v[1]} for k, v in profx.items()}}
        kx, (kxms, kxn) = "reconstruct", profx["reconstruct"]
        if kxn:
            ach = _rec_flop_per_cell(4) * cells * kxn / (kxms * 1e-3)
            forms["df64"]["roofline_reconstruct"] = {
                "bound": "alu", "achieved_fp64_equiv_tflops": ach / 1e12,
                "note": "algorithmic FP64-equivalent flop of the reconstruction per second; the FP32 pipe "
                        "executes ~6-15 FP32 instructions per double-float operation"}
        sx.close()

    if not args.no_forms and not args.no_fused:
        forms.update(run_fused_forms(torch, hweno, args, p, world, out64, peaks, hbm_gbps, hbm_src))

    if not args.no_forms and not args.no_1d:
        forms.update(run_shu_osher(torch, hweno, world))
        forms.update(run_shu_osher_long(torch, hweno, world, hbm_gbps, hbm_src))
    if args.full_run:
        forms.update(run_four_quadrant_full(torch, hweno, world, rank))
    if args.dmr:
        forms.update(run_double_mach(torch, hweno))
    if args.step:
        forms.update(run_forward_step(torch, hweno))

    if not args.no_forms and not args.no_batch:
        forms.update(run_batched(torch, hweno, args, world, rank))

    if not args.no_forms and not args.no_learned:
        forms.update(run_learned(torch, hweno, args, world, rank))

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
        try:
            va, cores, slow = time_oracle_all_cores(p.nx, 64)
            cpu["all_cores"] = {"value": va, "unit": UNIT, "cores": cores, "seconds": slow,
                                "sample": f"{cores} processes, each one SSP-RK3 step of a 128x128 centre window"}
        except Exception as e:     # the single-core figure stands on its own
            cpu["all_cores"] = {"unavailable": str(e)[:200]}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "strong",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": WORKLOAD, "nx": p.nx, "ny": p.ny, "precision": "fp64", "indicator": "kxrcf",
                           "cfl": CFL, "seed_per_rank": "rank",
                           "parallelism": "one GPU (N > 1 splits this grid into row slabs: strong scaling)",
                           "l2": "inputs larger than L2 (state 403 MB, point values 2.1 GB per stage)"},
                "roofline": roof, "hbm": hbm, "alu_peaks": peaks, "kernels": kernels, "forms": forms, "e2e": e2e,
                "cpu_baseline": cpu, "gpu_launches": launches * 1, "clocks": clk}
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
    if args.impl == "reference":
        # the oracle arm runs on rank 0 alone; other ranks exit without work
        # (and without a process group: the arm has no collective)
        run_reference(args, int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")))
        return
    world, rank, local = dist_init()
    if world > 1:
        run_decomposed(args, world, rank, local)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
