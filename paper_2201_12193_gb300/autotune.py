"""Tile-shape autotuner for batched steps (hweno_batch_set_tile).

Times each update-tile variant (32x4, 16x8, 64x2) on a throw-away copy of the
batch and caches the fastest per batch signature (precision, device, histogram
of grid sizes) in a JSON file ($HWENO_TUNE_CACHE, default
~/.cache/hweno/tune.json).  Results do not depend on the variant: only speed.
"""
from __future__ import annotations

import collections
import json
import os

VARIANTS = {0: "32x4", 1: "16x8", 2: "64x2"}


def cache_path():
    return os.environ.get("HWENO_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "hweno", "tune.json"))


def signature(problems, precision):
    import torch
    hist = collections.Counter((p.nx, p.ny) for p in problems)
    sizes = ",".join(f"{nx}x{ny}:{c}" for (nx, ny), c in sorted(hist.items()))
    return f"{torch.cuda.get_device_name()}|{precision}|{sizes}"


def _load():
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def tune_batch(problems, precision="fp32", steps=2, use_cache=True):
    """Fastest tile variant for this batch; returns (variant, {variant: ms per step})."""
    import torch

    from .hweno import BatchSolver
    key = signature(problems, precision)
    cache = _load()
    if use_cache and key in cache:
        return int(cache[key]["variant"]), cache[key]["ms"]
    s = BatchSolver(problems, precision=precision)
    s.set_positivity_check(False)      # timing only: a transient non-physical average does not matter
    init = [torch.from_numpy(p.m).cuda() for p in problems]
    times = {}
    for v in VARIANTS:
        for k, m in enumerate(init):   # every variant from the same initial state, 1 + steps steps
            s.set_moments(k, m)
        s.set_tile(v)
        s.step()
        s.sync()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            s.step()
        e1.record()
        torch.cuda.synchronize()
        times[v] = e0.elapsed_time(e1) / steps
    s.sync()
    s.close()
    best = min(times, key=times.get)
    cache[key] = {"variant": best, "tile": VARIANTS[best], "ms": {str(k): v for k, v in times.items()}}
    try:
        os.makedirs(os.path.dirname(cache_path()), exist_ok=True)
        with open(cache_path(), "w") as f:
            json.dump(cache, f, indent=1)
    except OSError:
        pass
    return best, times
