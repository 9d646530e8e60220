"""The multi-rank logic of bench.py on CPU: two gloo ranks (world size 2).

* dist_init / barrier / max_over_ranks over gloo: every rank gets the maximum.
* Weak scaling: each rank seeds its own problem (different moments per rank),
  and the whole-job value counts the cells of all ranks over the slowest time.
* The reference arm: rank 0 alone runs and prints; rank 1 exits 0 silently.
"""
from __future__ import annotations

import json
import os
import socket
import subprocess
import sys
import textwrap

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RANK_SCRIPT = textwrap.dedent("""
    import json, os, sys
    sys.path.insert(0, os.environ["HWENO_ROOT"])
    import numpy as np
    import bench
    from paper_2201_12193_gb300 import workloads as W
    world, rank, local = bench.dist_init()
    bench.barrier(world)
    mx = bench.max_over_ranks(10.0 + 5.0 * rank, world)
    p = W.four_quadrant_2d(16, seed=rank)
    out = {"rank": rank, "world": world, "max": mx, "checksum": float(np.abs(p.m).sum()),
           "value": bench.aggregate(p.nx * p.ny, 3, 4, world, mx)}
    bench.barrier(world)
    import torch.distributed as dist
    dist.destroy_process_group()
    print(json.dumps(out))
""")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _launch(script, extra_env, world=2, timeout=240):
    port = _free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, HWENO_ROOT=ROOT, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE=str(world),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), HWENO_BENCH_GLOO="1", CUDA_VISIBLE_DEVICES="",
                   **extra_env)
        procs.append(subprocess.Popen([sys.executable, "-c", script], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True, cwd=ROOT))
    outs = []
    for p in procs:
        try:
            o, e = p.communicate(timeout=timeout)
        except subprocess.TimeoutExpired:
            p.kill()
            o, e = p.communicate()
        outs.append((p.returncode, o, e))
    return outs


def test_two_gloo_ranks_max_and_weak_scaling():
    pytest.importorskip("torch")
    outs = _launch(RANK_SCRIPT, {})
    res = []
    for rc, o, e in outs:
        assert rc == 0, e[-2000:]
        res.append(json.loads(o.strip().splitlines()[-1]))
    assert {r["rank"] for r in res} == {0, 1} and all(r["world"] == 2 for r in res)
    assert all(r["max"] == 15.0 for r in res)                    # max over ranks, seen by every rank
    assert res[0]["checksum"] != res[1]["checksum"]              # each rank its own seeded problem
    cells = 16 * 16
    assert all(abs(r["value"] - cells * 3 * 4 * 2 / 15e-3) < 1e-6 * r["value"] for r in res)


def test_reference_arm_runs_on_rank_zero_only():
    port = _free_port()
    outs = []
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                                       "--warmup", "0", "--n", "160"], env=env, cwd=ROOT,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    for p in procs:
        o, e = p.communicate(timeout=600)
        outs.append((p.returncode, o, e))
    (rc0, o0, e0), (rc1, o1, e1) = outs
    assert rc0 == 0 and rc1 == 0, (e0[-2000:], e1[-2000:])
    assert o1.strip() == ""
    line = json.loads(o0.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"
