"""Row-slab decomposition across ranks on the CPU (gloo, world size 2): each
rank advances its slab of one 2D Euler problem with the oracle, the 4-row
halos travel through decomp.exchange_rows and the CFL wave speeds through an
all-reduce (the same partition, halo and transport code the GPU ranks use),
and the gathered result must equal the oracle run on the whole grid bit for
bit.

The slab's stage is the oracle's right-hand side combined in the oracle's
own Runge-Kutta arithmetic (eq. (Runge-Kutta), the modified first moments
written back as the oracle's default reading does), so any difference comes
from the decomposition: a halo row taken from the wrong neighbour, the wrong
rows, a missed wrap on a periodic side or a dt formed from one slab's speeds.
"""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2201_12193_gb300 import decomp, workloads as W  # noqa: E402

NSTEPS = 3


def _problem(kind):
    if kind == "four_quadrant":
        return W.four_quadrant_2d(32, seed=3, ny=26)
    p = W.vortex_2d(24, seed=2)                  # periodic in y: both slabs wrap
    return p


def _cfg(orc, q, p):
    return orc.make_cfg(2, q.nx, q.ny, dx=p.dx, dy=p.dy, eq="euler", bc=q.bc)


def _slab_step(orc, cfg, U, dt, exchange):
    """One SSP-RK3 step of a slab in the oracle's arithmetic, halos refreshed
    before every stage."""
    U = exchange(U)
    M0, L0, _, _, rc = orc.rhs(cfg, U)
    assert rc == 0
    Un = M0
    U1 = Un + dt * L0
    U1 = exchange(U1)
    M1, L1, _, _, rc = orc.rhs(cfg, U1)
    assert rc == 0
    U2 = 0.75 * Un + 0.25 * M1 + 0.25 * dt * L1
    U2 = exchange(U2)
    M2, L2, _, _, rc = orc.rhs(cfg, U2)
    assert rc == 0
    return Un / 3.0 + 2.0 / 3.0 * M2 + 2.0 / 3.0 * dt * L2


def _worker(rank, world, port, kind, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle as orc

        p = _problem(kind)
        periodic = p.bc[2] == "periodic"
        lay = decomp.slab_layout(p.ny, world, periodic)[rank]
        q = decomp.sub_problem(p, lay)
        cfg = _cfg(orc, q, p)
        own = lay["r1"] - lay["r0"]
        lo, hi = lay["lo"], lay["hi"]
        H = decomp.HALO

        def exchange(U):
            U = U.copy()
            s_lo = torch.from_numpy(np.ascontiguousarray(U[:, :, lo:lo + H, :])) if lo else None
            s_hi = torch.from_numpy(np.ascontiguousarray(U[:, :, lo + own - H:lo + own, :])) if hi else None
            r_lo = torch.empty((4, 3, H, p.nx), dtype=torch.float64) if lo else None
            r_hi = torch.empty((4, 3, H, p.nx), dtype=torch.float64) if hi else None
            decomp.exchange_rows(s_lo, s_hi, r_lo, r_hi, rank, world, periodic)
            if lo:
                U[:, :, :lo, :] = r_lo.numpy()
            if hi:
                U[:, :, lo + own:, :] = r_hi.numpy()
            return U

        U = q.m.copy()
        for _ in range(NSTEPS):
            ax, ay = orc.wave_speeds(cfg, U, lo, lo + own)
            sp = torch.tensor([ax, ay], dtype=torch.float64)
            dist.all_reduce(sp, op=dist.ReduceOp.MAX)
            dt = decomp.dt_from_speeds(float(sp[0]), float(sp[1]), p.dx, p.dy, 0.6)
            U = _slab_step(orc, cfg, U, dt, exchange)
        mine = torch.from_numpy(np.ascontiguousarray(U[:, :, lo:lo + own, :]))
        sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
        dist.all_gather(sizes, torch.tensor([own]))
        parts = [torch.empty((4, 3, int(n), p.nx), dtype=torch.float64) for n in sizes]
        dist.all_gather(parts, mine)
        if rank == 0:
            out.put(np.concatenate([t.numpy() for t in parts], axis=2))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("kind", ["four_quadrant", "vortex_periodic"])
def test_two_rank_slabs_equal_the_whole_grid(orc, kind):
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, kind, out)) for r in range(2)]
    for pr in procs:
        pr.start()
    got = out.get(timeout=300)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    p = _problem(kind)
    cfg = orc.make_cfg(2, p.nx, p.ny, dx=p.dx, dy=p.dy, eq="euler", bc=p.bc)
    m = p.m
    for _ in range(NSTEPS):
        m, masks, rc = orc.step(cfg, m, orc.max_dt(cfg, m, 0.6))
        assert rc == 0
    assert masks.sum() > 0 or kind == "vortex_periodic"
    np.testing.assert_array_equal(got, m)


def test_partition_and_layout():
    assert decomp.partition(26, 2) == [(0, 13), (13, 26)]
    assert decomp.partition(13, 3) == [(0, 5), (5, 9), (9, 13)]
    with pytest.raises(ValueError):
        decomp.partition(7, 2)
    lay = decomp.slab_layout(26, 3, periodic_y=False)
    assert [(x["lo"], x["hi"]) for x in lay] == [(0, 4), (4, 4), (4, 0)]
    lay = decomp.slab_layout(26, 2, periodic_y=True)
    assert [(x["lo"], x["hi"]) for x in lay] == [(4, 4), (4, 4)]
    p = W.vortex_2d(24, seed=2)
    q = decomp.sub_problem(p, decomp.slab_layout(24, 2, True)[0])
    assert q.ny == 20 and q.bc[2:] == ("transmissive", "transmissive")
    np.testing.assert_array_equal(q.m[:, :, :4], p.m[:, :, 20:24])      # the wrapped halo
    np.testing.assert_array_equal(q.m[:, :, 4:16], p.m[:, :, 0:12])
