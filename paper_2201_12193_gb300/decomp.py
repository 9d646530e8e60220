"""Row-slab decomposition of one 2D problem, with a 4-row halo exchange before
every Runge-Kutta stage.

Why 4 rows: in one stage the update of a cell reads the point values of its
edge neighbours (fluxes), which for a troubled neighbour come from the
modified moments of that neighbour's 3 x 3 stencil (Step 2.3), whose flags
need the pass-1 point values one cell further out (KXRCF, eq. (KXRCF_)), which
need the moments one cell further still (Step 1): 1 + 1 + 1 + 1 = 4.  A slab
that holds the stage input of 4 rows beyond each internal side therefore
advances its own rows exactly as the whole grid does; its outer halo rows come
out wrong (they see an artificial side) and are overwritten by the next
exchange.  The CFL step takes the maxima of the wave speeds over all slabs,
so dt is the whole grid's to the last bit.

Two transports move the halo rows: `LocalSlabs` keeps every slab on one GPU and
copies rows device to device; `DistSlab` holds one slab per rank and exchanges
rows with torch.distributed point-to-point messages (NCCL between GPUs; the
same code runs over gloo on the CPU).  Arithmetic happens only in the CUDA
library (hweno_stage, hweno_copy_rows, hweno_wave_speeds).
"""
from __future__ import annotations

import copy
import math

import numpy as np

HALO = 4


def partition(ny: int, nslabs: int):
    """Owned row ranges [(r0, r1)] of nslabs balanced slabs (each >= HALO rows)."""
    if nslabs < 1 or ny < HALO * nslabs:
        raise ValueError(f"{ny} rows cannot give {nslabs} slabs of at least {HALO} rows")
    base, extra = divmod(ny, nslabs)
    out, r = [], 0
    for s in range(nslabs):
        n = base + (1 if s < extra else 0)
        out.append((r, r + n))
        r += n
    return out


def slab_layout(ny: int, nslabs: int, periodic_y: bool):
    """Per slab: owned rows (r0, r1) and halo rows below / above (lo, hi).  A
    physical side keeps its boundary (no halo); an internal or periodic side
    has HALO rows copied from the neighbour."""
    out = []
    for s, (r0, r1) in enumerate(partition(ny, nslabs)):
        lo = HALO if (s > 0 or (periodic_y and nslabs > 1)) else 0
        hi = HALO if (s < nslabs - 1 or (periodic_y and nslabs > 1)) else 0
        out.append({"slab": s, "r0": r0, "r1": r1, "lo": lo, "hi": hi})
    return out


def sub_problem(p, lay):
    """The slab's problem: its owned rows plus halos (periodic rows wrap), the
    y domain shifted accordingly, and transmissive y sides where the slab's
    edge is internal (those sides only touch halo rows)."""
    q = copy.copy(p)
    r0, r1, lo, hi = lay["r0"], lay["r1"], lay["lo"], lay["hi"]
    rows = np.arange(r0 - lo, r1 + hi) % p.ny
    q.m = np.ascontiguousarray(p.m[:, :, rows, :])
    q.ny = r1 - r0 + lo + hi
    q.y0 = p.y0 + (r0 - lo) * p.dy
    q.y1 = q.y0 + q.ny * p.dy
    bc = list(p.bc)
    if lo:
        bc[2] = "transmissive"
    if hi:
        bc[3] = "transmissive"
    q.bc = tuple(bc)
    q.fixed = None
    return q


def dt_from_speeds(ax: float, ay: float, dx: float, dy: float, cfl: float) -> float:
    """The 2D CFL rule of hweno_max_dt (same expressions): cfl / (ax/dx + ay/dy)."""
    if not (math.isfinite(ax) and math.isfinite(ay)):
        raise FloatingPointError("non-physical cell average: no CFL step length")
    r = ax / dx + ay / dy
    return cfl / r if r > 0.0 else math.inf


class LocalSlabs:
    """Every slab of one problem on the current GPU, halos copied device to device."""

    def __init__(self, p, nslabs, stream=None, **solver_kw):
        import torch

        from . import hweno

        if p.dim != 2 or p.fixed:
            raise ValueError("row slabs are defined for 2D problems without fixed-state sides")
        self.p = p
        self.periodic = p.bc[2] == "periodic"
        self.lay = slab_layout(p.ny, nslabs, self.periodic)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.solvers = []
        for lay in self.lay:
            q = sub_problem(p, lay)
            s = hweno.Solver.from_problem(q, **solver_kw)
            s.set_stream(self.stream)
            s.set_owned_rows(lay["lo"], lay["lo"] + lay["r1"] - lay["r0"])
            self.solvers.append(s)
        nvm = self.solvers[0].nvar * self.solvers[0].nmom
        self.buf = torch.empty(nvm * HALO * p.nx, dtype=torch.float64, device="cuda")

    def set_moments(self, m):
        import torch

        for lay, s in zip(self.lay, self.solvers):
            rows = np.arange(lay["r0"] - lay["lo"], lay["r1"] + lay["hi"]) % self.p.ny
            s.set_moments(torch.from_numpy(np.ascontiguousarray(np.asarray(m)[:, :, rows, :])).cuda())

    def _exchange(self):
        n = len(self.solvers)
        for k, (lay, s) in enumerate(zip(self.lay, self.solvers)):
            if lay["lo"]:          # my bottom halo <- the top owned rows of the slab below
                b = (k - 1) % n
                src, sl = self.solvers[b], self.lay[b]
                src.copy_rows(sl["lo"] + (sl["r1"] - sl["r0"]) - HALO, HALO, self.buf, False)
                s.copy_rows(0, HALO, self.buf, True)
            if lay["hi"]:          # my top halo <- the bottom owned rows of the slab above
                a = (k + 1) % n
                src, sl = self.solvers[a], self.lay[a]
                src.copy_rows(sl["lo"], HALO, self.buf, False)
                s.copy_rows(lay["lo"] + (lay["r1"] - lay["r0"]), HALO, self.buf, True)

    def max_dt(self, cfl=0.6):
        ax = ay = 0.0
        for s in self.solvers:
            a, b = s.wave_speeds()
            ax, ay = max(ax, a), max(ay, b)
        return dt_from_speeds(ax, ay, self.p.dx, self.p.dy, cfl)

    def step(self, dt):
        for k in range(3):
            self._exchange()
            for s in self.solvers:
                s.stage(k, dt)

    def gather(self):
        out = np.empty(self.p.m.shape)
        for lay, s in zip(self.lay, self.solvers):
            m = s.get_moments()
            out[:, :, lay["r0"]:lay["r1"], :] = m[:, :, lay["lo"]:lay["lo"] + lay["r1"] - lay["r0"], :]
        return out

    def troubled_masks(self):
        out = np.empty((3, self.p.ny, self.p.nx), np.uint8)
        for lay, s in zip(self.lay, self.solvers):
            mk = s.troubled_mask()
            out[:, lay["r0"]:lay["r1"]] = mk[:, lay["lo"]:lay["lo"] + lay["r1"] - lay["r0"]]
        return out

    def close(self):
        for s in self.solvers:
            s.close()


def exchange_rows(send_lo, send_hi, recv_lo, recv_hi, rank, world, periodic):
    """Halo rows between neighbouring ranks (torch.distributed point to point).
    send_lo: my bottom owned rows (to the rank below), send_hi: my top owned
    rows (to the rank above); recv_lo / recv_hi receive the halos below /
    above.  Tensors may be None where a side is physical.  Tag 0 travels up,
    tag 1 down, so two ranks that are each other's neighbour on both sides
    (periodic, world 2) keep the messages apart."""
    import torch.distributed as dist

    below = rank - 1 if rank > 0 else (world - 1 if periodic else None)
    above = rank + 1 if rank < world - 1 else (0 if periodic else None)
    ops = []
    if above is not None and send_hi is not None:
        ops.append(dist.isend(send_hi, above, tag=0))
    if below is not None and send_lo is not None:
        ops.append(dist.isend(send_lo, below, tag=1))
    if below is not None and recv_lo is not None:
        ops.append(dist.irecv(recv_lo, below, tag=0))
    if above is not None and recv_hi is not None:
        ops.append(dist.irecv(recv_hi, above, tag=1))
    for op in ops:
        op.wait()


class DistSlab:
    """One slab per rank (torch.distributed initialised, one GPU per rank)."""

    def __init__(self, p, rank, world, stream=None, **solver_kw):
        import torch

        from . import hweno

        self.p, self.rank, self.world = p, rank, world
        self.periodic = p.bc[2] == "periodic"
        self.lay = slab_layout(p.ny, world, self.periodic)[rank]
        q = sub_problem(p, self.lay)
        self.own = self.lay["r1"] - self.lay["r0"]
        self.solver = hweno.Solver.from_problem(q, **solver_kw)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.solver.set_stream(self.stream)
        self.solver.set_owned_rows(self.lay["lo"], self.lay["lo"] + self.own)
        n = self.solver.nvar * self.solver.nmom * HALO * p.nx
        self.bufs = [torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(4)]

    def set_moments(self, m_local):
        self.solver.set_moments(m_local)

    def _exchange(self):
        import torch

        lo, hi = self.lay["lo"], self.lay["hi"]
        s_lo, s_hi, r_lo, r_hi = self.bufs
        if lo:
            self.solver.copy_rows(lo, HALO, s_lo, False)
        if hi:
            self.solver.copy_rows(lo + self.own - HALO, HALO, s_hi, False)
        torch.cuda.current_stream().synchronize()
        exchange_rows(s_lo if lo else None, s_hi if hi else None, r_lo if lo else None, r_hi if hi else None,
                      self.rank, self.world, self.periodic)
        if lo:
            self.solver.copy_rows(0, HALO, r_lo, True)
        if hi:
            self.solver.copy_rows(lo + self.own, HALO, r_hi, True)

    def max_dt(self, cfl=0.6):
        import torch
        import torch.distributed as dist

        sp = torch.tensor(self.solver.wave_speeds(), dtype=torch.float64, device="cuda")
        dist.all_reduce(sp, op=dist.ReduceOp.MAX)
        ax, ay = sp.tolist()
        return dt_from_speeds(ax, ay, self.p.dx, self.p.dy, cfl)

    def step(self, dt):
        for k in range(3):
            self._exchange()
            self.solver.stage(k, dt)

    def owned_moments(self):
        m = self.solver.get_moments()
        return m[:, :, self.lay["lo"]:self.lay["lo"] + self.own, :]

    def close(self):
        self.solver.close()
