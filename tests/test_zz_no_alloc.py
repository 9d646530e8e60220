"""hweno_max_dt_noalloc, the CFL reduction that allocates nothing, against the
handle-based hweno_max_dt.

The allocation-free entry point serves callers that cannot call cudaMalloc
(a frozen memory budget, no room for the implicit synchronisation of an
allocation, no handle to keep).  Its partial maxima live in a static device
array shared by every call, so each case makes two calls in a row (the largest
grid the array accepts, then the case's own grid) and checks both against the
existing entry point.  This file is collected last on purpose.
"""
from __future__ import annotations

import contextlib
import ctypes
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2201_12193_gb300 import hweno, workloads as W  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_12193_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _grid(p):
    g = hweno.Grid()
    g.dim, g.nx, g.ny = p.dim, p.nx, p.ny
    g.x0, g.x1, g.y0, g.y1 = p.x0, p.x1, p.y0, p.y1
    g.eq = hweno.EQ[p.eq]
    g.adv_a, g.adv_b = p.adv
    return g


def _handle_dt(p, cfl):
    s = hweno.Solver.from_problem(p)
    s.set_moments(p.m)
    dt = s.max_dt(cfl)
    s.close()
    return dt


CASES = [
    ("euler_2d", lambda: W.four_quadrant_2d(96, seed=7, ny=80)),
    ("euler_1d", lambda: W.shu_osher_1d(300)),
    ("advection_1d", lambda: W.advection_sin_1d(200)),
    ("burgers_1d", lambda: W.burgers_1d(160)),
    ("advection_2d", lambda: W.advection_2d(36)),
    ("burgers_2d", lambda: W.burgers_2d(40)),
]


@pytest.fixture(scope="module")
def largest():
    """The largest grid the scratch array takes, and its dt from the handle."""
    p = W.four_quadrant_2d(2048, seed=7)
    return p, _handle_dt(p, 0.6)


@pytest.mark.parametrize("side_stream", [False, True], ids=["current_stream", "side_stream"])
@pytest.mark.parametrize("name,make", CASES, ids=[n for n, _ in CASES])
def test_no_alloc_matches_handle_dt_on_two_calls(largest, name, make, side_stream):
    cfl = 0.6
    small = make()
    problems = [largest[0], small]
    want = [largest[1], _handle_dt(small, cfl)]
    stream = torch.cuda.Stream() if side_stream else None
    out = torch.full((3,), -1.0, dtype=torch.float64, device="cuda")
    for p, w in zip(problems, want):
        with torch.cuda.stream(stream) if stream is not None else contextlib.nullcontext():
            m = torch.from_numpy(p.m).cuda()
            hweno.max_dt_noalloc(_grid(p), p.gamma, m, cfl, out, stream=stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got)) and got[0] > 0.0
        assert math.isclose(got[2], w, rel_tol=1e-13), (got, w)


def test_no_alloc_gives_zero_dt_for_a_non_physical_average():
    """A cell average with p < 0 gives dt = 0 (the entry point always applies the
    positivity rule), after a call on a physical state that left its partials."""
    p = W.four_quadrant_2d(64, seed=1)
    out = torch.full((3,), -1.0, dtype=torch.float64, device="cuda")
    hweno.max_dt_noalloc(_grid(p), p.gamma, torch.from_numpy(p.m).cuda(), 0.6, out)
    torch.cuda.synchronize()
    assert out[2].item() > 0.0
    m = p.m.copy()
    rho, mu = m[0, 0, 10, 20], m[1, 0, 10, 20] / m[0, 0, 10, 20]
    m[3, 0, 10, 20] = 0.5 * rho * mu * mu - 0.1       # p = 0.4 * (E - kinetic) < 0
    hweno.max_dt_noalloc(_grid(p), p.gamma, torch.from_numpy(m).cuda(), 0.6, out)
    torch.cuda.synchronize()
    assert out[2].item() == 0.0


def test_no_alloc_rejects_grids_beyond_its_scratch():
    """The C entry point rejects the grid before it reads the state, so a small
    buffer is enough; the binding's own size check fires first for an
    undersized tensor."""
    p = W.four_quadrant_2d(64, seed=1)
    g = _grid(p)
    g.nx, g.ny, g.x1, g.y1 = 2050, 2048, 2050 / 2048, 1.0       # 4,198,400 > 4,194,304 cells
    m = torch.zeros(16, dtype=torch.float64, device="cuda")
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    st = hweno.lib().hweno_max_dt_noalloc(ctypes.byref(g), 1.4, ctypes.c_void_p(m.data_ptr()), 0.6,
                                          ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(0))
    assert st == -1
    with pytest.raises(ValueError):
        hweno.max_dt_noalloc(g, 1.4, m, 0.6, out)
    torch.cuda.synchronize()
