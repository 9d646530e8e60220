"""hweno_max_dt_noalloc, the CFL reduction that allocates nothing, against the
handle-based hweno_max_dt.

The allocation-free entry point serves callers that cannot call cudaMalloc
(a frozen memory budget, no room for the implicit synchronisation of an
allocation, no handle to keep).  Its partial maxima live in a static device
array shared by every call, so this test makes two calls in a row (the largest
grid the array accepts, then a smaller one) and checks both against the
existing entry point.  This file is collected last on purpose.
"""
from __future__ import annotations

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


def test_no_alloc_matches_handle_dt_on_two_calls():
    cfl = 0.6
    problems = [W.four_quadrant_2d(2048, seed=7), W.shu_osher_1d(300)]
    want = [_handle_dt(p, cfl) for p in problems]
    out = torch.full((3,), -1.0, dtype=torch.float64, device="cuda")
    for p, w in zip(problems, want):
        m = torch.from_numpy(p.m).cuda()
        hweno.max_dt_noalloc(_grid(p), p.gamma, m, cfl, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got)) and got[0] > 0.0
        assert math.isclose(got[2], w, rel_tol=1e-13), (got, w)


def test_no_alloc_rejects_grids_beyond_its_scratch():
    p = W.four_quadrant_2d(64, seed=1)
    g = _grid(p)
    g.nx, g.ny, g.x1, g.y1 = 2050, 2048, 2050 / 2048, 1.0       # 4,198,400 > 4,194,304 cells
    m = torch.zeros(4 * 3 * 2048 * 2050, dtype=torch.float64, device="cuda")
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    with pytest.raises(hweno.HwenoError) as e:
        hweno.max_dt_noalloc(g, 1.4, m, 0.6, out)
    assert e.value.status == -1
