"""Row-slab decomposition on one GPU (decomp.LocalSlabs): the grid split into
slabs with 4 halo rows, refilled device to device before every stage, must
advance exactly as the whole grid, bit for bit (the halo covers every cell a
stage reads: moments -> point values -> flags -> re-reconstruction -> fluxes).
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2201_12193_gb300 import decomp, hweno, workloads as W  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_12193_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _whole(p, nsteps, **kw):
    s = hweno.Solver.from_problem(p, **kw.get("solver", {}))
    if kw.get("fused"):
        s.set_fused(True)
    if kw.get("nopos"):
        s.set_positivity_check(False)
    s.set_stream(torch.cuda.current_stream())
    s.set_moments(torch.from_numpy(p.m).cuda())
    dts, masks = [], []
    for _ in range(nsteps):
        dt = s.max_dt(0.6)
        s.step(dt)
        dts.append(dt)
        masks.append(s.troubled_mask())
    m = s.get_moments()
    s.close()
    return m, dts, masks


def _slabs(p, nslabs, nsteps, **kw):
    d = decomp.LocalSlabs(p, nslabs, **kw.get("solver", {}))
    for s in d.solvers:
        if kw.get("fused"):
            s.set_fused(True)
        if kw.get("nopos"):
            s.set_positivity_check(False)
    d.set_moments(p.m)
    dts, masks = [], []
    for _ in range(nsteps):
        dt = d.max_dt(0.6)
        d.step(dt)
        dts.append(dt)
        masks.append(d.troubled_masks())
    m = d.gather()
    d.close()
    return m, dts, masks


@pytest.mark.parametrize("name,make,nslabs,nsteps,kw", [
    ("four_quadrant_2048", lambda: W.four_quadrant_2d(2048, seed=0), 4, 2, {}),
    ("four_quadrant_ragged", lambda: W.four_quadrant_2d(64, seed=3, ny=75), 3, 3, {}),
    ("vortex_periodic", lambda: W.vortex_2d(64, seed=2), 3, 3, {}),
    ("walled_blast", lambda: W.walled_blast_2d(64, seed=1, ncircles=3), 2, 3,
     {"solver": {"precision": "df64"}, "nopos": True}),
    ("four_quadrant_fused_fp32", lambda: W.four_quadrant_2d(256, seed=5), 3, 3,
     {"solver": {"precision": "fp32"}, "fused": True}),
], ids=["four_quadrant_2048", "four_quadrant_ragged", "vortex_periodic", "walled_blast_df64",
        "four_quadrant_fused_fp32"])
def test_slabs_equal_the_whole_grid(name, make, nslabs, nsteps, kw):
    p = make()
    m1, dt1, mk1 = _whole(p, nsteps, **kw)
    m2, dt2, mk2 = _slabs(p, nslabs, nsteps, **kw)
    assert dt1 == dt2
    for a, b in zip(mk1, mk2):
        np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(m1, m2)
    assert sum(int(a.sum()) for a in mk1) > 0 or name == "vortex_periodic"


def test_stage_by_stage_equals_step():
    """hweno_stage run three times equals hweno_step bit for bit, and a stage
    out of order is refused."""
    p = W.four_quadrant_2d(48, seed=2, ny=40)
    a = hweno.Solver.from_problem(p)
    b = hweno.Solver.from_problem(p)
    for s in (a, b):
        s.set_moments(p.m)
    dt = a.max_dt(0.6)
    a.step(dt)
    for k in range(3):
        b.stage(k, dt)
    np.testing.assert_array_equal(a.get_moments(), b.get_moments())
    with pytest.raises(hweno.HwenoError):
        b.stage(1, dt)
    b.stage(0, dt)
    with pytest.raises(hweno.HwenoError):
        b.stage(1, 0.5 * dt)
    a.close()
    b.close()
