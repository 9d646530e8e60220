"""The FP32-bulk pipeline's float copy of the state (the update kernel writes
each new state value rounded to nearest beside the FP64 one; the next
reconstruction gathers its 3 x 3 moments from it instead of converting FP64
moments one by one).  The copy must equal the FP64 state rounded to nearest at
every stage start, whatever last wrote the state: a stage, hweno_set_moments,
a halo copy (hweno_copy_rows) or the fused stage, which keeps no copy.
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


def _rhs(s, U):
    Ud = torch.from_numpy(np.ascontiguousarray(U)).cuda()
    Um, L = torch.empty_like(Ud), torch.empty_like(Ud)
    mask = torch.empty((s.ny, s.nx), dtype=torch.uint8, device="cuda")
    s.rhs(Ud, Um, L, mask, None)
    torch.cuda.synchronize()
    return Um.cpu().numpy(), L.cpu().numpy()


@pytest.mark.parametrize("make", [lambda: W.four_quadrant_2d(96, seed=4, ny=72),
                                  lambda: W.vortex_2d(64, seed=3)], ids=["four_quadrant", "vortex"])
def test_first_stage_equals_the_converting_path(make):
    """hweno_rhs reconstructs from its FP64 input converted moment by moment;
    the first stage of a step reconstructs from the float copy.  Both give
    the same L, so U^(1) = U' + dt L up to the one rounding of the FMA (the
    copy read through a wrong plane, a stale buffer or another rounding would
    move it by FP32 amounts)."""
    p = make()
    s = hweno.Solver.from_problem(p, precision="fp32")
    s.set_moments(p.m)
    dt = s.max_dt(0.6)
    Um, L = _rhs(s, p.m)
    s.stage(0, dt)
    U1 = torch.empty(p.m.size, dtype=torch.float64, device="cuda")
    s.copy_rows(0, p.ny, U1, False)          # the state the next stage reads: U^(1)
    U1 = U1.cpu().numpy().reshape(p.m.shape)
    s.close()
    want = Um + dt * L
    scale = np.abs(Um) + np.abs(dt * L)
    assert np.all(np.abs(U1 - want) <= 5e-16 * scale), float((np.abs(U1 - want) / (scale + 1e-300)).max())


def test_set_moments_renews_the_copy():
    """A second hweno_set_moments (other data) before stepping: the steps equal
    those of a fresh handle given the second data."""
    p = W.four_quadrant_2d(80, seed=2, ny=60)
    q = W.four_quadrant_2d(80, seed=7, ny=60)
    a = hweno.Solver.from_problem(p, precision="fp32")
    a.set_moments(p.m)
    a.step(a.max_dt(0.6))
    a.set_moments(q.m)
    b = hweno.Solver.from_problem(q, precision="fp32")
    b.set_moments(q.m)
    for _ in range(3):
        dt = b.max_dt(0.6)
        a.step(dt)
        b.step(dt)
    np.testing.assert_array_equal(a.get_moments(), b.get_moments())
    a.close()
    b.close()


def test_fused_then_pipeline_renews_the_copy():
    """Steps with the fused stage (no float copy kept), then the pipeline:
    equal to a pipeline handle started from the fused handle's state."""
    p = W.four_quadrant_2d(96, seed=5, ny=64)
    a = hweno.Solver.from_problem(p, precision="fp32")
    a.set_fused(True)
    a.set_moments(p.m)
    for _ in range(2):
        a.step(a.max_dt(0.6))
    mid = a.get_moments()
    a.set_fused(False)
    b = hweno.Solver.from_problem(p, precision="fp32")
    b.set_moments(mid)
    for _ in range(3):
        dt = b.max_dt(0.6)
        a.step(dt)
        b.step(dt)
    np.testing.assert_array_equal(a.get_moments(), b.get_moments())
    a.close()
    b.close()


def test_halo_copies_renew_the_copy():
    """Row slabs of the FP32 pipeline (halo rows written by hweno_copy_rows
    before every stage) equal the whole grid bit for bit."""
    p = W.four_quadrant_2d(128, seed=6, ny=90)
    whole = hweno.Solver.from_problem(p, precision="fp32")
    whole.set_moments(p.m)
    d = decomp.LocalSlabs(p, 3, precision="fp32")
    d.set_moments(p.m)
    for _ in range(3):
        dt = whole.max_dt(0.6)
        assert d.max_dt(0.6) == dt
        whole.step(dt)
        d.step(dt)
    np.testing.assert_array_equal(whole.get_moments(), d.gather())
    whole.close()
    d.close()


def test_device_driven_run_equals_host_loop_fp32():
    p = W.four_quadrant_2d(80, seed=3, ny=64)
    a = hweno.Solver.from_problem(p, precision="fp32")
    a.set_moments(p.m)
    t, n = a.advance(0.02, 0.6)
    b = hweno.Solver.from_problem(p, precision="fp32")
    b.set_moments(p.m)
    nb = b.run(0.02, 0.6)
    assert n == nb and n > 5
    np.testing.assert_array_equal(a.get_moments(), b.get_moments())
    a.close()
    b.close()


@pytest.mark.parametrize("make", [lambda: W.four_quadrant_2d(200, seed=4, ny=150),
                                  lambda: W.four_quadrant_2d(97, seed=8, ny=45),
                                  lambda: W.vortex_2d(128, seed=3)],
                         ids=["four_quadrant_200x150", "ragged_97x45", "vortex_periodic"])
def test_tma_staged_update_is_bitwise_the_global_path(make):
    """The FP32 update with interior tiles staged through TMA (each tile's
    point values in shared memory) against the same kernel code reading global
    memory: identical states, masks and step lengths over host-driven steps
    (all three stages) and a device-driven run."""
    p = make()
    a = hweno.Solver.from_problem(p, precision="fp32")
    a.set_tma(True)
    b = hweno.Solver.from_problem(p, precision="fp32")
    for s in (a, b):
        s.set_moments(p.m)
    for _ in range(4):
        dt = a.max_dt(0.6)
        assert b.max_dt(0.6) == dt
        a.step(dt)
        b.step(dt)
        np.testing.assert_array_equal(a.troubled_mask(), b.troubled_mask())
    np.testing.assert_array_equal(a.get_moments(), b.get_moments())
    ta, na = a.advance(a.time() + 0.01, 0.6)
    tb, nb = b.advance(b.time() + 0.01, 0.6)
    assert na == nb and ta == tb
    np.testing.assert_array_equal(a.get_moments(), b.get_moments())
    a.close()
    b.close()


def test_tma_refused_where_it_does_not_apply():
    for kw, p in (({"precision": "fp64"}, W.four_quadrant_2d(64, seed=1)),
                  ({"precision": "df64"}, W.four_quadrant_2d(64, seed=1)),
                  ({"precision": "fp32"}, W.burgers_2d(32)),
                  ({"precision": "fp32"}, W.shu_osher_1d(100))):
        s = hweno.Solver.from_problem(p, **kw)
        with pytest.raises(hweno.HwenoError):
            s.set_tma(True)
        s.set_tma(False)
        s.close()
