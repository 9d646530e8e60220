"""The fused stage kernel (hweno_set_fused: Steps 1-3 of Sec. 2.2 in one launch
per Runge-Kutta stage, point values in shared memory) against the CPU FP64
oracle and against the four-launch pipeline.

Bars as in test_gpu_parity: FP64 and double-float states within 1e-12
relative L1 of the oracle, masks identical on identical stage input, L per
element within 1e-10 relative plus 2e-11 of its plane's largest value; FP32
bulk within its stated 5e-6.  Against the pipeline the point values of
interior cells are the same numbers; the interior quadrature sums in another
order and ghost cells are reconstructed rather than mirrored, so the two
agree to a few units of rounding (1e-13 relative L1), not bit for bit.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2201_12193_gb300 import hweno, workloads as W  # noqa: E402
from test_gpu_parity import TOL, _window_oracle, assert_L_close, cfg_of, gpu_rhs, rel_l1  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_12193_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _perturbed(p, seed, amp=1e-3):
    rng = np.random.default_rng(seed)
    m = p.m.copy()
    m[:, 1:] += amp * rng.standard_normal(m[:, 1:].shape) * np.abs(m[:, :1]).mean()
    return m


PROBS = [
    ("four_quadrant_ragged", lambda: W.four_quadrant_2d(70, seed=3, ny=45)),
    ("four_quadrant_tall", lambda: W.four_quadrant_2d(30, seed=5, ny=150)),
    ("vortex_periodic", lambda: W.vortex_2d(48, seed=2)),
    ("blast", lambda: W.blast_2d(40, seed=1, ncircles=3)),
    ("walled_blast", lambda: W.walled_blast_2d(40, seed=1, ncircles=3)),
    ("walls_mixed", lambda: W.walled_blast_2d(36, seed=2, ncircles=2,
                                              walls=("periodic", "periodic", "reflective", "transmissive"))),
    ("smallest", lambda: W.four_quadrant_2d(4, seed=1)),
]
IDS = [n for n, _ in PROBS]


def fused_solver(p, **kw):
    s = hweno.Solver.from_problem(p, **kw)
    s.set_fused(True)
    return s


@pytest.mark.parametrize("name,make", PROBS, ids=IDS)
@pytest.mark.parametrize("indicator", ["kxrcf", "none", "all"])
def test_fused_rhs_parity(orc, name, make, indicator):
    """One evaluation of L with the troubled-cell steps on identical input."""
    p = make()
    s = fused_solver(p, indicator=indicator)
    for seed in (0, 1):
        U = p.m if seed == 0 else _perturbed(p, seed)
        Um_g, L_g, mask_g, aleph_g = gpu_rhs(s, U)
        Um_o, L_o, mask_o, aleph_o, rc = orc.rhs(cfg_of(orc, p, indicator=indicator), U)
        assert rc == 0
        assert not (np.abs(aleph_o - 1.0) < 1e-10).any()
        assert np.array_equal(mask_g, mask_o), (int(mask_g.sum()), int(mask_o.sum()))
        assert rel_l1(Um_g, Um_o) <= TOL
        assert_L_close(L_g, L_o)
        if indicator == "kxrcf":
            np.testing.assert_allclose(aleph_g, aleph_o, rtol=1e-9, atol=1e-9)
    s.close()


@pytest.mark.parametrize("name,make,nsteps", [
    ("four_quadrant", lambda: W.four_quadrant_2d(70, seed=3, ny=45), 5),
    ("vortex", lambda: W.vortex_2d(48, seed=2), 3),
    ("blast", lambda: W.blast_2d(48, seed=0, ncircles=3), 6),
    ("walled_blast", lambda: W.walled_blast_2d(40, seed=1, ncircles=3), 5),
], ids=["four_quadrant", "vortex", "blast", "walled_blast"])
@pytest.mark.parametrize("persist", [True, False], ids=["persist", "L_only"])
@pytest.mark.parametrize("precision", ["fp64", "df64"])
def test_fused_steps_parity(orc, name, make, nsteps, persist, precision):
    """SSP-RK3 steps with the CFL rule; masks of every stage identical; both
    readings of the modification's persistence."""
    p = make()
    s = fused_solver(p, precision=precision)
    s.set_persistence(persist)
    if "blast" in name:
        s.set_positivity_check(False)
    s.set_moments(torch.from_numpy(p.m).cuda())
    cfg = cfg_of(orc, p, mod_in_L_only=not persist)
    m = p.m
    for _ in range(nsteps):
        dt = s.max_dt(0.6)
        assert math.isclose(dt, orc.max_dt(cfg, m, 0.6), rel_tol=1e-13)
        s.step(dt)
        m, masks, rc = orc.step(cfg, m, dt)
        assert rc == 0
        assert np.array_equal(s.troubled_mask().reshape(3, -1), masks)
    assert rel_l1(s.get_moments(), m) <= TOL
    s.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-13), ("df64", 1e-13), ("fp32", 1e-6)])
def test_fused_matches_pipeline(precision, tol):
    """Fused against the four-launch pipeline in each precision: identical
    masks, states within a few units of rounding (FP32: of its own rounding)."""
    for p in (W.vortex_2d(64, seed=3), W.four_quadrant_2d(96, seed=4, ny=72)):
        a = hweno.Solver.from_problem(p, precision=precision)
        b = fused_solver(p, precision=precision)
        for s in (a, b):
            s.set_moments(p.m)
        for _ in range(4):
            dt = a.max_dt(0.6)
            a.step(dt)
            b.step(dt)
            assert np.array_equal(a.troubled_mask(), b.troubled_mask())
        assert rel_l1(b.get_moments(), a.get_moments()) <= tol
        a.close()
        b.close()


def test_fused_fp32_within_tolerance(orc):
    """FP32 bulk through the fused kernel against the FP64 oracle: 5 steps
    within the FP32 form's stated 5e-6."""
    p = W.four_quadrant_2d(64, seed=6)
    s = fused_solver(p, precision="fp32")
    s.set_moments(p.m)
    cfg = cfg_of(orc, p)
    m = p.m
    for _ in range(5):
        dt = orc.max_dt(cfg, m, 0.6)
        s.step(dt)
        m, _, rc = orc.step(cfg, m, dt)
        assert rc == 0
    assert rel_l1(s.get_moments(), m) <= 5e-6
    s.close()


def test_fused_conserves_on_periodic_grids():
    """Shared faces get one flux from both sides: the totals stay to FP64 rounding."""
    p = W.four_quadrant_2d(64, seed=4)
    p.bc = ("periodic",) * 4
    for prec in ("fp64", "fp32"):
        s = fused_solver(p, precision=prec)
        s.set_moments(p.m)
        t0 = s.totals()
        for _ in range(5):
            s.step(0.5 * s.max_dt(0.6))
        t1 = s.totals()
        assert np.all(np.abs(t1 - t0) <= 1e-13 * np.abs(t0).max()), (prec, t1 - t0)
        s.close()


def test_fused_advance_equals_host_driven_run():
    p = W.four_quadrant_2d(80, seed=2, ny=60)
    a = fused_solver(p)
    a.set_moments(p.m)
    t, n = a.advance(0.03, 0.6)
    b = fused_solver(p)
    b.set_moments(p.m)
    nb = b.run(0.03, 0.6)
    assert n == nb and n > 12
    assert np.array_equal(a.get_moments(), b.get_moments())
    a.close()
    b.close()


def test_fused_rerecon_count_equals_the_pipeline():
    p = W.four_quadrant_2d(96, seed=4, ny=72)
    counts = []
    for fused in (False, True):
        s = hweno.Solver.from_problem(p)
        s.set_fused(fused)
        s.set_moments(p.m)
        s.rerecon_count()
        s.step(s.max_dt(0.6))
        counts.append((s.rerecon_count(), int(s.troubled_mask().sum())))
        s.close()
    assert counts[0] == counts[1] and counts[0][0] > 0


def test_fused_rejected_where_it_does_not_apply():
    for kw, p in (({"indicator": "tvb", "tvb_m": 1.0}, W.four_quadrant_2d(16, seed=1)),
                  ({"charwise": True}, W.shu_osher_1d(100)), ({}, W.burgers_2d(16))):
        s = hweno.Solver.from_problem(p, **kw)
        with pytest.raises(hweno.HwenoError):
            s.set_fused(True)
        s.close()


@pytest.mark.parametrize("precision,tol", [("fp64", TOL), ("fp32", 5e-6)])
def test_fused_full_size_sampled(orc, precision, tol):
    """2048 x 2048 four-quadrant data (the benchmark's workload and launch
    configuration): one step, sampled cells against oracle windows, including
    cells on block-strip seams (columns 25/26, rows 63/64) and corners."""
    p = W.four_quadrant_2d(2048, seed=0)
    s = fused_solver(p, precision=precision)
    s.set_moments(torch.from_numpy(p.m).cuda())
    dt = s.max_dt(0.6)
    s.step(dt)
    got = s.get_moments()
    rng = np.random.default_rng(2)
    picks = [(1024, 1024), (25, 63), (26, 64), (1039, 1023), (0, 0), (2047, 2047), (2047, 0), (0, 2047)]
    picks += [(int(a), int(b)) for a in rng.integers(1000, 1048, 4) for b in rng.integers(0, 2048, 1)]
    for ci, cj in picks:
        want = _window_oracle(orc, p, p.m, ci, cj, 14, dt, 1)
        g = got[:, :, cj, ci]
        assert np.abs(g - want).sum() <= tol * np.abs(want).sum(), (ci, cj, g, want)
    s.close()
