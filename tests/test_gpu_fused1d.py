"""The fused 1D stage kernel (hweno_set_fused on a 1D handle: Steps 1-3 of
Sec. 2.1 in one launch per Runge-Kutta stage, the segment and its 4-cell halo in
shared memory) against the four-launch pipeline: the same device functions on
the same inputs, so states, troubled masks, KXRCF values, re-reconstruction
counts and step lengths must agree bit for bit, at every side kind (periodic,
transmissive, reflective), in every precision, across block seams."""
from __future__ import annotations

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


PROBS = [
    ("advection_periodic", lambda: W.advection_sin_1d(200), False),
    ("burgers", lambda: W.burgers_1d(160), False),
    ("shu_osher", lambda: W.shu_osher_1d(300), False),
    ("sod_ragged", lambda: W.sod_1d(131), False),
    ("lax", lambda: W.lax_1d(200), False),
    ("blast_wave_walls", lambda: W.blast_wave_1d(200), True),
    ("shu_osher_seams", lambda: W.shu_osher_1d(1000), False),
    # long grids take the 250-cell segments
    ("blast_wave_walls_long", lambda: W.blast_wave_1d(80000), True),
    ("advection_periodic_long", lambda: W.advection_sin_1d(76003), False),
]
IDS = [n for n, _, _ in PROBS]


def _pair(p, nopos, **kw):
    a = hweno.Solver.from_problem(p, **kw)
    b = hweno.Solver.from_problem(p, **kw)
    a.set_fused(False)
    b.set_fused(True)
    for s in (a, b):
        if nopos:
            s.set_positivity_check(False)
        s.set_moments(p.m)
    return a, b


@pytest.mark.parametrize("name,make,nopos", PROBS, ids=IDS)
@pytest.mark.parametrize("precision", ["fp64", "fp32", "df64"])
def test_fused1d_steps_equal_the_pipeline(name, make, nopos, precision):
    p = make()
    a, b = _pair(p, nopos, precision=precision)
    a.rerecon_count()
    b.rerecon_count()
    for _ in range(8):
        dt = a.max_dt(0.6)
        assert b.max_dt(0.6) == dt
        a.step(dt)
        b.step(dt)
        np.testing.assert_array_equal(a.troubled_mask(), b.troubled_mask())
    np.testing.assert_array_equal(a.get_moments(), b.get_moments())
    assert a.rerecon_count() == b.rerecon_count()
    a.close()
    b.close()


@pytest.mark.parametrize("indicator", ["kxrcf", "none", "all"])
def test_fused1d_rhs_equals_the_pipeline(indicator):
    """One evaluation of L (and the modified moments, flags, KXRCF values)."""
    for p in (W.shu_osher_1d(700), W.blast_wave_1d(300)):
        a = hweno.Solver.from_problem(p, indicator=indicator)
        b = hweno.Solver.from_problem(p, indicator=indicator)
        a.set_fused(False)
        b.set_fused(True)
        res = []
        for s in (a, b):
            U = torch.from_numpy(p.m).cuda()
            Um, L = torch.empty_like(U), torch.empty_like(U)
            mask = torch.empty(p.nx, dtype=torch.uint8, device="cuda")
            aleph = torch.zeros(p.nx, dtype=torch.float64, device="cuda")
            s.rhs(U, Um, L, mask, aleph)
            torch.cuda.synchronize()
            res.append([x.cpu().numpy() for x in (Um, L, mask, aleph)])
        for x, y in zip(*res):
            np.testing.assert_array_equal(x, y)
        a.close()
        b.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_fused1d_device_driven_run(precision):
    """Shu-Osher (N = 4000, the C1 size) run device-driven to t = 0.3, fused
    against the pipeline: the same number of steps and the same state."""
    p = W.shu_osher_1d(4000)
    a, b = _pair(p, False, precision=precision)
    ta, na = a.advance(0.3, 0.6)
    tb, nb = b.advance(0.3, 0.6)
    assert na == nb and ta == tb and na > 50
    np.testing.assert_array_equal(a.get_moments(), b.get_moments())
    a.close()
    b.close()


def test_fused1d_large_grid_sampled():
    """2^20 cells (4,195 segments of 250 cells): two steps, bitwise the pipeline."""
    p = W.shu_osher_1d(1 << 20)
    a, b = _pair(p, False, precision="fp32")
    for _ in range(2):
        dt = a.max_dt(0.6)
        a.step(dt)
        b.step(dt)
    np.testing.assert_array_equal(a.get_moments(), b.get_moments())
    a.close()
    b.close()


def _both(a, b, fn):
    """fn on both handles: the same status (a rolled-back step included)."""
    st = []
    for s in (a, b):
        try:
            fn(s)
            st.append(0)
        except hweno.HwenoError as e:
            st.append(e.status)
    assert st[0] == st[1], st
    return st[0]


@pytest.mark.parametrize("nx", [4, 5, 7, 31, 32, 33, 65, 257])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_fused1d_tiny_and_ragged_grids(nx, precision):
    """The smallest grids (every ghost's image inside a 4-cell grid) and ragged
    last segments, on every side kind: bitwise the pipeline, failures included."""
    for make, nopos in ((W.sod_1d, False), (W.blast_wave_1d, True), (W.advection_sin_1d, False),
                        (W.burgers_1d, False)):
        p = make(nx)
        a, b = _pair(p, nopos, precision=precision)
        for _ in range(3):
            dt = a.max_dt(0.6)
            if _both(a, b, lambda s: s.step(dt)):
                break
        np.testing.assert_array_equal(a.get_moments(), b.get_moments())
        np.testing.assert_array_equal(a.troubled_mask(), b.troubled_mask())
        a.close()
        b.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_fused1d_modification_in_L_only(precision):
    """Reading B of the persistence of eq. (vi) (hweno_set_persistence 0): the
    fused stage equals the pipeline bit for bit."""
    for p, nopos in ((W.shu_osher_1d(600), False), (W.blast_wave_1d(300), True)):
        a, b = _pair(p, nopos, precision=precision)
        for s in (a, b):
            s.set_persistence(False)
        for _ in range(6):
            dt = a.max_dt(0.6)
            a.step(dt)
            b.step(dt)
        np.testing.assert_array_equal(a.get_moments(), b.get_moments())
        a.close()
        b.close()


@pytest.mark.parametrize("indicator", ["kxrcf", "none", "all"])
def test_fused1d_rhs_scalar_laws(indicator):
    """L, the stage input with eq. (vi) applied, masks and KXRCF values of the
    scalar laws (LLF fluxes, periodic sides) against the pipeline."""
    for p in (W.advection_sin_1d(300), W.burgers_1d(260)):
        res = []
        for fused in (False, True):
            s = hweno.Solver.from_problem(p, indicator=indicator)
            s.set_fused(fused)
            U = torch.from_numpy(p.m).cuda()
            Um, L = torch.empty_like(U), torch.empty_like(U)
            mask = torch.empty(p.nx, dtype=torch.uint8, device="cuda")
            aleph = torch.zeros(p.nx, dtype=torch.float64, device="cuda")
            s.rhs(U, Um, L, mask, aleph)
            torch.cuda.synchronize()
            res.append([x.cpu().numpy() for x in (Um, L, mask, aleph)])
            s.close()
        for x, y in zip(*res):
            np.testing.assert_array_equal(x, y)


def test_fused1d_is_the_default():
    """A 1D handle runs the fused stage unless asked otherwise: one launch per
    stage; the characteristic-wise and TVB forms keep the pipeline."""
    p = W.shu_osher_1d(500)
    for kw, fused in (({}, True), ({"indicator": "none"}, True), ({"charwise": True}, False),
                      ({"indicator": "tvb", "tvb_m": 1.0}, False)):
        s = hweno.Solver.from_problem(p, **kw)
        s.set_moments(p.m)
        s.profile(True)
        s.step(s.max_dt(0.6))
        s.sync()
        prof = s.profile_read()
        assert (prof["fused_stage"][1] == 3) == fused, kw
        assert (prof["update"][1] == 3) == (not fused), kw
        s.close()


def test_fused1d_refused_for_characteristic_reconstruction():
    p = W.shu_osher_1d(100)
    s = hweno.Solver.from_problem(p, charwise=True)
    with pytest.raises(hweno.HwenoError):
        s.set_fused(True)
    s.close()
