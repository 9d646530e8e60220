"""Batched problems (hweno_create_batch): one persistent cooperative launch per
RK stage over every problem, against the single-problem path and the oracle."""
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


def small_batch():
    # uneven sizes, ragged against every tile shape, both problem kinds and boundary kinds
    return [W.four_quadrant_2d(16, seed=1), W.vortex_2d(32, seed=2), W.four_quadrant_2d(40, seed=3),
            W.vortex_2d(24, seed=4), W.four_quadrant_2d(64, seed=5), W.four_quadrant_2d(70, seed=6, ny=36)]


def rel_l1(a, b):
    return float(np.abs(a - b).sum() / max(np.abs(b).sum(), 1e-300))


def run_batch(problems, steps, variant=0, precision="fp64"):
    s = hweno.BatchSolver(problems, precision=precision)
    s.set_tile(variant)
    for k, p in enumerate(problems):
        s.set_moments(k, torch.from_numpy(p.m).cuda())
    dts, masks = [], []
    for _ in range(steps):
        s.step(cfl=0.6)
        dts.append(s.dts())
        masks.append([s.troubled_mask(k) for k in range(len(problems))])
    s.sync()
    out = [s.get_moments(k) for k in range(len(problems))]
    s.close()
    return out, dts, masks


def test_batch_equals_single_problem_path():
    probs = small_batch()
    got, dts, masks = run_batch(probs, 3)
    for k, p in enumerate(probs):
        s = hweno.Solver.from_problem(p)
        s.set_moments(p.m)
        for st in range(3):
            assert s.max_dt(0.6) == dts[st][k]
            s.step(dts[st][k])
            np.testing.assert_array_equal(s.troubled_mask(), masks[st][k])
        np.testing.assert_array_equal(s.get_moments(), got[k])
        s.close()


def test_batch_against_oracle(orc):
    probs = small_batch()[:3]
    got, dts, _ = run_batch(probs, 2)
    for k, p in enumerate(probs):
        cfg = orc.make_cfg(2, p.nx, p.ny, dx=p.dx, dy=p.dy, eq="euler", bc=p.bc)
        m = p.m
        for st in range(2):
            m, _, rc = orc.step(cfg, m, dts[st][k])
            assert rc == 0
        assert rel_l1(got[k], m) <= 1e-12


def test_tile_variants_give_identical_results():
    probs = small_batch()
    ref, _, _ = run_batch(probs, 2, variant=0)
    for v in (1, 2):
        got, _, _ = run_batch(probs, 2, variant=v)
        for a, b in zip(got, ref):
            np.testing.assert_array_equal(a, b)


def test_batch_fp32_within_tolerance():
    probs = small_batch()
    ref, _, _ = run_batch(probs, 3, precision="fp64")
    got, _, _ = run_batch(probs, 3, precision="fp32")
    for a, b in zip(got, ref):
        assert rel_l1(a, b) <= 5e-6


def test_autotuner_picks_a_variant(tmp_path, monkeypatch):
    from paper_2201_12193_gb300 import autotune
    monkeypatch.setenv("HWENO_TUNE_CACHE", str(tmp_path / "tune.json"))
    best, times = autotune.tune_batch(small_batch(), precision="fp32", steps=1)
    assert best in (0, 1, 2) and len(times) == 3
    best2, _ = autotune.tune_batch(small_batch(), precision="fp32", steps=1)
    assert best2 == best and (tmp_path / "tune.json").exists()


def test_batch_df64_meets_the_fp64_bar(orc):
    """Double-float batches: bitwise the single-problem double-float path, and
    within the FP64 parity bar (1e-12 relative L1) of the FP64 oracle."""
    probs = small_batch()
    got, dts, masks = run_batch(probs, 2, precision="df64")
    for k, p in enumerate(probs):
        s = hweno.Solver.from_problem(p, precision="df64")
        s.set_moments(p.m)
        for st in range(2):
            assert s.max_dt(0.6) == dts[st][k]
            s.step(dts[st][k])
            np.testing.assert_array_equal(s.troubled_mask(), masks[st][k])
        np.testing.assert_array_equal(s.get_moments(), got[k])
        s.close()
    for k, p in enumerate(probs[:3]):
        cfg = orc.make_cfg(2, p.nx, p.ny, dx=p.dx, dy=p.dy, eq="euler", bc=p.bc)
        m = p.m
        for st in range(2):
            m, _, rc = orc.step(cfg, m, dts[st][k])
            assert rc == 0
        assert rel_l1(got[k], m) <= 1e-12


def test_barrier_timeout_is_reported_and_the_handle_recovers():
    """The grid barrier's bounded wait: with one arrival more than the launched
    blocks every wait runs out after a short limit; the next synchronising call
    reports ETIMEOUT and rolls the step back, and once the barrier is set back
    the handle steps exactly as a fresh one."""
    probs = small_batch()[:3]
    want, _, _ = run_batch(probs, 1)
    s = hweno.BatchSolver(probs)
    for k, p in enumerate(probs):
        s.set_moments(k, torch.from_numpy(p.m).cuda())
    s.set_barrier(spin_limit=2000, extra_arrivals=1)
    s.step(cfl=0.6)
    with pytest.raises(hweno.HwenoError) as e:
        s.sync()
    assert e.value.status == -4
    for k, p in enumerate(probs):          # rolled back to the state before the step
        np.testing.assert_array_equal(s.get_moments(k), p.m)
    s.set_barrier()
    s.step(cfl=0.6)
    s.sync()
    for k in range(len(probs)):
        np.testing.assert_array_equal(s.get_moments(k), want[k])
    s.close()


def test_batch_reading_of_the_modification_matches_the_oracle(orc):
    """set_persistence(False): the modified first moments serve L only (the
    oracle's mod_in_L_only); bitwise the single-problem path with the same
    switch and within 1e-12 of the oracle."""
    probs = small_batch()[:3]
    s = hweno.BatchSolver(probs)
    s.set_persistence(False)
    for k, p in enumerate(probs):
        s.set_moments(k, torch.from_numpy(p.m).cuda())
    dts = []
    for _ in range(2):
        s.step(cfl=0.6)
        dts.append(s.dts())
    s.sync()
    got = [s.get_moments(k) for k in range(len(probs))]
    s.close()
    for k, p in enumerate(probs):
        one = hweno.Solver.from_problem(p)
        one.set_persistence(False)
        one.set_moments(p.m)
        for st in range(2):
            one.step(dts[st][k])
        np.testing.assert_array_equal(one.get_moments(), got[k])
        one.close()
        cfg = orc.make_cfg(2, p.nx, p.ny, dx=p.dx, dy=p.dy, eq="euler", bc=p.bc, mod_in_L_only=True)
        m = p.m
        for st in range(2):
            m, _, rc = orc.step(cfg, m, dts[st][k])
            assert rc == 0
        assert rel_l1(got[k], m) <= 1e-12
