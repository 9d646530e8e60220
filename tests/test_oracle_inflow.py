"""CPU pins of the oracle's fixed-state (inflow) ghost cells, their moving
segments and the Runge-Kutta stage times (the boundaries of Examples 3.9 and
3.10).

* A uniform flow entering through an inflow side that holds its own state is
  steady: L vanishes, no cell is flagged.
* Locality of a segment: far from the split, L equals that of the side made
  wholly of the segment's kind (fixed state) or wholly of the side's own kind.
* A moving segment at time t equals a resting one at c0 + speed t.
* orc_step evaluates its stages at t, t + dt and t + dt/2 (the SSP-RK3
  abscissae): three right-hand sides at those times, combined by the scheme's
  stage formulas, give the step.
* Corners: a problem mirror-symmetric about y = 0 (left inflow whose state has
  its y momentum reversed below y = 0) equals its upper half with a wall at
  y = 0, where the corner ghost is the wall image of the inflow ghost.
* The double Mach reflection runs a few steps with troubled cells on its shock.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

from paper_2201_12193_gb300 import workloads as W


def _smooth_state(nx, ny, seed=0, x0=0.0, y0=0.0, h=None):
    rng = np.random.default_rng(seed)
    h = h or 1.0 / ny
    xc = x0 + (np.arange(nx) + 0.5) * h
    yc = y0 + (np.arange(ny) + 0.5) * h
    X, Y = np.meshgrid(xc, yc)
    a = rng.uniform(0.1, 0.3, 4)
    rho = 1.0 + a[0] * np.sin(2 * X + Y)
    u = 0.6 + a[1] * np.cos(X - Y)
    v = 0.2 + a[2] * np.sin(X + 3 * Y)
    p = 1.0 + a[3] * np.cos(2 * Y)
    m = np.zeros((4, 3, ny, nx))
    m[:, 0] = W.prim_to_cons_2d(rho, u, v, p)
    m[:, 1] = 0.01 * np.cos(X)[None]
    m[:, 2] = 0.01 * np.sin(Y)[None]
    return m


def test_uniform_inflow_is_steady(orc):
    nx, ny = 12, 8
    s = tuple(float(x) for x in W.prim_to_cons_2d(1.3, 0.7, -0.2, 0.9))
    m = np.zeros((4, 3, ny, nx))
    m[:, 0] = np.array(s)[:, None, None]
    fixed = ({"b": s}, None, None, None)
    cfg = orc.make_cfg(2, nx, ny, dx=1.0 / ny, dy=1.0 / ny, bc=("inflow", "transmissive", "periodic", "periodic"),
                       fixed=fixed)
    _, L, mask, _, rc = orc.rhs(cfg, m)
    assert rc == 0 and mask.sum() == 0
    assert np.abs(L).max() <= 1e-12


@pytest.mark.parametrize("side_kind", ["reflective", "transmissive"])
def test_segment_is_local(orc, side_kind):
    nx, ny = 24, 8
    h = 1.0 / ny
    m = _smooth_state(nx, ny, seed=1, h=h)
    a = tuple(float(x) for x in W.prim_to_cons_2d(1.5, 0.3, 0.4, 1.2))
    c0 = 12 * h                      # ghost columns 0..11 take the fixed state
    kw = dict(dx=h, dy=h, indicator="kxrcf")
    bc = ("transmissive", "transmissive", side_kind, "transmissive")
    seg = orc.make_cfg(2, nx, ny, bc=bc, fixed=(None, None, {"a": a, "c0": c0}, None), **kw)
    whole_fixed = orc.make_cfg(2, nx, ny, bc=("transmissive", "transmissive", "inflow", "transmissive"),
                               fixed=(None, None, {"b": a}, None), **kw)
    whole_kind = orc.make_cfg(2, nx, ny, bc=bc, **kw)
    _, Ls, _, _, rc = orc.rhs(seg, m)
    _, Lf, _, _, _ = orc.rhs(whole_fixed, m)
    _, Lk, _, _, _ = orc.rhs(whole_kind, m)
    assert rc == 0
    np.testing.assert_array_equal(Ls[..., :8], Lf[..., :8])
    np.testing.assert_array_equal(Ls[..., 16:], Lk[..., 16:])
    assert np.abs(Ls[..., 0, :8] - Lk[..., 0, :8]).max() > 1e-6       # the fixed state matters


def test_moving_segment_equals_resting_one(orc):
    nx, ny = 24, 8
    h = 1.0 / ny
    m = _smooth_state(nx, ny, seed=2, h=h)
    a = tuple(float(x) for x in W.prim_to_cons_2d(2.0, 0.5, -0.3, 3.0))
    b = tuple(float(x) for x in W.prim_to_cons_2d(1.0, 0.1, 0.0, 1.0))
    c0, speed, t = 0.41, 7.3, 0.123
    bc = ("transmissive", "transmissive", "transmissive", "inflow")
    moving = orc.make_cfg(2, nx, ny, dx=h, dy=h, bc=bc, t=t, fixed=(None, None, None, {"a": a, "b": b, "c0": c0,
                                                                                        "speed": speed}))
    resting = orc.make_cfg(2, nx, ny, dx=h, dy=h, bc=bc, fixed=(None, None, None, {"a": a, "b": b,
                                                                                   "c0": c0 + speed * t}))
    at_zero = orc.make_cfg(2, nx, ny, dx=h, dy=h, bc=bc, fixed=(None, None, None, {"a": a, "b": b, "c0": c0}))
    _, L1, _, _, _ = orc.rhs(moving, m)
    _, L2, _, _, _ = orc.rhs(resting, m)
    _, L0, _, _, _ = orc.rhs(at_zero, m)
    np.testing.assert_array_equal(L1, L2)
    assert np.abs(L1 - L0).max() > 1e-6


def test_step_uses_the_rk_abscissae(orc):
    nx, ny = 24, 8
    h = 1.0 / ny
    m = _smooth_state(nx, ny, seed=3, h=h)
    a = tuple(float(x) for x in W.prim_to_cons_2d(2.0, 0.5, -0.3, 3.0))
    b = tuple(float(x) for x in W.prim_to_cons_2d(1.0, 0.1, 0.0, 1.0))
    fixed = (None, None, None, {"a": a, "b": b, "c0": 0.3, "speed": 40.0})
    kw = dict(dx=h, dy=h, bc=("transmissive", "transmissive", "transmissive", "inflow"), fixed=fixed)
    t, dt = 0.01, 0.004            # the split moves 0.16 = 1.3 cells per step
    got, _, rc = orc.step(orc.make_cfg(2, nx, ny, t=t, **kw), m, dt)
    assert rc == 0
    Um0, L0, _, _, _ = orc.rhs(orc.make_cfg(2, nx, ny, t=t, **kw), m)
    U1 = Um0 + dt * L0
    Um1, L1, _, _, _ = orc.rhs(orc.make_cfg(2, nx, ny, t=t + dt, **kw), U1)
    U2 = 0.75 * Um0 + 0.25 * Um1 + 0.25 * dt * L1
    Um2, L2, _, _, _ = orc.rhs(orc.make_cfg(2, nx, ny, t=t + 0.5 * dt, **kw), U2)
    want = Um0 / 3.0 + 2.0 / 3.0 * Um2 + 2.0 / 3.0 * dt * L2
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-13 * np.abs(want).max())
    # stages at t only would differ
    Um1b, L1b, _, _, _ = orc.rhs(orc.make_cfg(2, nx, ny, t=t, **kw), U1)
    assert np.abs(L1b - L1).max() > 1e-6


def test_inflow_corner_mirror_symmetry(orc):
    nx, nh = 10, 6                    # half height nh, full height 2 nh
    h = 1.0 / nh
    up = _smooth_state(nx, nh, seed=4, h=h)
    up[2, 0] = np.abs(up[2, 0]) + 0.05          # a y momentum that the mirror reverses
    full = np.concatenate([up[:, :, ::-1], up], axis=2)
    full[2, :, :nh] *= -1.0                     # y momentum reversed below y = 0
    full[:, 2, :nh] *= -1.0                     # y first moments reversed below y = 0
    s = tuple(float(x) for x in W.prim_to_cons_2d(1.4, 0.8, 0.3, 1.1))
    s_mirror = (s[0], s[1], -s[2], s[3])
    kw = dict(dx=h, dy=h, indicator="kxrcf")
    cfg_full = orc.make_cfg(2, nx, 2 * nh, y0=-1.0, bc=("inflow", "transmissive", "transmissive", "transmissive"),
                            fixed=({"a": s_mirror, "b": s, "c0": 0.0}, None, None, None), **kw)
    cfg_half = orc.make_cfg(2, nx, nh, bc=("inflow", "transmissive", "reflective", "transmissive"),
                            fixed=({"b": s}, None, None, None), **kw)
    _, Lf, mf, _, rc1 = orc.rhs(cfg_full, full)
    _, Lh, mh, _, rc2 = orc.rhs(cfg_half, up)
    assert rc1 == 0 and rc2 == 0
    np.testing.assert_allclose(Lf[:, :, nh:], Lh, rtol=0, atol=1e-12 * np.abs(Lh).max())
    np.testing.assert_array_equal(mf.reshape(2 * nh, nx)[nh:], mh.reshape(nh, nx))


def test_double_mach_first_steps(orc):
    p = W.double_mach_2d(12)
    cfg = orc.make_cfg(2, p.nx, p.ny, dx=p.dx, dy=p.dy, bc=p.bc, fixed=p.fixed, x0=p.x0, y0=p.y0)
    m, t = p.m, 0.0
    mass0 = m[0, 0].sum()
    for _ in range(3):
        cfg.t = t
        dt = orc.max_dt(cfg, m, 0.6)
        m, masks, rc = orc.step(cfg, m, dt)
        assert rc == 0 and masks.sum() > 0
        t += dt
    assert np.isfinite(m).all() and (m[0, 0] > 0).all()
    assert m[0, 0].sum() > mass0          # post-shock gas flows in from the left and the floor


def test_modification_in_L_only_variant(orc):
    """The oracle's mod_in_L_only switch (the modified first moments serve L
    only; the Runge-Kutta combination takes the stage states as they entered):
    a step equals three right-hand sides combined with the unmodified states;
    it equals the default step when no cell is troubled and differs when some
    are."""
    p = W.four_quadrant_2d(24, seed=2, ny=20)
    kw = dict(dx=p.dx, dy=p.dy, bc=p.bc)
    dt = 0.2 * orc.max_dt(orc.make_cfg(2, p.nx, p.ny, **kw), p.m, 0.6)
    cB = orc.make_cfg(2, p.nx, p.ny, mod_in_L_only=True, **kw)
    got, masks, rc = orc.step(cB, p.m, dt)
    assert rc == 0 and masks.sum() > 0
    _, L0, _, _, _ = orc.rhs(cB, p.m)
    U1 = p.m + dt * L0
    _, L1, _, _, _ = orc.rhs(cB, U1)
    U2 = 0.75 * p.m + 0.25 * U1 + 0.25 * dt * L1
    _, L2, _, _, _ = orc.rhs(cB, U2)
    want = p.m / 3.0 + 2.0 / 3.0 * U2 + 2.0 / 3.0 * dt * L2
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-13 * np.abs(want).max())
    default, _, _ = orc.step(orc.make_cfg(2, p.nx, p.ny, **kw), p.m, dt)
    assert np.abs(default - got).max() > 1e-8
    a, _, _ = orc.step(orc.make_cfg(2, p.nx, p.ny, indicator="none", mod_in_L_only=True, **kw), p.m, dt)
    b, _, _ = orc.step(orc.make_cfg(2, p.nx, p.ny, indicator="none", **kw), p.m, dt)
    np.testing.assert_array_equal(a, b)


def test_double_mach_initial_data():
    """The Example 3.9 input: total mass against the exact area left of the
    shock line x = 1/6 + y/sqrt(3) (area 1/6 + 1/(2 sqrt 3) of [0,4] x [0,1]),
    the two states far from the line, the post-shock state's Mach 10 shock
    relation (mass flux continuity across a shock moving at speed 10 normal to
    itself), and the top segment's trace at the ghost centre height."""
    ny = 50
    p = W.double_mach_2d(ny)
    s3 = math.sqrt(3.0)
    area_left = 1.0 / 6.0 + 1.0 / (2.0 * s3)
    mass = p.m[0, 0].sum() * p.dx * p.dy
    exact = 8.0 * area_left + 1.4 * (4.0 - area_left)
    assert abs(mass - exact) < 1e-3 * exact
    assert abs(p.m[0, 0, 10, 0] - 8.0) < 1e-12 and abs(p.m[0, 0, 10, -1] - 1.4) < 1e-12
    post = p.fixed[0]["b"]
    rho, un = post[0], (post[1] * s3 / 2.0 - post[2] * 0.5) / post[0]      # velocity normal to the shock
    assert abs(rho * (10.0 - un) - 1.4 * 10.0) < 1e-9 * 14.0             # mass flux in the shock frame
    top = p.fixed[3]
    assert top["c0"] == pytest.approx(1.0 / 6.0 + (1.0 + 0.5 / ny) / s3, rel=1e-15)
    assert top["speed"] == pytest.approx(20.0 / s3, rel=1e-15)
