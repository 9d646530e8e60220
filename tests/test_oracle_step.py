"""The solid block of the forward-facing step (Sec. 3, Example 3.10) in the
oracle, pinned against the reflective sides it generalises and against the
conservation a wall implies.

* A block over the full height, from column i0 on, is a wall at x = i0 dx:
  the operator on the fluid columns equals that of the narrower grid with a
  reflective right side (pinned in test_oracle_walls.py as a symmetry plane).
* A block over the full width, below row j1, is a wall at y = j1 dy: the
  operator on the fluid rows equals that of the shorter grid with a
  reflective bottom side.
* A closed box with a step: no mass and no energy cross the block's faces or
  its corner (cell sums of L over the fluid vanish to rounding); gas at rest
  in uniform pressure stays at rest; solid cells are never flagged, never
  updated and take no part in the CFL rule or the totals.
"""
from __future__ import annotations

import numpy as np
import pytest

from paper_2201_12193_gb300 import workloads as W


def _state(nx, ny, seed, h):
    """A smooth seeded 2D Euler state with moments (density, velocities,
    pressure positive) and small first moments."""
    rng = np.random.default_rng(seed)
    x = (np.arange(nx) + 0.5) * h
    y = (np.arange(ny) + 0.5) * h
    X, Y = np.meshgrid(x, y)
    a = rng.uniform(0.5, 1.5, 6)
    rho = 1.0 + 0.3 * np.sin(2 * np.pi * (a[0] * X + a[1] * Y)) ** 2
    u = 0.4 * np.cos(2 * np.pi * (a[2] * X - 0.3 * Y))
    v = 0.3 * np.sin(2 * np.pi * (a[3] * Y + 0.2 * X))
    p = 1.0 + 0.2 * np.cos(2 * np.pi * a[4] * (X + Y))
    m = np.zeros((4, 3, ny, nx))
    m[:, 0] = W.prim_to_cons_2d(rho, u, v, p)
    m[:, 1:] = 0.02 * rng.standard_normal((4, 2, ny, nx)) * np.abs(m[:, :1])
    return m


def test_full_height_block_is_a_right_wall(orc):
    nx, ny, i0, h = 20, 10, 12, 0.1
    m = _state(nx, ny, 1, h)
    step = orc.make_cfg(2, nx, ny, dx=h, dy=h, bc=("transmissive", "transmissive", "reflective", "reflective"),
                        solid=(i0, ny))
    wall = orc.make_cfg(2, i0, ny, dx=h, dy=h, bc=("transmissive", "reflective", "reflective", "reflective"))
    for ind in ("kxrcf", "all", "none"):
        step.indicator = wall.indicator = {"none": 0, "kxrcf": 1, "all": 2}[ind]
        Um1, L1, k1, a1, rc1 = orc.rhs(step, m)
        Um2, L2, k2, a2, rc2 = orc.rhs(wall, np.ascontiguousarray(m[:, :, :, :i0]))
        assert rc1 == 0 and rc2 == 0
        np.testing.assert_allclose(L1[:, :, :, :i0], L2, rtol=0, atol=1e-12 * np.abs(L2).max())
        np.testing.assert_array_equal(k1.reshape(ny, nx)[:, :i0].ravel(), k2)
        assert not L1[:, :, :, i0:].any() and not k1.reshape(ny, nx)[:, i0:].any()


def test_full_width_block_is_a_bottom_wall(orc):
    nx, ny, j1, h = 10, 16, 6, 0.1
    m = _state(nx, ny, 2, h)
    step = orc.make_cfg(2, nx, ny, dx=h, dy=h, bc=("periodic", "periodic", "transmissive", "reflective"),
                        solid=(0, j1))
    wall = orc.make_cfg(2, nx, ny - j1, dx=h, dy=h, bc=("periodic", "periodic", "reflective", "reflective"))
    Um1, L1, k1, _, rc1 = orc.rhs(step, m)
    Um2, L2, k2, _, rc2 = orc.rhs(wall, np.ascontiguousarray(m[:, :, j1:, :]))
    assert rc1 == 0 and rc2 == 0
    np.testing.assert_allclose(L1[:, :, j1:, :], L2, rtol=0, atol=1e-12 * np.abs(L2).max())
    np.testing.assert_array_equal(k1.reshape(ny, nx)[j1:].ravel(), k2)


@pytest.mark.parametrize("indicator", ["kxrcf", "all"])
def test_closed_box_with_a_step_conserves_mass_and_energy(orc, indicator):
    nx, ny, h = 16, 12, 0.1
    sol = (8, 5)
    m = _state(nx, ny, 3, h)
    cfg = orc.make_cfg(2, nx, ny, dx=h, dy=h, bc=("reflective",) * 4, solid=sol, indicator=indicator)
    Um, L, k, _, rc = orc.rhs(cfg, m)
    assert rc == 0
    fluid = np.ones((ny, nx), bool)
    fluid[: sol[1], sol[0]:] = False
    for v in (0, 3):             # mass, energy: only wall fluxes (pressure) at the borders
        s = (L[v, 0] * fluid).sum()
        assert abs(s) <= 1e-12 * np.abs(L[v, 0]).sum(), (v, s)
    assert not k.reshape(ny, nx)[~fluid].any()
    # the corner cell's two fluid neighbours see walls: their own reflections
    dt = 0.2 * orc.max_dt(cfg, m, 0.6)
    m2, masks, rc = orc.step(cfg, m, dt)
    assert rc == 0
    # solid cells are not updated (L = 0 there; the combination only rounds them)
    np.testing.assert_allclose(m2[:, :, ~fluid], m[:, :, ~fluid], rtol=4e-16, atol=0)
    t0, t1 = orc.totals(cfg, m), orc.totals(cfg, m2)
    assert abs(t1[0] - t0[0]) <= 1e-13 * t0[0] and abs(t1[3] - t0[3]) <= 1e-13 * t0[3]


def test_step_at_rest_stays_at_rest_and_solid_cells_are_left_out(orc):
    nx, ny, h = 16, 12, 0.1
    m = np.zeros((4, 3, ny, nx))
    m[:, 0] = np.array(W.prim_to_cons_2d(np.full((ny, nx), 1.4), np.zeros((ny, nx)), np.zeros((ny, nx)),
                                         np.ones((ny, nx))))
    solid = (np.arange(nx)[None, :] >= 9) & (np.arange(ny)[:, None] < 4)
    m[:, 0][:, solid] = 1e9                      # solid cells' own values must never be read
    cfg = orc.make_cfg(2, nx, ny, dx=h, dy=h, bc=("inflow", "transmissive", "reflective", "reflective"),
                       solid=(9, 4), fixed=({"b": tuple(m[:, 0, 6, 0])}, None, None, None))
    _, L, k, _, rc = orc.rhs(cfg, m)
    assert rc == 0 and not k.any()
    assert np.abs(L).max() <= 1e-12
    assert orc.max_dt(cfg, m, 0.6) == pytest.approx(orc.max_dt(cfg, np.where(solid, m[:, :, 6:7, 0:1], m), 0.6))
    tot = orc.totals(cfg, m)
    assert tot[0] == pytest.approx(1.4 * (nx * ny - solid.sum()) * h * h, rel=1e-14)


def test_faces_on_the_block_are_never_inflow_faces(orc):
    """Gas at rest (rho = 1, p = 1) except the cell just above the corner's left
    neighbour, which is denser (rho = 2) and moves right.  Seen from that cell
    (diagonal to the corner) the corner solid cell is its point reflection,
    moving left; seen from the corner's left neighbour it is that neighbour's
    own mirror, at rest: across the step's vertical face the left neighbour
    sees neither a flow into it nor a density jump (a face shared with a solid
    cell is a wall, never an inflow face), so it stays untroubled."""
    nx, ny, h, sol = 16, 12, 0.1, (9, 4)
    rho = np.ones((ny, nx))
    u = np.zeros((ny, nx))
    rho[sol[1], sol[0] - 1] = 2.0
    u[sol[1], sol[0] - 1] = 0.5
    m = np.zeros((4, 3, ny, nx))
    m[:, 0] = W.prim_to_cons_2d(rho, u, np.zeros((ny, nx)), np.ones((ny, nx)))
    cfg = orc.make_cfg(2, nx, ny, dx=h, dy=h, bc=("transmissive", "transmissive", "reflective", "reflective"),
                       solid=sol)
    _, _, k, a, rc = orc.rhs(cfg, m)
    assert rc == 0
    a = a.reshape(ny, nx)
    assert a[sol[1] - 1, sol[0] - 1] < 1e-3 and not k.reshape(ny, nx)[sol[1] - 1, sol[0] - 1]


def test_supersonic_flow_does_not_cross_the_step_face(orc):
    """Mach 3 flow straight into the step's vertical face: the face carries no
    mass and no energy (the cell in front of it keeps only its inflow: L of its
    mass = rho u / dx, of its energy = (E + p) u / dx), although the wave-speed
    estimate of eq. (COEF) would put the whole HLLC fan downstream of the face
    (s_L = 3 - 2.14 > 0) and the first branch of eq. (f_HLLC) would let the
    gas through.  Above the step every cell beyond the corner's column sees
    the block as its own mirror in y, a uniform stencil: its L of the averages
    is exactly zero (an image across the corner's diagonal would break the
    uniformity in the cells next to it)."""
    p = W.forward_step_2d(20)
    i0, j1 = p.meta["solid"]
    cfg = orc.make_cfg(2, p.nx, p.ny, dx=p.dx, dy=p.dy, bc=p.bc, fixed=p.fixed, solid=(i0, j1), indicator="none")
    _, L, _, _, rc = orc.rhs(cfg, p.m)
    assert rc == 0
    rho, u, pr = 1.4, 3.0, 1.0
    E = pr / 0.4 + 0.5 * rho * u * u
    for j in range(j1 - 1):          # below the corner row (its top face is a wall too)
        assert L[0, 0, j, i0 - 1] == pytest.approx(rho * u / p.dx, rel=1e-12)
        assert L[3, 0, j, i0 - 1] == pytest.approx((E + pr) * u / p.dx, rel=1e-12)
    assert np.abs(L[0, 0, j1:, :]).max() < 1e-8     # the uniform flow above the step is steady
    assert not L[:, 0, j1:, i0 + 1:].any()
