"""CPU pins of the reflective-wall boundary (a solid wall: the transmissive
mirror with the wall-normal momentum negated) in the oracle.

* No mass and no energy cross a wall: the cell sums of L for rho and E vanish
  to rounding with walls on every side (they do not with transmissive sides).
* A wall is a symmetry plane: a mirror-symmetric problem on [0, 1] with walls
  equals, on [0, 1/2], the half problem with a wall at 1/2 (one step, 1D and 2D).
"""
from __future__ import annotations

import numpy as np

from paper_2201_12193_gb300 import workloads as W


def _state_1d(n, rng):
    x = (np.arange(n) + 0.5) / n
    rho = 1.0 + 0.3 * rng.random(n)
    mu = 0.5 * rng.standard_normal(n)
    p = 1.0 + rng.random(n)
    m = np.zeros((3, 2, 1, n))
    m[:, 0, 0] = W.prim_to_cons_1d(rho, mu, p)
    m[:, 1, 0] = 0.02 * rng.standard_normal((3, n))
    return m


def test_no_mass_or_energy_through_walls_1d(orc):
    rng = np.random.default_rng(1)
    n = 40
    m = _state_1d(n, rng)
    for bc, zero in (("reflective", True), ("transmissive", False)):
        cfg = orc.make_cfg(1, n, dx=1.0 / n, eq="euler", bc=(bc,) * 4)
        _, L, _, _, rc = orc.rhs(cfg, m)
        assert rc == 0
        for v in (0, 2):
            tot, scale = L[v, 0].sum(), np.abs(L[v, 0]).sum()
            if zero:
                assert abs(tot) <= 1e-13 * scale, (v, tot, scale)
            else:
                assert abs(tot) > 1e-6 * scale


def test_no_mass_or_energy_through_walls_2d(orc):
    p = W.walled_blast_2d(24, seed=3, ncircles=2)
    rng = np.random.default_rng(2)
    m = p.m.copy()
    m[1:3, 0] += 0.1 * rng.standard_normal(m[1:3, 0].shape)        # moving fluid everywhere
    m[:, 1:] += 1e-3 * rng.standard_normal(m[:, 1:].shape)
    cfg = orc.make_cfg(2, p.nx, p.ny, dx=p.dx, dy=p.dy, eq="euler", bc=p.bc)
    _, L, _, _, rc = orc.rhs(cfg, m)
    assert rc == 0
    for v in (0, 3):
        assert abs(L[v, 0].sum()) <= 1e-13 * np.abs(L[v, 0]).sum()


def _mirror_1d(half):
    """Extend a state on [0, 1/2] to its mirror image on [0, 1] about x = 1/2."""
    full = np.concatenate([half, half[..., ::-1]], axis=-1)
    n = half.shape[-1]
    full[1, 0, :, n:] *= -1.0            # momentum average: antisymmetric
    full[0, 1, :, n:] *= -1.0            # first moments of rho and E: antisymmetric
    full[2, 1, :, n:] *= -1.0
    return full


def test_wall_is_a_symmetry_plane_1d(orc):
    rng = np.random.default_rng(4)
    n = 50
    half = _state_1d(n, rng)
    full = _mirror_1d(half)
    c_half = orc.make_cfg(1, n, dx=0.5 / n, eq="euler", bc=("reflective",) * 4)
    c_full = orc.make_cfg(1, 2 * n, dx=0.5 / n, eq="euler", bc=("reflective",) * 4)
    dt = 0.5 * orc.max_dt(c_full, full, 0.6)
    h, mh, rc1 = orc.step(c_half, half, dt)
    f, mf, rc2 = orc.step(c_full, full, dt)
    assert rc1 == 0 and rc2 == 0
    np.testing.assert_allclose(f[..., :n], h, rtol=0, atol=1e-12 * np.abs(h).max())
    assert np.array_equal(mf[:, :n], mh)


def _contact_state_2d(nx, ny, rng):
    """A density jump (a contact, KXRCF active) over smooth pressure and velocity."""
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / nx
    X, Y = np.meshgrid(x, y)
    rho = 1.0 + 0.5 * (X > 0.4) + 0.1 * np.sin(3 * Y)
    u = 0.2 * np.cos(2 * X) + 0.05 * Y
    v = 0.1 * np.sin(4 * X) * (1 + Y)
    p = 1.0 + 0.2 * np.cos(3 * X + Y)
    m = np.zeros((4, 3, ny, nx))
    m[:, 0] = W.prim_to_cons_2d(rho, u, v, p)
    m[:, 1:] = 1e-3 * rng.standard_normal(m[:, 1:].shape)
    return m


def test_wall_is_a_symmetry_plane_2d(orc):
    """Mirror in y about y = 1/2: the half box with a wall at the top."""
    rng = np.random.default_rng(6)
    half = _contact_state_2d(16, 8, rng)
    p = W.walled_blast_2d(16, seed=5, ncircles=2)     # grid spacing only
    full = np.concatenate([half, half[:, :, ::-1, :]], axis=2)
    full[2, 0, 8:] *= -1.0               # y momentum: antisymmetric
    for v in (0, 1, 3):
        full[v, 2, 8:] *= -1.0           # y first moments of the symmetric variables
    full[2, 1, 8:] *= -1.0               # x first moment of the y momentum: antisymmetric
    bc = ("transmissive", "transmissive", "reflective", "reflective")
    c_half = orc.make_cfg(2, 16, 8, dx=p.dx, dy=p.dy, eq="euler", bc=bc)
    c_full = orc.make_cfg(2, 16, 16, dx=p.dx, dy=p.dy, eq="euler", bc=bc)
    dt = 0.5 * orc.max_dt(c_full, full, 0.6)
    h, mh, rc1 = orc.step(c_half, half, dt)
    f, mf, rc2 = orc.step(c_full, full, dt)
    assert rc1 == 0 and rc2 == 0
    assert mh.sum() > 0                  # the indicator takes part
    np.testing.assert_allclose(f[:, :, :8], h, rtol=0, atol=1e-12 * np.abs(h).max())
    assert np.array_equal(mf.reshape(3, 16, 16)[:, :8], mh.reshape(3, 8, 16))


def _mirror(A, axis):
    """Mirror a 2D Euler state (or its L) in x (axis 'x') or y: reverse the cells,
    negate the first moment along the axis, and the momentum component along it
    (whose moment along the axis therefore keeps its sign)."""
    s = (A[:, :, :, ::-1] if axis == "x" else A[:, :, ::-1, :]).copy()
    mom, mvar = (1, 1) if axis == "x" else (2, 2)
    for v in range(4):
        if v == mvar:
            s[v, 0] *= -1.0
            s[v, 3 - mom] *= -1.0
        else:
            s[v, mom] *= -1.0
    return s


def test_2d_operator_is_mirror_equivariant(orc):
    """L(mirror U) = mirror L(U) in x and in y, on discontinuous four-quadrant
    data with KXRCF active: catches a sign or index slip in any direction."""
    for seed in range(2):
        p = W.four_quadrant_2d(24, seed=seed)
        rng = np.random.default_rng(seed)
        A = p.m.copy()
        A[:, 1:] += 1e-3 * rng.standard_normal(A[:, 1:].shape)
        c = orc.make_cfg(2, 24, 24, dx=p.dx, dy=p.dy, eq="euler", bc=("transmissive",) * 4)
        _, L, mk, _, rc = orc.rhs(c, A)
        assert rc == 0 and mk.sum() > 0
        for axis in ("x", "y"):
            _, Lm, mkm, _, _ = orc.rhs(c, _mirror(A, axis))
            np.testing.assert_allclose(Lm, _mirror(L, axis), rtol=0, atol=1e-12 * np.abs(L).max())
            mk2 = mk.reshape(24, 24)
            assert np.array_equal(mkm.reshape(24, 24), mk2[:, ::-1] if axis == "x" else mk2[::-1, :])


# ------------------------------------------------------------------ TVB indicator (Remark 2)
# Reading: the TVB test acts on the cell's linear polynomial of its moments,
# whose face deviation is a = 6 vbar; troubled when the modified minmod
# (identity for |a| <= M h^2) changes a against the neighbour differences.

def _euler_1d_lin(n, slope, vbar_scale=1.0):
    """rho = 1 + slope x with its exact first moments (times vbar_scale)."""
    x = (np.arange(n) + 0.5) / n
    m = np.zeros((3, 2, 1, n))
    rho = 1.0 + slope * x
    m[:, 0, 0] = W.prim_to_cons_1d(rho, np.full(n, 0.3), np.ones(n))
    m[0, 1, 0] = vbar_scale * slope / n / 12.0          # vbar of a linear function: slope dx / 12
    return m


def test_tvb_indicator_pins(orc):
    n = 40
    cfg = lambda M: orc.make_cfg(1, n, dx=1.0 / n, eq="euler", bc=("periodic",) * 4, indicator="tvb", tvb_m=M)
    interior = slice(2, n - 2)
    # consistent linear data: a = half the neighbour differences, same sign: not troubled
    _, _, mk, _, rc = orc.rhs(cfg(0.0), _euler_1d_lin(n, 0.5))
    assert rc == 0 and mk[interior].sum() == 0
    # first moments three times too steep: a = 1.5 x the differences, changed by the minmod
    _, _, mk, _, _ = orc.rhs(cfg(0.0), _euler_1d_lin(n, 0.5, 3.0))
    assert mk[interior].all()
    # ... unless M h^2 exceeds |a|
    _, _, mk, _, _ = orc.rhs(cfg(1e6), _euler_1d_lin(n, 0.5, 3.0))
    assert mk.sum() == 0
    # a first moment against the trend of the averages: minmod 0
    _, _, mk, _, _ = orc.rhs(cfg(0.0), _euler_1d_lin(n, 0.5, -1.0))
    assert mk[interior].all()


def test_tvb_indicator_2d_sees_both_directions(orc):
    """The x first moment triggers it through x differences, the y first moment
    through y differences."""
    n = 16
    x = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(x, x)
    for axis, mom in (("x", 1), ("y", 2)):
        rho = 1.0 + 0.5 * (X if axis == "x" else Y)
        m = np.zeros((4, 3, n, n))
        m[:, 0] = W.prim_to_cons_2d(rho, np.full_like(rho, 0.2), np.full_like(rho, 0.1), np.ones_like(rho))
        c = orc.make_cfg(2, n, n, dx=1.0 / n, dy=1.0 / n, eq="euler", bc=("periodic",) * 4, indicator="tvb",
                         tvb_m=0.0)
        m[0, mom] = 0.5 / n / 12.0                        # consistent: not troubled
        _, _, mk, _, rc = orc.rhs(c, m)
        inner = mk.reshape(n, n)[2:-2, 2:-2]
        assert rc == 0 and inner.sum() == 0
        m[0, mom] *= 3.0                                  # too steep in that direction: troubled
        _, _, mk, _, _ = orc.rhs(c, m)
        assert mk.reshape(n, n)[2:-2, 2:-2].all()
