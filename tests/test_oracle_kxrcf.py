"""Hand-computed values of the KXRCF indicator (eq. (KXRCF) with eq.
(line-integral-average) in 1D, eq. (KXRCF_) with eq. (line-integral-average_)
in 2D; Remarks 2 and 3) on the oracle.

The inputs are piecewise-constant Euler states (zero first moments) whose
density jumps between whole cells.  A cell whose three-cell stencil is constant
reconstructs that constant exactly; a cell next to the jump reconstructs its
own average up to the small nonlinear weights of the higher levels (the
smoothness indicator of the one-sided difference vanishes, so the first level
takes the weight), a few 1e-7 here.  The point values on each side of the jump
are therefore its two averages, and the indicator of a cell follows by hand:

    1D:  aleph = |sum over inflow faces of (own trace - neighbour's trace)| / (h^2 ||rho||)
    2D:  aleph = |sum over inflow faces of sum_l len w_l (own - neighbour)| / |dI-| / (h^2 ||rho||)

with h^{(l+1)/3} = h^2 for l = 5, ||rho|| the largest |point value| of the
cell, |dI-| the summed length of the inflow faces, and a face inflow when the
velocity averaged over both sides points into the cell.  Each case is chosen so
that a plausible slip gives a different number: the outflow face in place of
the inflow face, h in place of h^2, no division by |dI-|, counting only the
faces that carry a jump, the neighbour's norm in place of the cell's own.
"""
from __future__ import annotations

import numpy as np
import pytest

from paper_2201_12193_gb300 import workloads as W

GAMMA = 1.4
REL = 1e-5          # the near-constant reconstructions differ from the averages by ~1e-7


def _euler_1d(rho, mu, p):
    n = len(rho)
    m = np.zeros((3, 2, 1, n))
    m[:, 0, 0] = W.prim_to_cons_1d(np.asarray(rho, float), np.asarray(mu, float), np.asarray(p, float))
    return m


def _aleph_1d(orc, m):
    n = m.shape[-1]
    cfg = orc.make_cfg(1, n, dx=1.0 / n, eq="euler", bc=("transmissive",) * 4)
    _, _, mask, aleph, rc = orc.rhs(cfg, m)
    assert rc == 0
    return aleph, mask


N1 = 40
H1 = 1.0 / N1


def _step_1d(mu):
    rho = np.where(np.arange(N1) < 20, 1.0, 2.0)
    return _euler_1d(rho, np.full(N1, mu), np.ones(N1))


@pytest.mark.parametrize("mu", [0.5, 1e-9], ids=["mu_0.5", "mu_1e-9_still_inflow"])
def test_1d_step_flow_to_the_right(orc, mu):
    """Density 1 | 2 between cells 19 and 20, velocity mu > 0: each cell's inflow
    face is its left face.  Cell 20 sees the jump there: aleph = |2 - 1| / (h^2 * 2)
    = 800 (its own norm 2).  Cell 19's left neighbour is its own constant: ~0.
    A velocity of 1e-9 is still inflow (the indicator's dead band is 1e-12)."""
    aleph, mask = _aleph_1d(orc, _step_1d(mu))
    want = abs(2.0 - 1.0) / (H1 ** 2 * 2.0)
    assert want == pytest.approx(800.0)
    assert aleph[20] == pytest.approx(want, rel=REL)
    assert aleph[19] < 1e-2
    assert np.all(aleph[:18] == 0.0) and np.all(aleph[23:] == 0.0)
    assert mask[20] == 1 and mask[19] == 0


def test_1d_step_flow_to_the_left(orc):
    """Velocity -0.5: the inflow face is the right face.  Cell 19 sees the jump:
    aleph = |1 - 2| / (h^2 * 1) = 1600 (its own norm 1); cell 20: ~0."""
    aleph, mask = _aleph_1d(orc, _step_1d(-0.5))
    assert aleph[19] == pytest.approx(1.0 / H1 ** 2, rel=REL)
    assert aleph[20] < 1e-2
    assert mask[19] == 1 and mask[20] == 0


def test_1d_step_at_rest_has_no_inflow_face(orc):
    """A density jump in gas at rest: no face is inflow, aleph = 0 everywhere."""
    aleph, mask = _aleph_1d(orc, _step_1d(0.0))
    assert np.all(aleph == 0.0) and mask.sum() == 0


def test_1d_two_inflow_faces_add_without_division(orc):
    """A one-cell density spike 2 in gas 1, converging flow (+0.5 left of it,
    -0.5 right of it, 0 inside): both faces of the spike are inflow and eq.
    (line-integral-average) adds the two signed jumps (2 - 1) + (2 - 1) with no
    division: aleph = 2 / (h^2 * 2) = 1600 (one face alone, or a division by
    the two faces, would give 800)."""
    rho = np.ones(N1)
    rho[20] = 2.0
    mu = np.where(np.arange(N1) < 20, 0.5, -0.5)
    mu[20] = 0.0
    aleph, mask = _aleph_1d(orc, _euler_1d(rho, mu, np.ones(N1)))
    assert aleph[20] == pytest.approx(2.0 / (H1 ** 2 * 2.0), rel=REL)
    assert mask[20] == 1


N2 = 16
H2 = 1.0 / N2


def _aleph_2d(orc, rho, mu, nu):
    n = N2
    m = np.zeros((4, 3, n, n))
    m[:, 0] = W.prim_to_cons_2d(rho, mu, nu, np.ones((n, n)))
    cfg = orc.make_cfg(2, n, n, dx=H2, dy=H2, eq="euler", bc=("transmissive",) * 4)
    _, _, mask, aleph, rc = orc.rhs(cfg, m)
    assert rc == 0
    return aleph.reshape(n, n), mask.reshape(n, n)


def _xstep():
    i = np.arange(N2)[None, :].repeat(N2, 0)
    return np.where(i < 8, 1.0, 2.0)           # rho[j, i]: 1 left of x = 1/2, 2 right of it


def test_2d_two_inflow_faces_one_jump(orc):
    """Density 1 | 2 across x = 1/2, uniform along y, velocity (0.5, 0.5): the
    left and bottom faces are inflow.  Along the left face of the first column
    of 2 the jump is 1 at every Gauss-Lobatto point (weights summing to 1), along
    the bottom face 0:  aleph = |dy * 1 + dx * 0| / (dx + dy) / (h^2 * 2)
    = 1 / (4 h^2) = 64.  No division by |dI-| would give 8; dividing by the
    jumping face alone, 128."""
    aleph, mask = _aleph_2d(orc, _xstep(), np.full((N2, N2), 0.5), np.full((N2, N2), 0.5))
    want = (H2 * 1.0) / (H2 + H2) / (H2 ** 2 * 2.0)
    assert want == pytest.approx(64.0)
    np.testing.assert_allclose(aleph[:, 8], want, rtol=REL)
    assert np.all(aleph[:, 7] < 1e-2)
    assert np.all(aleph[:, :6] == 0.0) and np.all(aleph[:, 11:] == 0.0)
    assert np.all(mask[:, 8] == 1) and np.all(mask[:, 7] == 0)


def test_2d_inflow_from_the_right_and_the_top(orc):
    """The same step with velocity (-0.5, -0.5): inflow through the right and top
    faces; the last column of 1 sees the jump: aleph = dy * 1 / (dx + dy) /
    (h^2 * 1) = 128, the first column of 2 sees none."""
    aleph, mask = _aleph_2d(orc, _xstep(), np.full((N2, N2), -0.5), np.full((N2, N2), -0.5))
    np.testing.assert_allclose(aleph[:, 7], 1.0 / (2.0 * H2 ** 2), rtol=REL)
    assert np.all(aleph[:, 8] < 1e-2)
    assert np.all(mask[:, 7] == 1) and np.all(mask[:, 8] == 0)


def test_2d_single_inflow_face(orc):
    """Velocity (0.5, 0) (the y velocity inside the dead band): only the left face
    is inflow, |dI-| = dy: aleph = 1 / (h^2 * 2) = 128."""
    aleph, _ = _aleph_2d(orc, _xstep(), np.full((N2, N2), 0.5), np.zeros((N2, N2)))
    np.testing.assert_allclose(aleph[:, 8], 1.0 / (2.0 * H2 ** 2), rtol=REL)


def test_2d_at_rest(orc):
    aleph, mask = _aleph_2d(orc, _xstep(), np.zeros((N2, N2)), np.zeros((N2, N2)))
    assert np.all(aleph == 0.0) and mask.sum() == 0


# ---------------------------------------------------------------- the norm over all the cell's points
# ||rho|| in eq. (KXRCF) / (KXRCF_) is the largest |point value| over all the
# cell's Gauss-Lobatto points, the interior ones included.  On point values
# chosen by hand (the oracle's test entry takes them in place of the
# reconstruction's), a cell whose density peaks at its interior points tells
# that norm from one over the boundary points only.

def test_norm_counts_the_interior_points_1d():
    """1D, flow to the right (u = 1 everywhere): the left face is the inflow face,
    the jump there is 1 - 1.5; the cell's points are (1, 3, 3, 1), so
    aleph = 0.5 / (h^2 * 3), not 0.5 / (h^2 * 1)."""
    from oracle import kxrcf_aleph, make_cfg
    h = 0.1
    cfg = make_cfg(1, 3, dx=h, eq="euler", bc=("periodic",) * 4)
    G = np.zeros((3, 3, 4))
    rho = np.ones((3, 4))
    rho[1] = (1.0, 3.0, 3.0, 1.0)
    rho[0, 3] = 1.5
    G[:, 0, :] = rho
    G[:, 1, :] = rho          # momentum = rho: velocity 1
    G[:, 2, :] = 2.5 + 0.5 * rho
    assert kxrcf_aleph(cfg, G, 1) == pytest.approx(0.5 / (h * h * 3.0), rel=1e-13)


def test_norm_counts_the_interior_points_2d():
    """2D, flow along +x (u = 1, v = 0): only the left face is inflow, with the
    jump 1 - 1.5 at every point of it; the cell's density is 3 at its four
    interior points and 1 at the twelve boundary points, so
    aleph = |dy * (-0.5)| / dy / (h^2 * 3)."""
    from oracle import kxrcf_aleph, make_cfg
    h = 0.1
    cfg = make_cfg(2, 3, 3, dx=h, dy=h, eq="euler", bc=("periodic",) * 4)
    rho = np.ones((3, 3, 4, 4))               # [j][i][k][l]
    rho[1, 1, 1:3, 1:3] = 3.0
    rho[1, 0, 3, :] = 1.5                     # the left neighbour's trace on the shared face
    G = np.zeros((3, 3, 4, 4, 4))
    G[:, :, 0] = rho
    G[:, :, 1] = rho                          # x momentum = rho: u = 1
    G[:, :, 3] = 2.5 + 0.5 * rho
    assert kxrcf_aleph(cfg, G, 1, 1) == pytest.approx(0.5 / (h * h * 3.0), rel=1e-13)
