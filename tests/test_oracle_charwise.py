"""CPU pins of the characteristic-wise reconstruction option (1D Euler).

* A contact discontinuity (density jump, velocity and pressure constant) lives
  in one characteristic field only: projected on the fields, the other two are
  constant across the stencil, so velocity and pressure stay exactly constant
  at the Gauss-Lobatto points and L of momentum and energy are u0 and u0^2/2
  times L of density.  Component-wise reconstruction does not have this.
* A constant state is steady.
* The interacting blast waves (Example 3.7) run to t = 0.038 with the density
  peak of the problem's known solution (about 6, near x = 0.78); component-wise
  they lose positivity at the collision (t ~ 0.028).
"""
from __future__ import annotations

import numpy as np
import pytest

from paper_2201_12193_gb300 import workloads as W


def _contact(n, u0=0.7, p0=2.0):
    x = (np.arange(n) + 0.5) / n
    rho = np.where(np.abs(x - 0.5) < 0.2, 3.0, 1.0) + 0.3 * np.sin(6 * x)
    m = np.zeros((3, 2, 1, n))
    m[:, 0, 0] = W.prim_to_cons_1d(rho, np.full(n, u0), np.full(n, p0))
    return m, u0


def test_contact_keeps_velocity_and_pressure(orc):
    n = 60
    m, u0 = _contact(n)
    dev = {}
    for cw in (True, False):
        cfg = orc.make_cfg(1, n, dx=1.0 / n, eq="euler", bc=("periodic",) * 4, indicator="none", charwise=cw)
        _, L, _, _, rc = orc.rhs(cfg, m)
        assert rc == 0
        scale = np.abs(L[0]).max()
        dev[cw] = max(np.abs(L[1] - u0 * L[0]).max(), np.abs(L[2] - 0.5 * u0 * u0 * L[0]).max()) / scale
    assert dev[True] <= 1e-12, dev
    assert dev[False] > 1e-8, dev


def test_constant_state_is_steady_charwise(orc):
    n = 16
    m = np.zeros((3, 2, 1, n))
    m[:, 0, 0] = np.array(W.prim_to_cons_1d(np.full(n, 1.3), np.full(n, -0.4), np.full(n, 0.9)))
    cfg = orc.make_cfg(1, n, dx=1.0 / n, eq="euler", bc=("periodic",) * 4, charwise=True)
    _, L, mk, _, rc = orc.rhs(cfg, m)
    assert rc == 0 and mk.sum() == 0 and np.abs(L).max() <= 1e-12


def test_blast_waves_run_through_with_characteristic_reconstruction(orc):
    n = 400
    p = W.blast_wave_1d(n)
    cfg = orc.make_cfg(1, n, dx=p.dx, eq="euler", bc=p.bc, charwise=True)
    m, t = p.m.copy(), 0.0
    mass0 = m[0, 0].sum()
    while t < p.t_end - 1e-14:
        dt = min(orc.max_dt(cfg, m, 0.6), p.t_end - t)
        m, _, rc = orc.step(cfg, m, dt)
        assert rc == 0 and (m[0, 0] > 0).all()
        t += dt
    rho = m[0, 0, 0]
    assert 5.5 < rho.max() < 6.5 and 0.74 < (np.argmax(rho) + 0.5) / n < 0.80
    assert abs(m[0, 0].sum() - mass0) <= 1e-12 * mass0          # walls: no mass leaves


def test_eigenvectors_diagonalise_the_flux_jacobian(orc):
    """L R = I, and R diag(u - c, u, u + c) L equals the Jacobian of the oracle's
    own 1D Euler flux by central differences (states at rest, subsonic and
    supersonic, either direction)."""
    cfg = orc.make_cfg(1, 8, eq="euler")
    g = 1.4
    for rho, mu, p in ((1.0, 0.0, 1.0), (0.3, 0.7, 2.0), (5.0, -3.1, 0.4), (1.2, 4.0, 0.1)):
        u = np.array(W.prim_to_cons_1d(np.array(rho), np.array(mu), np.array(p)), dtype=np.float64)
        R, L = orc.euler1d_eig(g, u)
        np.testing.assert_allclose(L @ R, np.eye(3), atol=1e-13)
        c = np.sqrt(g * p / rho)
        A = R @ np.diag([mu - c, mu, mu + c]) @ L
        J = np.empty((3, 3))
        for k in range(3):
            h = 1e-6 * max(1.0, abs(u[k]))
            up, um = u.copy(), u.copy()
            up[k] += h
            um[k] -= h
            J[:, k] = (orc.phys_flux(cfg, up) - orc.phys_flux(cfg, um)) / (2 * h)
        np.testing.assert_allclose(A, J, rtol=1e-7, atol=1e-7 * np.abs(J).max())


@pytest.mark.parametrize("name", ["sod", "lax"])
def test_charwise_shock_tubes_converge_to_exact_riemann(orc, name):
    """The characteristic-wise option against the exact Riemann solution: the
    density L1 error falls under refinement and stays within 1.25x of the
    component-wise default's (the option changes how systems are reconstructed,
    not the scheme's resolution)."""
    import exact
    errs = {}
    for cw in (True, False):
        e = []
        for n in (100, 200):
            p = W.sod_1d(n) if name == "sod" else W.lax_1d(n)
            cfg = orc.make_cfg(1, n, dx=p.dx, eq="euler", bc=p.bc, charwise=cw)
            m, _ = orc.run(cfg, p.m, p.t_end)
            assert np.all(np.isfinite(m))
            ex = exact.riemann_density_averages(p.meta["left"], p.meta["right"], p.x0, p.x1, n,
                                                p.meta["xs"], p.t_end)
            e.append(np.abs(m[0, 0, 0] - ex).mean())
        errs[cw] = e
    assert errs[True][1] < 0.85 * errs[True][0], errs
    assert errs[True][1] < 1.25 * errs[False][1], errs


def test_modification_in_L_only_runs_the_blast_waves_through(orc):
    """Component-wise, Example 3.7 stops at the collision (t ~ 0.028) when the
    modified first moments persist in the state (the default reading), and runs
    to t = 0.038 with them used inside L only (mod_in_L_only)."""
    p = W.blast_wave_1d(400)
    reached = {}
    for b in (False, True):
        cfg = orc.make_cfg(1, 400, dx=p.dx, eq="euler", bc=p.bc, mod_in_L_only=b)
        m, t = p.m.copy(), 0.0
        while t < p.t_end - 1e-14:
            dt = min(orc.max_dt(cfg, m, 0.6), p.t_end - t)
            if not (np.isfinite(dt) and dt > 0):
                break
            m, _, rc = orc.step(cfg, m, dt)
            if rc != 0:
                break
            t += dt
        reached[b] = t
    assert reached[False] < 0.03 and reached[True] == pytest.approx(p.t_end, rel=1e-12), reached
