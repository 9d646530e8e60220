"""Pins of the CPU FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: values the
paper prints (tests/golden/paper_values.json, each with its citation), closed
forms worked out by hand, exact solutions (tests/exact.py), independent
numerical integration, or invariants of the scheme.  None of these tests
touch the CUDA library.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np
import pytest

import exact
from paper_2201_12193_gb300 import workloads as W

GBAR = (1.0, 10.0, 100.0, 1000.0)
XG, WG = np.polynomial.legendre.leggauss(10)
XG, WG = 0.5 * XG, 0.5 * WG          # on [-1/2, 1/2], weights sum to 1


def frac(s):
    return float(Fraction(s))


def golden_nodes(golden):
    out = []
    for s in golden["gauss_lobatto"]["nodes_xi"]:
        sgn = -1.0 if s.startswith("-") else 1.0
        out.append(sgn * math.sqrt(5.0) / 10.0 if "sqrt" in s else frac(s))
    return np.array(out)


# ------------------------------------------------------------- helpers

def poly1_moments(c):
    """1D data (ubar_{-1,0,1}, vbar_{-1,0,1}) of P(xi) = sum c[a] xi^a by quadrature."""
    P = np.polynomial.polynomial.Polynomial(c)
    ub, vb = [], []
    for o in (-1, 0, 1):
        x = o + XG
        ub.append(np.sum(WG * P(x)))
        vb.append(np.sum(WG * P(x) * (x - o)))
    return np.array(ub + vb)


def poly2_eval(c, x, y):
    s = 0.0
    for a in range(6):
        for b in range(6 - a):
            s = s + c[a, b] * x ** a * y ** b
    return s


def poly2_moments(c):
    """2D data (ubar[9], vbar[9], wbar[9]) in paper label order (bottom row first)."""
    ub, vb, wb = [], [], []
    for oy in (-1, 0, 1):
        for ox in (-1, 0, 1):
            X = ox + XG[:, None]
            Y = oy + XG[None, :]
            w2 = WG[:, None] * WG[None, :]
            P = poly2_eval(c, X, Y)
            ub.append(np.sum(w2 * P))
            vb.append(np.sum(w2 * P * (X - ox)))
            wb.append(np.sum(w2 * P * (Y - oy)))
    return np.array(ub + vb + wb)


def rand_poly2(rng, deg):
    c = np.zeros((6, 6))
    for a in range(deg + 1):
        for b in range(deg + 1 - a):
            c[a, b] = rng.standard_normal()
    return c


# ------------------------------------------------------------- printed constants

def test_modification_constants_match_eq_vi(orc, golden):
    want = [frac(s) for s in golden["modification_vi"]["weights_ubar_im1_ubar_i_ubar_ip1_vbar_im1_vbar_ip1"]]
    got = orc.modification_weights()
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-15)


@pytest.mark.parametrize("dim", [1, 2])
def test_p_from_q_matches_eq_pq(orc, golden, dim):
    rng = np.random.default_rng(1)
    data = rng.standard_normal(6 if dim == 1 else 27)
    q = {l: orc.poly(dim, l, data, "q") for l in (1, 2, 3, 4)}
    for l in (2, 3, 4):
        row = golden["pq_relations"][f"p{l}"]
        want = frac(row[f"q{l}"]) * q[l] + frac(row[f"q{l - 1}"]) * q[l - 1]
        np.testing.assert_allclose(orc.poly(dim, l, data, "p"), want, atol=1e-12, rtol=1e-13)


@pytest.mark.parametrize("dim", [1, 2])
@pytest.mark.parametrize("gbar", [(1.0, 10.0, 100.0, 1000.0), (1.0, 1.0, 1.0, 1.0), (1.0, 2.0, 4.0, 8.0),
                                  (3.0, 0.5, 7.0, 2.0)])
def test_linear_weight_polynomial_is_q4(orc, dim, gbar):
    """sum_l gamma_{l,4} p_l == q_4 for any positive linear weights (eq. (p) inverted)."""
    rng = np.random.default_rng(2)
    data = rng.standard_normal(6 if dim == 1 else 27)
    np.testing.assert_allclose(orc.poly(dim, 4, data, "lin", gbar), orc.poly(dim, 4, data, "q"),
                               atol=1e-12, rtol=1e-12)


# ------------------------------------------------------------- reproduction

@pytest.mark.parametrize("level,deg", [(2, 2), (3, 3), (4, 5)])
def test_reproduction_1d(orc, level, deg):
    rng = np.random.default_rng(level)
    for _ in range(5):
        c = rng.standard_normal(deg + 1)
        q = orc.poly(1, level, poly1_moments(c), "q")
        np.testing.assert_allclose(q[: deg + 1, 0], c, atol=1e-12)
        assert np.all(np.abs(q[deg + 1:, 0]) < 1e-12)


@pytest.mark.parametrize("level,deg", [(2, 2), (3, 3), (4, 5)])
def test_reproduction_2d_least_squares(orc, level, deg):
    """Consistent data: the constrained least-squares fit has zero residual."""
    rng = np.random.default_rng(10 + level)
    for _ in range(5):
        c = rand_poly2(rng, deg)
        q = orc.poly(2, level, poly2_moments(c), "q")
        np.testing.assert_allclose(q, c, atol=1e-11)


@pytest.mark.parametrize("dim", [1, 2])
def test_linear_weight_reconstruction_reproduces_quintics(orc, dim):
    rng = np.random.default_rng(20 + dim)
    for gbar in [GBAR, (1.0, 2.0, 4.0, 8.0)]:
        if dim == 1:
            c = rng.standard_normal(6)
            np.testing.assert_allclose(orc.poly(1, 4, poly1_moments(c), "lin", gbar)[:, 0], c, atol=1e-11)
        else:
            c = rand_poly2(rng, 5)
            np.testing.assert_allclose(orc.poly(2, 4, poly2_moments(c), "lin", gbar), c, atol=1e-10)


def test_constants_reproduced_and_weights_linear(orc):
    for dim in (1, 2):
        data = np.zeros(6 if dim == 1 else 27)
        if dim == 1:
            data[:3] = 2.5
        else:
            data[:9] = 2.5
        vals, beta, omega = orc.recon_cell(dim, data, GBAR)
        np.testing.assert_allclose(vals, 2.5, rtol=0, atol=1e-14)
        assert np.all(beta < 1e-24)          # zero up to rounding of the solved tables
        np.testing.assert_allclose(omega, np.array(GBAR) / sum(GBAR), rtol=1e-13)


@pytest.mark.parametrize("dim", [1, 2])
def test_point_values_at_printed_gauss_lobatto_nodes(orc, golden, dim):
    """A tiny quintic on a constant: beta ~ delta^2 and tau_4 ~ delta^4, so with
    delta = 1e-8 the weights equal gamma to ~1e-10 and the point values are the
    quintic at the paper's nodes."""
    rng = np.random.default_rng(30 + dim)
    nodes = golden_nodes(golden)
    delta, C = 1e-8, 1.7
    if dim == 1:
        c = rng.standard_normal(6) * delta
        c[0] += C
        vals, _, _ = orc.recon_cell(1, poly1_moments(c), GBAR)
        want = np.polynomial.polynomial.polyval(nodes, c)
    else:
        c = rand_poly2(rng, 5) * delta
        c[0, 0] += C
        vals, _, _ = orc.recon_cell(2, poly2_moments(c), GBAR)
        want = np.array([poly2_eval(c, nodes[k], nodes[l]) for k in range(4) for l in range(4)])
    np.testing.assert_allclose((vals - C) / delta, (want - C) / delta, atol=1e-5)


def test_ls_2d_matches_independent_null_space_solve(orc):
    """Brute force: rebuild each 2D least-squares problem from quadrature moments of
    the monomials and solve it with a null-space method (numpy), then compare."""
    for level in (2, 3, 4):
        M, mono, conds = orc.level_matrix(2, level)
        A = np.zeros((len(conds), len(mono)))
        for r, (kind, ox, oy) in enumerate(conds):
            X = ox + XG[:, None]
            Y = oy + XG[None, :]
            w2 = WG[:, None] * WG[None, :]
            wt = 1.0 if kind == 0 else ((X - ox) if kind == 1 else (Y - oy))
            for k, (a, b) in enumerate(mono):
                A[r, k] = np.sum(w2 * wt * X ** a * Y ** b)
        assert conds[0] == (0, 0, 0)
        c0, Ar = A[0], A[1:]
        # x = c0 / |c0|^2 * b0 + N z,  N spans the null space of c0^T
        _, _, Vt = np.linalg.svd(c0[None, :])
        N = Vt[1:].T
        xp = c0 / (c0 @ c0)
        Mi = np.zeros_like(M)
        for r in range(len(conds)):
            e = np.zeros(len(conds))
            e[r] = 1.0
            b0, br = e[0], e[1:]
            z, *_ = np.linalg.lstsq(Ar @ N, br - Ar @ (xp * b0), rcond=None)
            Mi[:, r] = xp * b0 + N @ z
        np.testing.assert_allclose(M, Mi, atol=1e-12, rtol=1e-11)


# ------------------------------------------------------------- smoothness indicators

def test_beta2_closed_form_quadratic(orc):
    """beta(a + b xi + c xi^2) = b^2 + 13/3 c^2 (Jiang-Shu); p_2 = 11/10 q_2 - 1/10 q_1
    so beta_2 = (11/10)^2 (b^2 + 13/3 c^2) with b, c from the three averages."""
    rng = np.random.default_rng(3)
    for _ in range(10):
        d = rng.standard_normal(6)
        um, u0, up = d[:3]
        b = 0.5 * (up - um)
        c = 0.5 * (up - 2 * u0 + um)
        _, beta, _ = orc.recon_cell(1, d, GBAR)
        np.testing.assert_allclose(beta[1], 1.21 * (b * b + 13.0 / 3.0 * c * c), rtol=1e-13)


def test_betas_of_linear_data(orc):
    """Linear data of slope s: beta_1 = s^2 (eq. (beta1)), beta_2 = 1.21 s^2, beta_3 = beta_4 = s^2."""
    s = 0.3
    d = np.array([-s, 0.0, s, s / 12.0, s / 12.0, s / 12.0])
    _, beta, _ = orc.recon_cell(1, d, GBAR)
    np.testing.assert_allclose(beta, [s * s, 1.21 * s * s, s * s, s * s], rtol=1e-13)


@pytest.mark.parametrize("dim", [1, 2])
def test_beta_by_numerical_integration(orc, dim):
    """beta_l against independent quadrature of the squared derivatives of p_l
    (each multi-index counted once in 2D)."""
    rng = np.random.default_rng(40 + dim)
    kappa = {2: 2, 3: 3, 4: 5}
    for _ in range(3):
        data = rng.standard_normal(6 if dim == 1 else 27)
        _, beta, _ = orc.recon_cell(dim, data, GBAR)
        for l in (2, 3, 4):
            p = orc.poly(dim, l, data, "p")
            if dim == 1:
                P = np.polynomial.polynomial.Polynomial(p[:, 0])
                want = sum(np.sum(WG * P.deriv(a)(XG) ** 2) for a in range(1, kappa[l] + 1))
            else:
                want = 0.0
                X, Y = np.meshgrid(XG, XG, indexing="ij")
                w2 = WG[:, None] * WG[None, :]
                for t in range(1, kappa[l] + 1):
                    for ay in range(t + 1):
                        ax = t - ay
                        d = np.polynomial.polynomial.polyder(np.polynomial.polynomial.polyder(p, ax, axis=0), ay, axis=1)
                        want += np.sum(w2 * np.polynomial.polynomial.polyval2d(X, Y, d) ** 2)
            np.testing.assert_allclose(beta[l - 1], want, rtol=1e-11, atol=1e-14)


def test_weights_shift_away_from_discontinuity(orc):
    """A jump inside the stencil: the high-degree weights collapse (WENO-Z)."""
    d = np.array([0.0, 0.0, 1.0, 0.0, 0.0, 0.0])
    _, _, omega = orc.recon_cell(1, d, GBAR)
    assert omega[3] < 1e-3 * GBAR[3] / sum(GBAR)
    assert abs(sum(omega) - 1.0) < 1e-14


# ------------------------------------------------------------- fluxes

def _rand_euler(rng, dim):
    rho = rng.uniform(0.2, 2.0)
    u = rng.uniform(-2.0, 2.0, dim)
    p = rng.uniform(0.1, 3.0)
    E = p / 0.4 + 0.5 * rho * np.sum(u * u)
    return np.concatenate([[rho], rho * u, [E]])


@pytest.mark.parametrize("dim", [1, 2])
def test_hllc_consistency(orc, dim):
    cfg = orc.make_cfg(dim, 8, 8, eq="euler")
    rng = np.random.default_rng(5)
    for _ in range(50):
        u = _rand_euler(rng, dim)
        for d in range(dim):
            np.testing.assert_allclose(orc.num_flux(cfg, u, u, d), orc.phys_flux(cfg, u, d), rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("dim", [1, 2])
def test_hllc_stationary_contact_exact(orc, dim):
    cfg = orc.make_cfg(dim, 8, 8, eq="euler")
    p = 0.7
    uL = np.array([1.3] + [0.0] * dim + [p / 0.4])
    uR = np.array([0.2] + [0.0] * dim + [p / 0.4])
    F = orc.num_flux(cfg, uL, uR, 0)
    want = np.zeros(dim + 2)
    want[1] = p
    np.testing.assert_allclose(F, want, atol=1e-15)


def test_hllc_supersonic_upwind_and_mirror(orc):
    cfg = orc.make_cfg(1, 8, eq="euler")
    rng = np.random.default_rng(6)
    for _ in range(20):
        uL = _rand_euler(rng, 1)
        uR = _rand_euler(rng, 1)
        # mirror symmetry: swap sides and negate the velocity -> flux mirrored
        F = orc.num_flux(cfg, uL, uR, 0)
        mL = uR * np.array([1, -1, 1])
        mR = uL * np.array([1, -1, 1])
        Fm = orc.num_flux(cfg, mL, mR, 0)
        np.testing.assert_allclose(F, Fm * np.array([-1, 1, -1]), rtol=1e-12, atol=1e-12)
    # supersonic to the right: upwind
    uL = np.array([1.0, 5.0, 0.5 / 0.4 + 0.5 * 25.0])
    uR = np.array([0.5, 0.5 * 4.0, 0.3 / 0.4 + 0.5 * 0.5 * 16.0])
    np.testing.assert_allclose(orc.num_flux(cfg, uL, uR, 0), orc.phys_flux(cfg, uL, 0), rtol=1e-14)


def test_hllc_2d_rotation(orc):
    """The y-flux of a state equals the x-flux of the state with (mu, nu) swapped."""
    cfg = orc.make_cfg(2, 8, 8, eq="euler")
    rng = np.random.default_rng(7)
    swap = [0, 2, 1, 3]
    for _ in range(20):
        uL, uR = _rand_euler(rng, 2), _rand_euler(rng, 2)
        G = orc.num_flux(cfg, uL, uR, 1)
        F = orc.num_flux(cfg, uL[swap], uR[swap], 0)
        np.testing.assert_allclose(G, F[swap], rtol=1e-13, atol=1e-13)


def test_llf_is_upwind_for_advection(orc):
    cfg = orc.make_cfg(1, 8, eq="advection", adv=(1.5, 0.0))
    np.testing.assert_allclose(orc.num_flux(cfg, [0.3], [2.0], 0), [1.5 * 0.3], rtol=1e-15)
    cfg = orc.make_cfg(1, 8, eq="advection", adv=(-0.5, 0.0))
    np.testing.assert_allclose(orc.num_flux(cfg, [0.3], [2.0], 0), [-0.5 * 2.0], rtol=1e-15)


# ------------------------------------------------------------- semi-discrete consistency

def _order(e1, e2):
    return math.log2(e1 / e2)


def _rhs_error_1d(orc, eq, n):
    if eq == "advection":
        p = W.advection_sin_1d(n)
        dmdt = W.moments_1d(lambda x: -np.cos(x), p.x0, p.x1, n)
    else:
        p = W.density_wave_1d(n)

        def f(x):
            r_t = -0.2 * math.pi * np.cos(math.pi * x)
            return np.stack([r_t, r_t, 0.5 * r_t])
        dmdt = W.moments_1d(f, p.x0, p.x1, n)
    cfg = orc.make_cfg(1, n, dx=p.dx, eq=eq, indicator="kxrcf", bc=p.bc)
    _, L, mask, _, rc = orc.rhs(cfg, p.m)
    assert rc == 0 and mask.sum() == 0
    return np.abs(L - dmdt).mean()


def _rhs_error_2d(orc, eq, n):
    if eq == "advection":
        p = W.advection_2d(n, 1.0, 0.5)

        def f(X, Y):
            ux = np.cos(X) * np.sin(Y) - 0.5 * np.sin(X + Y)
            uy = np.sin(X) * np.cos(Y) - 0.5 * np.sin(X + Y)
            return -(1.0 * ux + 0.5 * uy)
        dmdt = W.moments_2d(f, p.x0, p.x1, p.y0, p.y1, n, n)
    elif eq == "burgers":
        p = W.burgers_2d(n)

        def f(X, Y):
            u = 0.5 + np.sin(math.pi * (X + Y) / 2.0)
            g = 0.5 * math.pi * np.cos(math.pi * (X + Y) / 2.0)
            return -(u * g + u * g)
        dmdt = W.moments_2d(f, p.x0, p.x1, p.y0, p.y1, n, n)
    else:
        L0 = 4.0

        def ic(X, Y):
            rho = 1.0 + 0.2 * np.sin(math.pi * (X + 2.0 * Y) / 2.0)
            one = np.ones_like(X)
            return W.prim_to_cons_2d(rho, one, 0.5 * one, one)
        m = W.moments_2d(ic, 0.0, L0, 0.0, L0, n, n)
        p = W.Problem("dw2d", 2, n, n, 0.0, L0, 0.0, L0, "euler", ("periodic",) * 4, m)

        def f(X, Y):
            rx = 0.2 * math.pi / 2.0 * np.cos(math.pi * (X + 2.0 * Y) / 2.0)
            ry = 2.0 * rx
            r_t = -(1.0 * rx + 0.5 * ry)       # rho_t = -(mu rho_x + nu rho_y)
            return np.stack([r_t, r_t, 0.5 * r_t, 0.5 * (1.0 + 0.25) * r_t])
        dmdt = W.moments_2d(f, 0.0, L0, 0.0, L0, n, n)
    cfg = orc.make_cfg(2, n, n, dx=p.dx, dy=p.dy, eq=eq, adv=p.adv, indicator="kxrcf", bc=p.bc)
    _, L, mask, _, rc = orc.rhs(cfg, p.m)
    assert rc == 0 and mask.sum() == 0
    return np.abs(L - dmdt).mean()


# L(U) at t = 0 against the exact time derivative of the moments.  Mean errors:
# at critical points of u the literal beta_1 of eq. (beta1) / (2D-beta1) vanishes
# and the weights leave gamma for a few cells on coarse grids, so the grids are
# taken where that effect has died out.
@pytest.mark.parametrize("eq", ["advection", "euler"])
def test_semidiscrete_operator_converges_1d(orc, eq):
    e1, e2 = _rhs_error_1d(orc, eq, 64), _rhs_error_1d(orc, eq, 128)
    assert _order(e1, e2) > 4.7, (e1, e2)


@pytest.mark.parametrize("eq", ["advection", "burgers", "euler"])
def test_semidiscrete_operator_converges_2d(orc, eq):
    e1, e2 = _rhs_error_2d(orc, eq, 32), _rhs_error_2d(orc, eq, 64)
    assert _order(e1, e2) > 4.5, (e1, e2)


# ------------------------------------------------------------- conservation

def test_conservation_with_troubled_cells(orc):
    p = W.four_quadrant_2d(24, seed=3)
    cfg = orc.make_cfg(2, 24, 24, dx=p.dx, dy=p.dy, eq="euler", bc=("periodic",) * 4)
    m = p.m
    t0 = orc.totals(cfg, m)
    nflag = 0
    for _ in range(3):
        Um, _, mask, _, _ = orc.rhs(cfg, m)
        np.testing.assert_array_equal(Um[:, 0], m[:, 0])     # the modification leaves ubar alone
        m, masks, rc = orc.step(cfg, m, 0.3 * orc.max_dt(cfg, m))
        assert rc == 0
        nflag += masks.sum()
    assert nflag > 0
    np.testing.assert_allclose(orc.totals(cfg, m), t0, rtol=1e-13, atol=1e-14)


def test_conservation_1d_euler_periodic(orc):
    p = W.shu_osher_1d(200)
    cfg = orc.make_cfg(1, 200, dx=p.dx, eq="euler", bc=("periodic",) * 4)
    m = p.m
    t0 = orc.totals(cfg, m)
    for _ in range(5):
        m, _, rc = orc.step(cfg, m, orc.max_dt(cfg, m))
        assert rc == 0
    np.testing.assert_allclose(orc.totals(cfg, m), t0, rtol=1e-13)


# ------------------------------------------------------------- convergence and the paper's tables

def _advect(orc, n, indicator, gbar=GBAR, t_end=1.0):
    p = W.advection_sin_1d(n)
    cfg = orc.make_cfg(1, n, dx=p.dx, eq="advection", indicator=indicator, gbar=gbar)
    nst = int(math.ceil(t_end / (0.5 * p.dx ** 2)))
    dt = t_end / nst
    m, flagged = p.m, 0
    for _ in range(nst):
        m, masks, rc = orc.step(cfg, m, dt)
        flagged += int(masks.sum())
    ex = W.moments_1d(lambda x: np.sin(x - t_end), p.x0, p.x1, n)
    return np.abs(m[0, 0, 0] - ex[0, 0, 0]).mean(), flagged


def test_advection_order_and_empty_mask(orc):
    e40, f40 = _advect(orc, 40, "kxrcf")
    e80, f80 = _advect(orc, 80, "kxrcf")
    assert f40 == 0 and f80 == 0
    assert _order(e40, e80) > 5.0


@pytest.mark.parametrize("gbar", [(1.0, 1.0, 1.0, 1.0), (1.0, 2.0, 4.0, 8.0), (1.0, 10.0, 100.0, 1000.0)])
def test_order_independent_of_linear_weights_with_beta_of_q(orc, gbar):
    """Remark 1 claims the smooth-region order does not depend on the linear
    weights because every beta_l = u'^2 dx^2 + O(dx^4).  That expansion holds
    when beta_l is taken of q_l (diagnostic switch of the oracle)."""
    orc.set_beta_source(True)
    try:
        e1, f1 = _advect(orc, 80, "kxrcf", gbar, t_end=0.25)
        e2, f2 = _advect(orc, 160, "kxrcf", gbar, t_end=0.25)
    finally:
        orc.set_beta_source(False)
    assert f1 == 0 and f2 == 0
    assert _order(e1, e2) > 5.5, (e1, e2)


def test_literal_beta_order_depends_on_linear_weights(orc):
    """With beta_l of p_l as eq. (beta) is written (the scheme as implemented),
    beta_2 = (11/10)^2 u'^2 dx^2 + ..., tau_4 = O(dx^4) and the weights leave
    gamma by O(dx^2): the paper's weights 1, 10, 100, 1000 keep sixth order,
    flat weights drop to fourth order asymptotically."""
    e1, _ = _advect(orc, 80, "kxrcf", GBAR, t_end=0.25)
    e2, _ = _advect(orc, 160, "kxrcf", GBAR, t_end=0.25)
    assert _order(e1, e2) > 5.5, (e1, e2)
    e1, f1 = _advect(orc, 160, "kxrcf", (1.0, 1.0, 1.0, 1.0), t_end=0.25)
    e2, f2 = _advect(orc, 320, "kxrcf", (1.0, 1.0, 1.0, 1.0), t_end=0.25)
    assert f1 == 0 and f2 == 0
    assert 3.5 < _order(e1, e2) < 4.8, (e1, e2)


def _burgers1d_errors(orc, n, indicator, mod_in_L_only=False):
    T = 0.5 / math.pi
    p = W.burgers_1d(n)
    cfg = orc.make_cfg(1, n, dx=p.dx, eq="burgers", indicator=indicator, mod_in_L_only=mod_in_L_only)
    nst = int(math.ceil(T / (0.2 * p.dx ** 2)))
    m = p.m
    for _ in range(nst):
        m, _, rc = orc.step(cfg, m, T / nst)
        assert rc == 0
    s, w = 0.5 * np.polynomial.legendre.leggauss(8)[0], 0.5 * np.polynomial.legendre.leggauss(8)[1]
    X = ((np.arange(n) + 0.5) * p.dx)[:, None] + s[None, :] * p.dx
    u = exact.burgers_characteristics(lambda x: 0.5 + np.sin(math.pi * x),
                                      lambda x: math.pi * np.cos(math.pi * x), X, T)
    e = m[0, 0, 0] - (u * w).sum(1)
    return np.abs(e).mean(), np.abs(e).max()


def test_table1_burgers_1d_n80(orc, golden):
    """Errors of Table 1 at N = 80 (I and NI) reproduced within a factor 1.5; the
    paper's reduced time step is unstated, ours is 0.2 dx^2."""
    row = {r[0]: r for r in golden["table1_burgers_1d"]["rows"]}[80]
    l1, linf = _burgers1d_errors(orc, 80, "kxrcf")
    assert row[1] / 1.5 < l1 < row[1] * 1.5 and row[2] / 1.5 < linf < row[2] * 1.5
    l1, linf = _burgers1d_errors(orc, 80, "all")
    assert row[3] / 1.5 < l1 < row[3] * 1.5 and row[4] / 1.5 < linf < row[4] * 1.5


def test_table1_ni_column_fixes_the_persistence_of_the_modification(orc, golden):
    """Table 1's NI column (every cell modified) decides how Step 2.2's modified
    first moments are used: written back into the stage state (so the
    Runge-Kutta combination of eq. (Runge-Kutta) takes them) the N = 80 errors
    are 5.96e-8 / 9.39e-7 against the printed 5.96E-08 / 9.36E-07; used inside
    L only, the state's own first moments drift from the averages' and the
    error is four orders larger (6.5e-4), below first order in N."""
    row = {r[0]: r for r in golden["table1_burgers_1d"]["rows"]}[80]
    l1, linf = _burgers1d_errors(orc, 80, "all")
    assert abs(l1 - row[3]) < 0.01 * row[3] and abs(linf - row[4]) < 0.01 * row[4], (l1, linf)
    l1b, _ = _burgers1d_errors(orc, 80, "all", mod_in_L_only=True)
    assert l1b > 1e3 * row[3], l1b


def test_table2_burgers_2d_n40(orc, golden):
    """Errors of Table 2 at 40 x 40 (I scheme) within a factor 1.5; dt = 0.3 dx^2."""
    n, T = 40, 0.5 / math.pi
    row = {r[0]: r for r in golden["table2_burgers_2d"]["rows"]}[n]
    p = W.burgers_2d(n)
    cfg = orc.make_cfg(2, n, n, dx=p.dx, dy=p.dy, eq="burgers", indicator="kxrcf")
    nst = int(math.ceil(T / (0.3 * p.dx ** 2)))
    m = p.m
    for _ in range(nst):
        m, masks, rc = orc.step(cfg, m, T / nst)
        assert rc == 0 and masks.sum() == 0

    def f(X, Y):
        return exact.burgers_characteristics(lambda s: 0.5 + np.sin(math.pi * s / 2.0),
                                             lambda s: 0.5 * math.pi * np.cos(math.pi * s / 2.0),
                                             X + Y, T, c=2.0)
    ex = W.moments_2d(f, 0.0, 4.0, 0.0, 4.0, n, n)
    e = m[0, 0] - ex[0, 0]
    l1, linf = np.abs(e).mean(), np.abs(e).max()
    assert row[1] / 1.5 < l1 < row[1] * 1.5, l1
    assert row[2] / 1.5 < linf < row[2] * 1.5, linf


# ------------------------------------------------------------- shock tubes

@pytest.mark.parametrize("name", ["sod", "lax"])
def test_shock_tube_converges_to_exact_riemann(orc, golden, name):
    errs = []
    for n in (100, 200):
        p = W.sod_1d(n) if name == "sod" else W.lax_1d(n)
        cfg = orc.make_cfg(1, n, dx=p.dx, eq="euler", bc=p.bc)
        m, _ = orc.run(cfg, p.m, p.t_end)
        assert np.all(np.isfinite(m))
        ex = exact.riemann_density_averages(p.meta["left"], p.meta["right"], p.x0, p.x1, n,
                                            p.meta["xs"], p.t_end)
        errs.append(np.abs(m[0, 0, 0] - ex).mean())
    assert errs[1] < (0.75 if name == "sod" else 0.85) * errs[0], errs
    assert errs[1] < (4e-3 if name == "sod" else 8e-3), errs
    if name == "lax":
        lax = golden["lax_problem"]
        assert list(p.meta["left"]) == lax["left"] and list(p.meta["right"]) == lax["right"]


# ------------------------------------------------------------- linear stability (a property of the scheme)

def test_linear_spectrum_and_ssp_rk3_limit(orc):
    """Jacobian of L for linear advection at tiny amplitude (the weights sit at
    their linear values): no eigenvalue in the right half plane (the upwind
    flux is dissipative or neutral), and SSP-RK3 keeps |R(dt lambda)| <= 1 up to
    CFL ~ 0.569 only.  The paper's CFL 0.6 is just beyond: its largest
    amplification is ~1.17 per step, which rounding noise excites."""
    N = 48
    dx = 2 * math.pi / N
    cfg = orc.make_cfg(1, N, dx=dx, eq="advection", adv=(1.0, 0.0), indicator="none")
    amp, n = 1e-9, 2 * N
    A = np.zeros((n, n))
    for k in range(n):
        U = np.zeros(n)
        U[k] = amp
        A[:, k] = orc.rhs(cfg, U.reshape(1, 2, 1, N))[1].reshape(-1) / amp
    lam = np.linalg.eigvals(A) * dx
    assert lam.real.max() < 1e-12

    def amp_max(cfl):
        z = cfl * lam
        return np.abs(1 + z + z * z / 2 + z ** 3 / 6).max()
    assert amp_max(0.56) <= 1.0 + 1e-12
    assert 1.15 < amp_max(0.6) < 1.2
