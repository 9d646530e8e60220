"""Closed-form and exact solutions used to pin the oracle (test helpers).

* Burgers' equation before shock formation, by characteristics
  (u = u0(x - u t)), solved by Newton at each quadrature point.
* The exact Riemann solution of the 1D Euler equations for an ideal gas,
  written from the pressure-function formulation (Toro, "Riemann Solvers and
  Numerical Methods for Fluid Dynamics", ch. 4): Newton on
  f_L(p) + f_R(p) + (u_R - u_L) = 0, then sampling at x/t.
"""
from __future__ import annotations

import math

import numpy as np


def burgers_characteristics(u0, du0, X, t, c=1.0, iters=60):
    """Solve u = u0(X - c u t) for u at points X (c = 2 for u0(x+y) in 2D)."""
    u = u0(X)
    for _ in range(iters):
        arg = X - c * u * t
        F = u - u0(arg)
        dF = 1.0 + du0(arg) * c * t
        u = u - F / dF
    return u


def _pressure_fn(p, rho, pk, ck, g):
    if p > pk:   # shock
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        f = (p - pk) * math.sqrt(A / (p + B))
        df = math.sqrt(A / (B + p)) * (1.0 - (p - pk) / (2.0 * (B + p)))
    else:        # rarefaction
        f = 2.0 * ck / (g - 1.0) * ((p / pk) ** ((g - 1.0) / (2.0 * g)) - 1.0)
        df = 1.0 / (rho * ck) * (p / pk) ** (-(g + 1.0) / (2.0 * g))
    return f, df


def riemann_star(left, right, g=1.4):
    rl, ul, pl = left
    rr, ur, pr = right
    cl = math.sqrt(g * pl / rl)
    cr = math.sqrt(g * pr / rr)
    p = max(1e-8, 0.5 * (pl + pr) - 0.125 * (ur - ul) * (rl + rr) * (cl + cr))
    for _ in range(100):
        fl, dfl = _pressure_fn(p, rl, pl, cl, g)
        fr, dfr = _pressure_fn(p, rr, pr, cr, g)
        dp = (fl + fr + ur - ul) / (dfl + dfr)
        pn = max(1e-12, p - dp)
        if abs(pn - p) <= 1e-14 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _pressure_fn(p, rl, pl, cl, g)
    fr, _ = _pressure_fn(p, rr, pr, cr, g)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def riemann_sample(left, right, S, g=1.4):
    """Primitive (rho, u, p) of the exact solution at similarity coordinates S = x/t."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl = math.sqrt(g * pl / rl)
    cr = math.sqrt(g * pr / rr)
    ps, us = riemann_star(left, right, g)
    g6 = (g - 1.0) / (g + 1.0)
    out = np.zeros((3,) + np.shape(S))
    S = np.asarray(S, dtype=float)
    for idx, s in np.ndenumerate(S):
        if s <= us:
            if ps > pl:
                sl = ul - cl * math.sqrt((g + 1.0) / (2.0 * g) * ps / pl + (g - 1.0) / (2.0 * g))
                w = (rl, ul, pl) if s <= sl else (rl * (ps / pl + g6) / (g6 * ps / pl + 1.0), us, ps)
            else:
                shl = ul - cl
                csl = cl * (ps / pl) ** ((g - 1.0) / (2.0 * g))
                stl = us - csl
                if s <= shl:
                    w = (rl, ul, pl)
                elif s > stl:
                    w = (rl * (ps / pl) ** (1.0 / g), us, ps)
                else:
                    u = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * ul + s)
                    c = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * (ul - s))
                    w = (rl * (c / cl) ** (2.0 / (g - 1.0)), u, pl * (c / cl) ** (2.0 * g / (g - 1.0)))
        else:
            if ps > pr:
                sr = ur + cr * math.sqrt((g + 1.0) / (2.0 * g) * ps / pr + (g - 1.0) / (2.0 * g))
                w = (rr, ur, pr) if s >= sr else (rr * (ps / pr + g6) / (g6 * ps / pr + 1.0), us, ps)
            else:
                shr = ur + cr
                csr = cr * (ps / pr) ** ((g - 1.0) / (2.0 * g))
                str_ = us + csr
                if s >= shr:
                    w = (rr, ur, pr)
                elif s <= str_:
                    w = (rr * (ps / pr) ** (1.0 / g), us, ps)
                else:
                    u = 2.0 / (g + 1.0) * (-cr + 0.5 * (g - 1.0) * ur + s)
                    c = 2.0 / (g + 1.0) * (cr - 0.5 * (g - 1.0) * (ur - s))
                    w = (rr * (c / cr) ** (2.0 / (g - 1.0)), u, pr * (c / cr) ** (2.0 * g / (g - 1.0)))
        out[(slice(None),) + idx] = w
    return out


def riemann_density_averages(left, right, x0, x1, nx, xs, t, g=1.4, sub=64):
    """Cell averages of the exact density (midpoint rule on sub-cells)."""
    dx = (x1 - x0) / nx
    xe = x0 + (np.arange(nx * sub) + 0.5) * dx / sub
    rho = riemann_sample(left, right, (xe - xs) / t, g)[0]
    return rho.reshape(nx, sub).mean(axis=1)
