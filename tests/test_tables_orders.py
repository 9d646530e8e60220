"""Convergence sweeps of the paper's Tables 1 and 2 (Sec. 3, Examples 3.1 and
3.2: Burgers u0 = 0.5 + sin(pi x) on (0, 2) and 0.5 + sin(pi (x + y) / 2) on
(0, 4)^2, periodic, to T = 0.5/pi), HWENO6-M5-I (KXRCF) and -NI (every cell
modified), N = 10 ... 320, with the observed orders printed beside the paper's.

The paper's time step is "suitably reduced" and not stated; ours is 0.2 dx^2
(1D) and 0.3 dx^2 (2D), small enough that the spatial error dominates.  1D runs
on the CPU oracle (slow: about four minutes; HWENO_SLOW=1); 2D on the GPU FP64
path (parity-tested against the oracle to 1e-12), which covers 320^2 in
seconds.  Asserted where the scheme is asymptotic (N >= 80): errors within a
factor 2 of the printed ones and the finest observed orders within 0.6 of the
printed ones; the NI column, which fixes the persistence reading of Step 2.2,
is matched to 5 % in 1D.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

from paper_2201_12193_gb300 import workloads as W

NS = (10, 20, 40, 80, 160, 320)


def _orders(errs):
    return [None] + [math.log2(a / b) for a, b in zip(errs[:-1], errs[1:])]


def _report(title, rows, printed):
    print(f"\n{title}: N, L1, Linf, order L1, order Linf  |  paper L1, Linf, orders")
    o1, oi = _orders([r[0] for r in rows]), _orders([r[1] for r in rows])
    p1, pi = _orders([r[0] for r in printed]), _orders([r[1] for r in printed])
    for k, n in enumerate(NS):
        f = lambda x: "  -  " if x is None else f"{x:5.2f}"   # noqa: E731
        print(f"{n:4d} {rows[k][0]:.2e} {rows[k][1]:.2e} {f(o1[k])} {f(oi[k])}  |  "
              f"{printed[k][0]:.2e} {printed[k][1]:.2e} {f(p1[k])} {f(pi[k])}")
    return o1, oi, p1, pi


def _check(rows, printed, o1, oi, p1, pi, tight=None):
    for k, n in enumerate(NS):
        if n < 80:
            continue
        for a, b in zip(rows[k], printed[k]):
            assert b / 2 < a < 2 * b, (n, rows[k], printed[k])
            if tight:
                assert abs(a - b) <= tight * b, (n, rows[k], printed[k])
    assert abs(o1[-1] - p1[-1]) < 0.6 and abs(oi[-1] - pi[-1]) < 0.6, (o1, oi, p1, pi)


def _burgers_1d(orc, exact, n, indicator):
    T = 0.5 / math.pi
    p = W.burgers_1d(n)
    cfg = orc.make_cfg(1, n, dx=p.dx, eq="burgers", indicator=indicator)
    nst = int(math.ceil(T / (0.2 * p.dx ** 2)))
    m = p.m
    for _ in range(nst):
        m, _, rc = orc.step(cfg, m, T / nst)
        assert rc == 0
    s, w = np.polynomial.legendre.leggauss(8)
    X = ((np.arange(n) + 0.5) * p.dx)[:, None] + 0.5 * s[None, :] * p.dx
    u = exact.burgers_characteristics(lambda x: 0.5 + np.sin(math.pi * x),
                                      lambda x: math.pi * np.cos(math.pi * x), X, T)
    e = m[0, 0, 0] - (u * 0.5 * w).sum(1)
    return float(np.abs(e).mean()), float(np.abs(e).max())


@pytest.mark.slow
@pytest.mark.parametrize("column,indicator", [(1, "kxrcf"), (3, "all")], ids=["I", "NI"])
def test_table1_orders_1d_burgers(orc, golden, column, indicator):
    import exact
    printed = [(r[column], r[column + 1]) for r in golden["table1_burgers_1d"]["rows"]]
    rows = [_burgers_1d(orc, exact, n, indicator) for n in NS]
    o1, oi, p1, pi = _report(f"Table 1 ({indicator})", rows, printed)
    _check(rows, printed, o1, oi, p1, pi, tight=0.05 if indicator == "all" else None)


@pytest.mark.gpu
@pytest.mark.parametrize("column,indicator", [(1, "kxrcf"), (3, "all")], ids=["I", "NI"])
def test_table2_orders_2d_burgers(golden, column, indicator):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import exact
    from paper_2201_12193_gb300 import build, hweno
    build.build()
    printed = [(r[column], r[column + 1]) for r in golden["table2_burgers_2d"]["rows"]]
    T = 0.5 / math.pi
    rows = []
    for n in NS:
        p = W.burgers_2d(n)
        s = hweno.Solver.from_problem(p, indicator=indicator)
        s.set_moments(torch.from_numpy(p.m).cuda())
        nst = int(math.ceil(T / (0.3 * p.dx ** 2)))
        for _ in range(nst):
            s.step(T / nst)
        m = s.get_moments()
        s.close()

        def f(X, Y):
            return exact.burgers_characteristics(lambda z: 0.5 + np.sin(math.pi * z / 2.0),
                                                 lambda z: 0.5 * math.pi * np.cos(math.pi * z / 2.0),
                                                 X + Y, T, c=2.0)
        ex = W.moments_2d(f, 0.0, 4.0, 0.0, 4.0, n, n)
        e = m[0, 0] - ex[0, 0]
        rows.append((float(np.abs(e).mean()), float(np.abs(e).max())))
    o1, oi, p1, pi = _report(f"Table 2 ({indicator})", rows, printed)
    _check(rows, printed, o1, oi, p1, pi)
