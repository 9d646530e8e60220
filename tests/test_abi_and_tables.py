"""CPU-only checks of the boundary and of the kernel tables.

* libhweno.so builds for sm_103a and exports every function include/hweno.h
  declares (no compute call: there is no GPU here).
* The generated value tables and smoothness-indicator rows (exact rational
  derivation for the CUDA path) agree with the oracle's own run-time solves.
"""
from __future__ import annotations

import importlib.util
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2201_12193_gb300", "csrc")


def _gen():
    spec = importlib.util.spec_from_file_location("gen_tables", os.path.join(CSRC, "gen_tables.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_header_declares_and_library_exports():
    from paper_2201_12193_gb300 import build
    lib = build.build()
    decl = set()
    for name in os.listdir(os.path.join(ROOT, "include")):
        if name.endswith(".h"):
            text = open(os.path.join(ROOT, "include", name)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)          # drop comments
            decl |= set(re.findall(r"^\s*(?:[\w\*]+\s+)+\**(hweno_\w+)\s*\(", text, flags=re.M))
    assert {"hweno_create", "hweno_step", "hweno_set_moments", "hweno_get_moments", "hweno_troubled_mask"} <= decl
    out = subprocess.check_output(["nm", "-D", "--defined-only", lib], text=True)
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    missing = decl - exported
    assert not missing, missing


def test_library_loads_without_gpu():
    import ctypes
    from paper_2201_12193_gb300 import build, hweno
    build.build()
    lib = hweno.lib()
    assert lib.hweno_version() >= 100
    assert isinstance(lib, ctypes.CDLL)


def test_generated_header_is_current():
    gen = _gen()
    import io
    buf = io.StringIO()
    gen.emit_parity(buf)
    with open(os.path.join(CSRC, "hweno_parity.h")) as f:
        assert f.read() == buf.getvalue()


def _oracle_data(d4, dvec, dim):
    if dim == 1:
        return dvec.copy()
    data = np.zeros(27)
    for c, (kind, ox, oy) in enumerate(d4):
        data[kind * 9 + (oy + 1) * 3 + (ox + 1)] = dvec[c]
    return data


@pytest.mark.parametrize("dim", [1, 2])
def test_parity_form_matches_oracle(orc, dim):
    """The form the kernels evaluate: parity split, per-class value rows at the base
    points with the mirror signs, and per-class indicator rows, against the
    oracle's polynomials and smoothness indicators."""
    gen = _gen()
    P = gen.build_parity(dim)
    d4, basis, sl, bases, VP, RCP = P
    lay = gen.beta_layout(dim, P)
    classes = gen.parity_classes(dim)
    nodes = [-0.5, -np.sqrt(5) / 10, np.sqrt(5) / 10, 0.5]
    rng = np.random.default_rng(5 + dim)
    gbar = (1.0, 2.0, 4.0, 8.0)
    S = np.cumsum((0.0,) + gbar)
    for _ in range(3):
        dvec = rng.standard_normal(len(d4))
        s = np.zeros(len(d4))
        for c in classes:
            for j, r in enumerate(basis[c]):
                s[sl[c][j]] = np.dot(r, dvec)
        data = _oracle_data(d4, dvec, dim)
        for lvl in (2, 3, 4):
            cf = orc.poly(dim, lvl, data, "q")
            for b in bases:
                for sx in (1, -1):
                    for sy in ((1, -1) if dim == 2 else (1,)):
                        k = b[0] if sx > 0 else 3 - b[0]
                        l = b[1] if (dim == 1 or sy > 0) else 3 - b[1]
                        got = 0.0
                        for c in classes:
                            chi = (sx if c[0] else 1) * (sy if c[1] else 1)
                            got += chi * sum(float(g.to_decimal()) * s[sl[c][j]] for j, g in enumerate(VP[(lvl, b, c)]))
                        x, y = nodes[k], (nodes[l] if dim == 2 else 0.0)
                        want = sum(cf[a, bb] * x ** a * y ** bb for a in range(6) for bb in range(6))
                        assert abs(got - want) <= 1e-12 * (1 + abs(want))
        _, beta, _ = orc.recon_cell(dim, data, gbar)
        for lvl in (2, 3, 4):
            a, bcoef = S[lvl] / gbar[lvl - 1], -S[lvl - 1] / gbar[lvl - 1]
            tot = 0.0
            for ent in lay[lvl]:
                r = sum((a * float(x) + bcoef * float(y)) * s[j] for (j, x, y) in ent)
                tot += r * r
            np.testing.assert_allclose(tot, beta[lvl - 1], rtol=1e-11)


@pytest.mark.parametrize("dim", [1, 2])
def test_value_tables_match_oracle(orc, dim):
    """q_l at the Gauss-Lobatto points: generator tables vs the oracle's polynomials."""
    gen = _gen()
    d4, V, _ = gen.build(dim)
    rng = np.random.default_rng(7 + dim)
    nodes = [-0.5, -np.sqrt(5) / 10, np.sqrt(5) / 10, 0.5]
    for _ in range(3):
        dvec = rng.standard_normal(len(d4))
        # oracle data layout: 1D (u-1,u0,u1,v-1,v0,v1); 2D ubar[9], vbar[9], wbar[9]
        if dim == 1:
            data = dvec.copy()
        else:
            data = np.zeros(27)
            for c, (kind, ox, oy) in enumerate(d4):
                data[kind * 9 + (oy + 1) * 3 + (ox + 1)] = dvec[c]
        pts = [(k, 0) for k in range(4)] if dim == 1 else [(k, l) for k in range(4) for l in range(4)]
        for lvl in (2, 3, 4):
            c = orc.poly(dim, lvl, data, "q")
            want = [sum(c[a, b] * nodes[k] ** a * (nodes[l] ** b if dim == 2 else (1.0 if b == 0 else 0.0))
                        for a in range(6) for b in range(6)) for (k, l) in pts]
            got = [sum(float(V[lvl][p][q]) * dvec[q] for q in range(len(d4))) for p in range(len(pts))]
            np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("dim", [1, 2])
def test_indicator_rows_match_oracle_beta(orc, dim):
    """|a RC_{l,l} d + b RC_{l,l-1} d|^2 equals the oracle's beta_l of p_l."""
    gen = _gen()
    d4, _, RC = gen.build(dim)
    gbar = (1.0, 10.0, 100.0, 1000.0)
    S = np.cumsum((0.0,) + gbar)
    rng = np.random.default_rng(11 + dim)
    for _ in range(3):
        dvec = rng.standard_normal(len(d4))
        if dim == 1:
            data = dvec.copy()
        else:
            data = np.zeros(27)
            for c, (kind, ox, oy) in enumerate(d4):
                data[kind * 9 + (oy + 1) * 3 + (ox + 1)] = dvec[c]
        _, beta, _ = orc.recon_cell(dim, data, gbar)
        for lvl in (2, 3, 4):
            a = S[lvl] / gbar[lvl - 1]
            b = -S[lvl - 1] / gbar[lvl - 1]
            y = np.array([[float(v) for v in row] for row in RC[(lvl, lvl)]]) @ dvec * a
            if (lvl, lvl - 1) in RC:
                y += np.array([[float(v) for v in row] for row in RC[(lvl, lvl - 1)]]) @ dvec * b
            np.testing.assert_allclose(y @ y, beta[lvl - 1], rtol=1e-11)
