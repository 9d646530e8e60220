#!/usr/bin/env python3
"""Generate hweno_tables.h: the constant tables of the CUDA stage kernels.

Everything is derived in exact rational arithmetic (``fractions``), with the
Gauss-Lobatto nodes +-sqrt(5)/10 carried exactly in Q(sqrt 5), and rounded to
double once, at the end, through 60-digit decimals.  Nothing here is shared
with the CPU oracle, which solves its own systems at run time.

Tables (scaled coordinates xi = (x - x_i)/dx, eta = (y - y_j)/dy):

  value tables  V_l[pt][d]  : q_l at the Gauss-Lobatto points, as linear maps
                              of the level's data vector (eq. (q) in 1D,
                              eqs. (2D-q2)-(2D-q4) in 2D: least squares with
                              the target-cell average exact);
  indicator tables RC[l][m] : rows R_kappa C_m, where C_m maps the data to the
                              non-constant monomial coefficients of q_m and
                              R_kappa^T R_kappa is the Gram matrix of
                              sum_{1<=|a|<=kappa} int (D^a .)(D^a .) over the
                              cell, so that beta(p) = |R_kappa c(p)|^2
                              (eq. (beta) / (2D-beta); kappa = 2, 3, 5).
  The kernels combine RC rows with the run-time linear weights:
  p_l = (S_l q_l - S_{l-1} q_{l-1}) / g_l  (eq. (p) with g = gbar, S_l = g_1+..+g_l).

Run:  python gen_tables.py > hweno_tables.h
"""
from __future__ import annotations

import decimal
import struct
import sys
from fractions import Fraction as F

decimal.getcontext().prec = 60
SQRT5 = decimal.Decimal(5).sqrt()


class Q5:
    """a + b sqrt(5) with rational a, b."""
    __slots__ = ("a", "b")

    def __init__(self, a, b=0):
        self.a, self.b = F(a), F(b)

    def __add__(self, o):
        o = o if isinstance(o, Q5) else Q5(o)
        return Q5(self.a + o.a, self.b + o.b)

    __radd__ = __add__

    def __mul__(self, o):
        o = o if isinstance(o, Q5) else Q5(o)
        return Q5(self.a * o.a + 5 * self.b * o.b, self.a * o.b + self.b * o.a)

    __rmul__ = __mul__

    def to_decimal(self):
        return decimal.Decimal(self.a.numerator) / decimal.Decimal(self.a.denominator) + \
            decimal.Decimal(self.b.numerator) / decimal.Decimal(self.b.denominator) * SQRT5


NODES = [Q5(F(-1, 2)), Q5(0, F(-1, 10)), Q5(0, F(1, 10)), Q5(F(1, 2))]


def qpow(x, n):
    r = Q5(1)
    for _ in range(n):
        r = r * x
    return r


def cell_int(n, o):
    """int_{o-1/2}^{o+1/2} s^n ds, exact."""
    hi, lo = F(2 * o + 1, 2), F(2 * o - 1, 2)
    return (hi ** (n + 1) - lo ** (n + 1)) / (n + 1)


def moment(kind, a, b, ox, oy):
    ix = cell_int(a, ox) if kind != 1 else cell_int(a + 1, ox) - ox * cell_int(a, ox)
    iy = cell_int(b, oy) if kind != 2 else cell_int(b + 1, oy) - oy * cell_int(b, oy)
    return ix * iy


def monomials(dim, deg):
    out = []
    for t in range(deg + 1):
        for b in range(t + 1):
            if dim == 1 and b:
                continue
            out.append((t - b, b))
    return out


def solve(A, B):
    """Exact Gauss-Jordan: A (n x n) X = B (n x m)."""
    n, m = len(A), len(B[0])
    M = [list(A[i]) + list(B[i]) for i in range(n)]
    for c in range(n):
        p = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[p] = M[p], M[c]
        inv = 1 / M[c][c]
        M[c] = [v * inv for v in M[c]]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c]
                M[r] = [vr - f * vc for vr, vc in zip(M[r], M[c])]
    return [row[n:] for row in M]


def level_matrix(dim, deg, conds):
    """Coefficient map (nmono x ncond).  conds[0] is the target-cell average;
    1D: square interpolation; 2D: that row exact, the others least squares."""
    mono = monomials(dim, deg)
    A = [[moment(k, a, b, ox, oy) for (a, b) in mono] for (k, ox, oy) in conds]
    n, m = len(mono), len(conds)
    if m == n:
        I = [[F(int(i == j)) for j in range(m)] for i in range(m)]
        return mono, solve(A, I)
    # KKT: [Ar^T Ar  c; c^T 0] [x; lam] = [Ar^T e_r ; e_0]
    K = [[sum(A[r][i] * A[r][k] for r in range(1, m)) for k in range(n)] + [A[0][i]] for i in range(n)]
    K.append([A[0][k] for k in range(n)] + [F(0)])
    R = [[(A[r][i] if r >= 1 else F(0)) for r in range(m)] for i in range(n)]
    R.append([F(int(r == 0)) for r in range(m)])
    X = solve(K, R)
    return mono, X[:n]


LBL = {1: (-1, -1), 2: (0, -1), 3: (1, -1), 4: (-1, 0), 5: (0, 0), 6: (1, 0), 7: (-1, 1), 8: (0, 1), 9: (1, 1)}


def conds_1d():
    u = [(0, -1, 0), (0, 0, 0), (0, 1, 0)]
    v = [(1, -1, 0), (1, 0, 0), (1, 1, 0)]
    d4 = u + v                                  # data order of the kernels
    return {2: [u[1], u[0], u[2]], 3: [u[1], u[0], u[2], v[1]], 4: [u[1], u[0], u[2], v[0], v[1], v[2]]}, d4


def conds_2d():
    u = [(0,) + LBL[k] for k in range(1, 10)]
    vx = [(1,) + LBL[k] for k in (1, 3, 4, 5, 6, 7, 9)]
    wy = [(2,) + LBL[k] for k in (1, 2, 3, 5, 7, 8, 9)]
    d4 = u + vx + wy                            # 23 data of q_4; q_3 uses u + v5 + w5; q_2 uses u
    first = [(0, 0, 0)]
    others = [c for c in u if c != (0, 0, 0)]
    return {2: first + others, 3: first + others + [(1, 0, 0), (2, 0, 0)],
            4: first + others + vx + wy}, d4


def to_d4(dim, conds, M, d4):
    """Re-index a coefficient map from the level's condition order to d4 order."""
    idx = [d4.index(c) for c in conds]
    out = [[F(0)] * len(d4) for _ in M]
    for i, row in enumerate(M):
        for r, v in enumerate(row):
            out[i][idx[r]] += v
    return out


def gram(dim, kappa):
    """Gram matrix over the non-constant monomials of degree <= kappa."""
    mono = [mm for mm in monomials(dim, kappa) if mm != (0, 0)]

    def dcoef(a, k):
        f = 1
        for t in range(k):
            f *= (a - t)
        return f

    def mixed(m1, m2):
        s = F(0)
        for t in range(1, kappa + 1):
            for ay in range(0, (t if dim == 2 else 0) + 1):
                ax = t - ay
                (a1, b1), (a2, b2) = m1, m2
                if a1 < ax or a2 < ax or b1 < ay or b2 < ay:
                    continue
                c = dcoef(a1, ax) * dcoef(b1, ay) * dcoef(a2, ax) * dcoef(b2, ay)
                s += c * cell_int(a1 - ax + a2 - ax, 0) * cell_int(b1 - ay + b2 - ay, 0)
        return s
    return mono, [[mixed(m1, m2) for m2 in mono] for m1 in mono]


def ldl_root(Gm):
    """G = L diag(D) L^T exactly; returns R = sqrt(D) L^T in Decimal."""
    n = len(Gm)
    L = [[F(0)] * n for _ in range(n)]
    D = [F(0)] * n
    for j in range(n):
        D[j] = Gm[j][j] - sum(L[j][k] ** 2 * D[k] for k in range(j))
        L[j][j] = F(1)
        for i in range(j + 1, n):
            L[i][j] = (Gm[i][j] - sum(L[i][k] * L[j][k] * D[k] for k in range(j))) / D[j]
    assert all(d > 0 for d in D)
    dec = lambda q: decimal.Decimal(q.numerator) / decimal.Decimal(q.denominator)
    return [[dec(D[r]).sqrt() * dec(L[c][r]) for c in range(n)] for r in range(n)]


def dfmt(x):
    v = float(x)
    return repr(v) if v != 0.0 else "0.0"


def ffmt(x):
    """Round to binary32 (via the correctly rounded double) and print exactly."""
    v = struct.unpack("f", struct.pack("f", float(x)))[0]
    return (repr(v) + "f") if v != 0.0 else "0.0f"


def emit_matrix(qual, name, rows, ctype="double"):
    r, c = len(rows), len(rows[0])
    fmt = dfmt if ctype == "double" else ffmt
    body = ",\n".join("  {" + ", ".join(fmt(v) for v in row) + "}" for row in rows)
    return f"{qual} {ctype} {name}[{r}][{c}] = {{\n{body}}};\n"


def level_columns(dim, d4):
    """Positions in d4 of the data each level uses (d2 subset d3 subset d4)."""
    if dim == 1:
        return {2: [0, 1, 2], 3: [0, 1, 2, 4], 4: list(range(6))}
    return {2: list(range(9)), 3: list(range(9)) + [d4.index((1, 0, 0)), d4.index((2, 0, 0))],
            4: list(range(23))}


def build(dim):
    conds, d4 = conds_1d() if dim == 1 else conds_2d()
    deg = {2: 2, 3: 3, 4: 5}
    C = {}
    V = {}
    pts = [(k, 0) for k in range(4)] if dim == 1 else [(k, l) for k in range(4) for l in range(4)]
    for lvl in (2, 3, 4):
        mono, M = level_matrix(dim, deg[lvl], conds[lvl])
        M4 = to_d4(dim, conds[lvl], M, d4)
        C[lvl] = (mono, M4)
        vals = []
        for (k, l) in pts:
            row = [Q5(0)] * len(d4)
            for i, (a, b) in enumerate(mono):
                e = qpow(NODES[k], a) * (qpow(NODES[l], b) if dim == 2 else Q5(1))
                for d in range(len(d4)):
                    if M4[i][d] != 0:
                        row[d] = row[d] + e * M4[i][d]
            vals.append([x.to_decimal() for x in row])
        V[lvl] = vals
    # indicator rows: beta of a degree-kappa polynomial from its non-constant coefficients
    RC = {}
    for lvl, kap in ((2, 2), (3, 3), (4, 5)):
        gmono, Gm = gram(dim, kap)
        R = ldl_root(Gm)
        for src in (lvl, lvl - 1):
            if src < 2:
                continue
            mono, M4 = C[src]
            coef = {m: M4[i] for i, m in enumerate(mono)}
            Cm = [coef.get(m, [F(0)] * len(d4)) for m in gmono]
            rows = []
            for r in range(len(gmono)):
                rows.append([sum((R[r][c] * (decimal.Decimal(Cm[c][d].numerator) / decimal.Decimal(Cm[c][d].denominator))
                                  for c in range(len(gmono)) if Cm[c][d] != 0), decimal.Decimal(0))
                             for d in range(len(d4))])
            RC[(lvl, src)] = rows
    return d4, V, RC


def main(out=sys.stdout):
    w = out.write
    w("// Generated by gen_tables.py from exact rational arithmetic; do not edit.\n")
    w("// Scaled coordinates xi = (x - x_i)/dx, eta = (y - y_j)/dy; Gauss-Lobatto nodes\n")
    w("// (-1/2, -sqrt5/10, sqrt5/10, 1/2) (eq. (F)); 2D points ordered [k*4 + l] for (xi_k, eta_l).\n")
    w("//\n// The includer defines HWT_VALUE_QUAL (e.g. `static __constant__` in kernels,\n")
    w("// `static const` on the host); the indicator rows are host-only.\n")
    w("#pragma once\n\nnamespace hwt {\n\n")
    for dim in (1, 2):
        d4, V, RC = build(dim)
        cols = level_columns(dim, d4)
        tag = f"D{dim}"
        w(f"// {dim}D data vector d4 (kernel gather order): " +
          ", ".join(("u" if k == 0 else "v" if k == 1 else "w") + f"({ox},{oy})" for (k, ox, oy) in d4) + "\n")
        for lvl in (2, 3, 4):
            w(f"// q_{lvl} uses d4 positions {cols[lvl]}\n")
        w(f"static const int {tag}_N2 = {len(cols[2])}, {tag}_N3 = {len(cols[3])}, {tag}_N4 = {len(cols[4])};\n")
        w(f"static const int {tag}_I3[{len(cols[3])}] = {{{', '.join(map(str, cols[3]))}}};\n")
        for lvl in (2, 3, 4):
            w(emit_matrix("HWT_VALUE_QUAL", f"{tag}_V{lvl}", [[row[c] for c in cols[lvl]] for row in V[lvl]]))
        for lvl in (2, 3, 4):
            w(emit_matrix("HWT_VALUE_QUAL", f"{tag}_V{lvl}f", [[row[c] for c in cols[lvl]] for row in V[lvl]],
                          ctype="float"))
        w("#ifdef HWT_WITH_INDICATOR_ROWS\n")
        for (lvl, src), rows in sorted(RC.items()):
            w(emit_matrix("static const", f"{tag}_RC{lvl}_{src}", rows))
        w("#endif\n\n")
    w("}  // namespace hwt\n")


if __name__ == "__main__":
    main()
