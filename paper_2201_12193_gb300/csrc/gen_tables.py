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

Run:  python gen_tables.py > hweno_parity.h

The plain tables (build()) are kept for the checks against the oracle; the
kernels use the mirror-parity form derived from them (build_parity(),
emit_parity()).
"""
from __future__ import annotations

import decimal
import math
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


def _exact(dim):
    """Exact pieces shared by both emitters: data order d4, per level the
    monomials and coefficient maps (Fractions, over d4), and the value rows at
    the Gauss-Lobatto points (Q5)."""
    conds, d4 = conds_1d() if dim == 1 else conds_2d()
    deg = {2: 2, 3: 3, 4: 5}
    C, VQ = {}, {}
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
            vals.append(row)
        VQ[lvl] = vals
    return d4, C, VQ, pts


def _dec(q):
    return decimal.Decimal(q.numerator) / decimal.Decimal(q.denominator)


def build(dim):
    d4, C, VQ, _ = _exact(dim)
    V = {lvl: [[x.to_decimal() for x in row] for row in rows] for lvl, rows in VQ.items()}
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
                rows.append([sum((R[r][c] * _dec(Cm[c][d]) for c in range(len(gmono)) if Cm[c][d] != 0),
                                 decimal.Decimal(0)) for d in range(len(d4))])
            RC[(lvl, src)] = rows
    return d4, V, RC


# ---------------------------------------------------------------- mirror-parity form
#
# The stencils, the conditions of every q_l and the Gauss-Lobatto points are
# symmetric under the mirrors x -> -x and y -> -y, under which the first moment
# in the mirrored direction changes sign.  The data then split into parity
# classes c = (px, py) (even/odd under each mirror), every coefficient of a
# monomial xi^a eta^b is a functional of the class (a mod 2, b mod 2) only, and
# a point value at (s_x xi, s_y eta) is sum_c s_x^px s_y^py E_c(xi, eta).  The
# kernels evaluate the same reconstruction in this basis: the same numbers up to
# rounding, with about a third of the multiply-adds.

def mirror_group(dim, d4):
    """Signed permutations (perm, sign, (mx, my)): (g d)[p] = sign[p] * d[perm[p]]."""
    out = []
    for mx in (0, 1):
        for my in ((0, 1) if dim == 2 else (0,)):
            perm, sign = [], []
            for (k, ox, oy) in d4:
                q = d4.index((k, -ox if mx else ox, -oy if my else oy))
                sg = (-1 if (mx and k == 1) else 1) * (-1 if (my and k == 2) else 1)
                perm.append(q)
                sign.append(sg)
            out.append((perm, sign, (mx, my)))
    return out


def parity_classes(dim):
    return [(0, 0), (1, 0)] if dim == 1 else [(0, 0), (1, 0), (0, 1), (1, 1)]


def parity_basis(dim, d4):
    """Per class: orthogonal integer rows r (over d4) spanning the class; s_j = r_j . d."""
    G = mirror_group(dim, d4)
    basis = {}
    for c in parity_classes(dim):
        rows = []
        for p in range(len(d4)):
            r = [0] * len(d4)
            for perm, sign, (mx, my) in G:
                chi = (-1) ** (c[0] * mx + c[1] * my)
                r[perm[p]] += chi * sign[p]
            if not any(r):
                continue
            g = 0
            for v in r:
                g = math.gcd(g, abs(v))
            r = [v // g for v in r]
            first = next(v for v in r if v)
            if first < 0:
                r = [-v for v in r]
            if r not in rows:
                rows.append(r)
        basis[c] = rows
    allr = [r for c in parity_classes(dim) for r in basis[c]]
    assert len(allr) == len(d4)
    for i in range(len(allr)):
        for j in range(i + 1, len(allr)):
            assert sum(a * b for a, b in zip(allr[i], allr[j])) == 0
    return basis


def over_class(f, rows):
    """Coefficients g of the class projection of functional f: (f P_c) d = sum_j g_j s_j."""
    return [sum((F(a) * b for a, b in zip(r, f)), F(0)) / sum(a * a for a in r) if not isinstance(f[0], Q5)
            else _q5_over(f, r) for r in rows]


def _q5_over(f, r):
    n = sum(a * a for a in r)
    acc = Q5(0)
    for a, b in zip(r, f):
        if a:
            acc = acc + b * F(a, n)
    return acc


def build_parity(dim):
    d4, C, VQ, pts = _exact(dim)
    basis = parity_basis(dim, d4)
    classes = parity_classes(dim)
    # class slices of s
    order = [(c, j) for c in classes for j in range(len(basis[c]))]
    sl = {}
    pos = 0
    for c in classes:
        sl[c] = list(range(pos, pos + len(basis[c])))
        pos += len(basis[c])
    # base points: positive coordinates (k, l in {2, 3}); mirror image of index k is 3 - k
    bases = [(k, 0) for k in (2, 3)] if dim == 1 else [(k, l) for k in (2, 3) for l in (2, 3)]
    VP = {}
    for lvl in (2, 3, 4):
        for b in bases:
            for c in classes:
                VP[(lvl, b, c)] = _over_q5_rows(VQ[lvl][pts.index(b)], basis[c])
        # identity check: every mirrored point is reproduced
        for b in bases:
            for sx in (1, -1):
                for sy in ((1, -1) if dim == 2 else (1,)):
                    k = b[0] if sx > 0 else 3 - b[0]
                    l = b[1] if (dim == 1 or sy > 0) else 3 - b[1]
                    want = VQ[lvl][pts.index((k, l))]
                    got = [Q5(0) for _ in d4]
                    for c in classes:
                        chi = (sx if c[0] else 1) * (sy if c[1] else 1)
                        for g, r in zip(VP[(lvl, b, c)], basis[c]):
                            for d in range(len(d4)):
                                if r[d]:
                                    got[d] = got[d] + g * (chi * r[d])
                    assert all(a.a == w.a and a.b == w.b for a, w in zip(got, want)), (lvl, b, sx, sy)
    # smoothness-indicator rows per class: R_c C_{l,c} over s_c
    RCP = {}
    for lvl, kap in ((2, 2), (3, 3), (4, 5)):
        gmono, Gm = gram(dim, kap)
        for c in classes:
            idx = [i for i, m in enumerate(gmono) if (m[0] % 2, m[1] % 2) == c]
            if not idx:
                continue
            Gc = [[Gm[i][j] for j in idx] for i in idx]
            R = ldl_root(Gc)
            for src in (lvl, lvl - 1):
                if src < 2:
                    continue
                mono, M4 = C[src]
                coef = {m: M4[i] for i, m in enumerate(mono)}
                Cc = [coef.get(gmono[i], [F(0)] * len(d4)) for i in idx]
                for row in Cc:          # each class-c coefficient is a class-c functional
                    for c2 in classes:
                        if c2 != c:
                            assert all(v == 0 for v in over_class(row, basis[c2]))
                Cs = [over_class(row, basis[c]) for row in Cc]
                RCP[(lvl, src, c)] = [[sum((R[r][k] * _dec(Cs[k][j]) for k in range(len(idx)) if Cs[k][j] != 0),
                                           decimal.Decimal(0)) for j in range(len(basis[c]))] for r in range(len(idx))]
    return d4, basis, sl, bases, VP, RCP


def _over_q5_rows(vrow, rows):
    return [_q5_over(vrow, r) for r in rows]


def _lit(x):
    v = float(x)
    return repr(v)


def beta_layout(dim, P):
    """Flat layout of the run-time indicator rows: for levels 2, 3, 4, class, row,
    the s indices used (union of the q_l and q_{l-1} patterns) and the two
    coefficient rows (q_l part, q_{l-1} part)."""
    d4, basis, sl, bases, VP, RCP = P
    lay = {}
    for lvl in (2, 3, 4):
        ent = []
        for c in parity_classes(dim):
            if (lvl, lvl, c) not in RCP:
                continue
            A = RCP[(lvl, lvl, c)]
            Bm = RCP.get((lvl, lvl - 1, c))
            for r in range(len(A)):
                cols = [j for j in range(len(basis[c])) if A[r][j] != 0 or (Bm is not None and Bm[r][j] != 0)]
                ent.append([(sl[c][j], A[r][j], Bm[r][j] if Bm is not None else decimal.Decimal(0)) for j in cols])
        lay[lvl] = ent
    return lay


def flop_count(dim):
    """Floating-point operations of split + beta_2..4 + values for one variable,
    as emitted (fma = 2, add/mul = 1; value expressions that repeat are counted once)."""
    P = build_parity(dim)
    d4, basis, sl, bases, VP, RCP = P
    classes = parity_classes(dim)
    n = sum(sum(1 for a in r if a) - 1 for c in classes for r in basis[c])          # split
    for lvl, ents in beta_layout(dim, P).items():                                    # beta
        for ent in ents:
            n += 2 * len(ent) - 1 + 2
    n += 1                                                                           # K = c1 u0
    for b in bases:
        seen = set()
        for cl in classes:
            levels = 0
            for lvl in (2, 3, 4):
                terms = tuple((sl[cl][j], str(g.to_decimal())) for j, g in enumerate(VP[(lvl, b, cl)])
                              if (g.a != 0 or g.b != 0))
                if not terms:
                    continue
                levels += 1
                if terms not in seen:
                    seen.add(terms)
                    n += 2 * len(terms) - 1
            n += 2 * levels - 1                                                      # E_c
        n += 3 if dim == 1 else 9                                                    # butterflies
    return n


def emit_parity(out):
    w = out.write
    w("// Generated by gen_tables.py (mirror-parity form); do not edit.\n")
    w("// Reconstruction of one variable in the parity basis s of the stencil data:\n")
    w("// split (d -> s), smoothness indicators beta_2..beta_4 from run-time rows, and the\n")
    w("// Gauss-Lobatto values u = c1 q1 + c2 q2 + c3 q3 + c4 q4 at all points.\n")
    w("#pragma once\n\nnamespace hwp {\n\n")
    host = []
    for dim in (1, 2):
        P = build_parity(dim)
        d4, basis, sl, bases, VP, RCP = P
        classes = parity_classes(dim)
        n = len(d4)
        tag = f"D{dim}"
        lay = beta_layout(dim, P)
        for lvl in (2, 3, 4):
            w(f"constexpr int {tag}_NB{lvl} = {sum(len(e) for e in lay[lvl])};\n")
        w(f"// floating-point operations of split + beta + values per variable, as emitted\n")
        w(f"constexpr int {tag}_FLOP_SBV = {flop_count(dim)};\n")
        # split
        w(f"\n// s = parity combinations of d ({n} data; classes {classes} -> slices "
          + ", ".join(f"{c}:{sl[c][0]}..{sl[c][-1]}" for c in classes) + ")\n")
        w(f"template <typename T>\n__device__ __forceinline__ void split{dim}d(const T (&d)[{n}], T (&s)[{n}]) {{\n")
        for c in classes:
            for j, r in enumerate(basis[c]):
                terms = []
                for q, a in enumerate(r):
                    if a:
                        terms.append(("+" if a > 0 else "-") + (f"d[{q}]" if abs(a) == 1 else f"T({abs(a)}) * d[{q}]"))
                expr = " ".join(terms).lstrip("+ ").replace("+", "+ ").replace("-", "- ") if terms else "T(0)"
                if expr.startswith("- "):
                    expr = "-" + expr[2:]
                w(f"  s[{sl[c][j]}] = {expr};\n")
        w("}\n\n")
        # beta
        w(f"template <typename T>\n__device__ __forceinline__ void beta{dim}d(const T* __restrict__ B2, "
          f"const T* __restrict__ B3, const T* __restrict__ B4, const T (&s)[{n}], T& b2, T& b3, T& b4) {{\n")
        w("  T r;\n")
        for lvl in (2, 3, 4):
            w(f"  b{lvl} = T(0);\n")
            k = 0
            for ent in lay[lvl]:
                first = True
                for (j, _, _) in ent:
                    if first:
                        w(f"  r = B{lvl}[{k}] * s[{j}];")
                        first = False
                    else:
                        w(f" r = fma(B{lvl}[{k}], s[{j}], r);")
                    k += 1
                w(f" b{lvl} = fma(r, r, b{lvl});\n")
        w("}\n\n")
        # values
        npt = 4 if dim == 1 else 16
        w(f"template <typename T>\n__device__ __forceinline__ void values{dim}d(const T (&s)[{n}], T u0, "
          f"const T (&c)[4], T (&out)[{npt}]) {{\n")
        w("  const T K = c[0] * u0;\n")
        for b in bases:
            w("  {\n")
            E = []
            for ci, cl in enumerate(classes):
                parts = []
                for lvl in (2, 3, 4):
                    coefs = VP[(lvl, b, cl)]
                    terms = [(sl[cl][j], g.to_decimal()) for j, g in enumerate(coefs) if (g.a != 0 or g.b != 0)]
                    if not terms:
                        continue
                    expr = f"T({_lit(terms[0][1])}) * s[{terms[0][0]}]"
                    for (j, v) in terms[1:]:
                        expr = f"fma(T({_lit(v)}), s[{j}], {expr})"
                    w(f"    const T q{lvl}_{ci} = {expr};\n")
                    parts.append(lvl)
                e = f"c[{parts[0] - 1}] * q{parts[0]}_{ci}"
                for lvl in parts[1:]:
                    e = f"fma(c[{lvl - 1}], q{lvl}_{ci}, {e})"
                w(f"    const T E{ci} = {e};\n")
            if dim == 1:
                k = b[0]
                w("    const T A = K + E0;\n")
                w(f"    out[{k}] = A + E1;\n    out[{3 - k}] = A - E1;\n")
            else:
                k, l = b
                pp, mp, pm, mm = k * 4 + l, (3 - k) * 4 + l, k * 4 + (3 - l), (3 - k) * 4 + (3 - l)
                w("    const T A = K + E0;\n    const T P = A + E2, Q = E1 + E3, R = A - E2, S = E1 - E3;\n")
                w(f"    out[{pp}] = P + Q;\n    out[{mp}] = P - Q;\n    out[{pm}] = R + S;\n    out[{mm}] = R - S;\n")
            w("  }\n")
        w("}\n\n")
        for lvl in (2, 3, 4):
            flat = [e for ent in lay[lvl] for e in ent]
            host.append(f"static const double {tag}P_RC{lvl}_{lvl}[{len(flat)}] = {{" +
                        ", ".join(_lit(a) for (_, a, _) in flat) + "};\n")
            host.append(f"static const double {tag}P_RC{lvl}_{lvl - 1}[{len(flat)}] = {{" +
                        ", ".join(_lit(b) for (_, _, b) in flat) + "};\n")
    w("}  // namespace hwp\n\n")
    w("#ifdef HWP_HOST_TABLES\n// Host: coefficient rows in the flat order the beta functions read them;\n")
    w("// B_l = (S_l/g_l) RC_l_l - (S_{l-1}/g_l) RC_l_(l-1)  (eq. (p)), or RC_l_l alone for beta of q_l.\n")
    w("namespace hwp {\n")
    for h in host:
        w(h)
    w("}  // namespace hwp\n#endif\n")


if __name__ == "__main__":
    emit_parity(sys.stdout)
