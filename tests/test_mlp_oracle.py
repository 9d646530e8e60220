"""CPU pins of the learned-indicator reference (oracle/mlp.py) and of the
oracle's given-decision mode (indicator 3).

* Backward: the FP64 gradient against central finite differences of the FP64
  loss (relative 1e-6), every parameter block.
* BF16 rounding against torch's own float -> bfloat16 conversion.
* GELU: the identity gelu(x) - gelu(-x) = x, Phi(1) from the normal table,
  and gelu' against finite differences.
* Features: invariance under scaling a variable (and the sign rule under a
  negative scale), shift invariance at h = 0, the closed form on a linear
  field, flatness below the KXRCF scale h^2 max|u|, the mirror image at a
  transmissive boundary, and the clip.
* Indicator 3 of the oracle reduces to indicators 0, 1 and 2 for the decisions
  that mean the same thing (all 0, the KXRCF flags or all 2, all 1).
"""
from __future__ import annotations

import math

import numpy as np
import pytest

from oracle import mlp


def _theta64(seed):
    return mlp.init(seed).astype(np.float64)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    n = 9
    X = rng.normal(0, 1.5, (n, mlp.NIN))
    y = (rng.random(n) < 0.4).astype(np.float64)
    w = rng.uniform(0.5, 2.0, n)
    th = _theta64(1)
    th[mlp.NPARAM - 1] = 0.3                 # b3
    _, g = mlp.loss_grad(th, X, y, w, bf=False)
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in mlp.SIZES])
    idx = []
    for b in range(len(mlp.SIZES)):
        lo, hi = offs[b], offs[b + 1]
        idx += list(rng.choice(np.arange(lo, hi), size=min(12, hi - lo), replace=False))
    h = 1e-5
    for q in idx:
        tp, tm = th.copy(), th.copy()
        tp[q] += h
        tm[q] -= h
        fd = (mlp.loss_grad(tp, X, y, w, bf=False)[0] - mlp.loss_grad(tm, X, y, w, bf=False)[0]) / (2 * h)
        assert abs(fd - g[q]) <= 1e-6 * max(abs(g[q]), 1e-3 * np.max(np.abs(g))), (q, fd, g[q])


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    x = np.concatenate([rng.normal(0, 3, 4000), rng.normal(0, 1e-3, 1000),
                        # exact ties (halfway between two bf16 values) in both parities
                        np.array([1 + 2 ** -8, 1 + 3 * 2 ** -8, -(1 + 2 ** -8), 2 ** -8 + 2 ** -16, 0.0, -0.0])])
    x = x.astype(np.float32)
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(mlp.bf16(x), want)


def test_gelu_pins():
    x = np.linspace(-6, 6, 241)
    np.testing.assert_allclose(mlp.gelu(x) - mlp.gelu(-x), x, rtol=0, atol=1e-14)
    assert abs(mlp.gelu(1.0) - 0.8413447460685429) < 1e-15          # Phi(1)
    h = 1e-6
    np.testing.assert_allclose(mlp.gelu_grad(x), (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h), atol=1e-8)


def _rand_state(rng, ny, nx):
    m = rng.normal(0, 1, (4, 3, ny, nx))
    m[:, 0] += 3.0
    return m


def test_features_invariances():
    rng = np.random.default_rng(5)
    ny, nx = 7, 9
    m = _rand_state(rng, ny, nx)
    cells = np.arange(nx * ny)
    bc = ("transmissive",) * 4
    h = 0.05
    f0 = mlp.features(m, cells, bc, h)
    m2 = m.copy()
    m2[1] *= 3.5                                  # one variable scaled: its features unchanged
    np.testing.assert_allclose(mlp.features(m2, cells, bc, h), f0, atol=1e-9)
    m2[3] *= -2.0                                 # sign flip: only the centre slot changes sign
    f2 = mlp.features(m2, cells, bc, h)
    np.testing.assert_allclose(f2[:, 81 + 4], -f0[:, 81 + 4], atol=1e-9)
    np.testing.assert_allclose(np.delete(f2[:, 81:], 4, axis=1), -np.delete(f0[:, 81:], 4, axis=1), atol=1e-9)
    assert np.all(np.abs(f0) <= mlp.CLIP)
    # with h = 0 and a constant added to a positive variable's averages, only
    # the centre slot changes
    m1 = m.copy()
    m1[0, 0] += 17.0
    fa, fb = mlp.features(m, cells, bc, 0.0), mlp.features(m1, cells, bc, 0.0)
    np.testing.assert_allclose(np.delete(fb, 4, axis=1), np.delete(fa, 4, axis=1), atol=1e-12)


def test_features_linear_field_and_mirror():
    ny, nx = 6, 8
    m = np.zeros((4, 3, ny, nx))
    jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    m[0, 0] = 2.0 * ii + 0.5 * jj                 # linear averages: D = 2 + 0.5
    m[0, 1] = 0.25
    cell = 3 * nx + 4                             # interior: averages 9.5 + 2 ox + 0.5 oy
    h = 0.1
    f = mlp.features(m, [cell], ("periodic",) * 4, h)[0]
    D = 2.5 + h * h * 12.0
    for oy in (-1, 0, 1):
        for ox in (-1, 0, 1):
            k = (oy + 1) * 3 + ox + 1
            want = 9.5 / 12.0 if k == 4 else (2.0 * ox + 0.5 * oy) / (D + 1e-12)
            assert f[k] == pytest.approx(want, abs=1e-12)
            assert f[9 + k] == pytest.approx(0.25 / (D + 1e-12), abs=1e-12)
    assert np.all(f[27:] == 0.0)                  # other variables identically zero
    # variations far below h^2 max|u| read as flat
    m2 = m.copy()
    m2[0, 0] = 1e3 + 1e-6 * ii
    assert np.all(np.abs(mlp.features(m2, [cell], ("periodic",) * 4, h)[0][[3, 5]]) < 1e-6)
    # transmissive left boundary: the x-image of the cell left of column 0 is
    # column 0 itself with its x first moment negated
    f = mlp.features(m, [3 * nx], ("transmissive",) * 4, h)[0]
    for oy in (-1, 0, 1):
        kl, kc = (oy + 1) * 3, (oy + 1) * 3 + 1
        if kc != 4:
            assert f[kl] == pytest.approx(f[kc], abs=1e-12)
        assert f[9 + kl] == pytest.approx(-f[9 + kc], abs=1e-12)
    # clip: a large first moment
    m[0, 1, 3, 4] = 1e6
    assert mlp.features(m, [cell], ("periodic",) * 4, h)[0][9 + 4] == mlp.CLIP


def test_given_decisions_reduce_to_the_plain_indicators(orc):
    from paper_2201_12193_gb300 import workloads as W
    p = W.four_quadrant_2d(24, seed=2, ny=20)
    kw = dict(dx=p.dx, dy=p.dy, eq="euler", gamma=p.gamma, bc=p.bc)
    c_kx = orc.make_cfg(2, p.nx, p.ny, indicator="kxrcf", **kw)
    c_gv = orc.make_cfg(2, p.nx, p.ny, indicator="given", **kw)
    Um1, L1, mask1, al1, rc = orc.rhs(c_kx, p.m)
    assert rc == 0 and mask1.sum() > 0
    nc = p.nx * p.ny
    for dec in (np.full(nc, 2, np.uint8), mask1.copy()):
        Um3, L3, mask3, _, rc = orc.rhs(c_gv, p.m, decisions=dec)
        assert rc == 0
        np.testing.assert_array_equal(mask3, mask1)
        np.testing.assert_array_equal(L3, L1)
        np.testing.assert_array_equal(Um3, Um1)
    for val, ind in ((1, "all"), (0, "none")):
        Um0, L0, mask0, _, _ = orc.rhs(orc.make_cfg(2, p.nx, p.ny, indicator=ind, **kw), p.m)
        Um3, L3, mask3, _, _ = orc.rhs(c_gv, p.m, decisions=np.full(nc, val, np.uint8))
        np.testing.assert_array_equal(mask3, mask0)
        np.testing.assert_array_equal(L3, L0)
    # a genuine mix: given flags change what KXRCF sees in the deferred cells
    dec = np.full(nc, 2, np.uint8)
    dec[np.flatnonzero(mask1)[::2]] = 1
    _, L3, mask3, _, rc = orc.rhs(c_gv, p.m, decisions=dec)
    assert rc == 0 and np.all(mask3[dec == 1] == 1)
