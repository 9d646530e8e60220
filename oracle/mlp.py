"""CPU FP64 reference of the learned troubled-cell indicator (test infrastructure).

TEST INFRASTRUCTURE ONLY (like the rest of oracle/): it checks the GPU feature,
forward and backward kernels; the library never calls it.

Features (108 per cell): for each of the 4 conserved variables of 2D Euler and
each cell k of the 3x3 neighbourhood (boundary images as in the scheme:
periodic wrap, or mirror with the mirrored first moment negated and, at a
reflective wall, the wall-normal momentum negated), the triple
(ubar_k - ubar_c, vbar_k, wbar_k) / D with
    D = max_k |ubar_k - ubar_c| + h^2 max_k |ubar_k| + 1e-12,
h = dx, except that the centre's own (always zero) average slot carries
ubar_c / (max_k |ubar_k| + 1e-12); all clipped to [-8, 8].  The h^2 max|u| term
is KXRCF's own scale (eq. (KXRCF_): jumps against h^2 times the norm), so that
variations far below it read as flat.  Order: var, moment (ubar, vbar, wbar),
label 1..9.

Network: 108 -> 64 -> 64 -> 1, GELU (0.5 x (1 + erf(x / sqrt 2))) hidden units,
sigmoid output.  Parameters (flat, float): W1[64][108], b1[64], W2[64][64],
b2[64], W3[64], b3[1].  The GPU runs the contractions in BF16 with FP32
accumulation; `bf16=True` here rounds the inputs, weights and hidden activations
to BF16 the same way so that only the accumulation order differs.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

NIN, NH = 108, 64
SIZES = [("W1", (NH, NIN)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)), ("W3", (NH,)), ("b3", (1,))]
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)
CLIP = 8.0


def unpack(theta):
    out, o = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = np.asarray(theta[o:o + n], dtype=np.float64).reshape(shape)
        o += n
    return out


def init(seed=0):
    rng = np.random.default_rng(seed)
    th = []
    for name, shape in SIZES:
        if name.startswith("W"):
            fan_in = shape[-1] if len(shape) == 2 else NH
            th.append(rng.normal(0.0, math.sqrt(2.0 / fan_in), size=shape).ravel())
        else:
            th.append(np.zeros(int(np.prod(shape))))
    return np.concatenate(th).astype(np.float32)


def bf16(x):
    """Round to bfloat16 (nearest, ties to even) and back to float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def _image(i, n, kind):
    """(image index, mirror sign, wall flag) of index i under boundary kind."""
    if 0 <= i < n:
        return i, 1, False
    if kind == "periodic":
        return i % n, 1, False
    return ((-1 - i) if i < 0 else (2 * n - 1 - i)), -1, kind == "reflective"


def features(m, cells, bc, h):
    """m: state [4][3][ny][nx]; cells: flat indices j*nx+i; bc: 4 kinds; h = dx."""
    nv, _, ny, nx = m.shape
    out = np.zeros((len(cells), NIN))
    for r, c in enumerate(cells):
        i, j = c % nx, c // nx
        for v in range(nv):
            vals = np.zeros((3, 9))
            for oy in (-1, 0, 1):
                jj, sy, wy = _image(j + oy, ny, bc[2] if j + oy < 0 else bc[3])
                for ox in (-1, 0, 1):
                    ii, sx, wx = _image(i + ox, nx, bc[0] if i + ox < 0 else bc[1])
                    k = (oy + 1) * 3 + ox + 1
                    g = -1.0 if (v == 1 and wx) or (v == 2 and wy) else 1.0   # wall: normal momentum negated
                    vals[0, k] = g * m[v, 0, jj, ii]
                    vals[1, k] = g * sx * m[v, 1, jj, ii]
                    vals[2, k] = g * sy * m[v, 2, jj, ii]
            u0 = vals[0, 4]
            umax = np.max(np.abs(vals[0]))
            D = np.max(np.abs(vals[0] - u0)) + h * h * umax + 1e-12
            f = np.concatenate([(vals[0] - u0) / D, vals[1] / D, vals[2] / D])
            f[4] = u0 / (umax + 1e-12)
            out[r, v * 27:(v + 1) * 27] = np.clip(f, -CLIP, CLIP)
    return out


def forward(theta, X, bf=True):
    P = unpack(theta)
    rnd = bf16 if bf else (lambda a: np.asarray(a, np.float64))
    x = rnd(X)
    a1 = x @ rnd(P["W1"]).T + P["b1"]
    h1 = rnd(gelu(a1))
    a2 = h1 @ rnd(P["W2"]).T + P["b2"]
    h2 = gelu(a2)
    z = h2 @ P["W3"] + P["b3"][0]
    return z, dict(x=x, a1=a1, h1=h1, a2=a2, h2=h2)


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def loss_grad(theta, X, y, w=None, bf=True):
    """Mean weighted BCE of sigmoid(z) and its gradient w.r.t. the parameters.
    With bf=False this is the exact derivative of the FP64 forward."""
    P = unpack(theta)
    n = X.shape[0]
    w = np.ones(n) if w is None else np.asarray(w, np.float64)
    z, c = forward(theta, X, bf)
    p = sigmoid(z)
    eps = 1e-12
    loss = -np.sum(w * (y * np.log(p + eps) + (1 - y) * np.log(1 - p + eps))) / n
    dz = w * (p - y) / n
    rnd = bf16 if bf else (lambda a: np.asarray(a, np.float64))
    g = {}
    g["W3"] = c["h2"].T @ dz
    g["b3"] = np.array([dz.sum()])
    da2 = np.outer(dz, P["W3"]) * gelu_grad(c["a2"])
    g["b2"] = da2.sum(0)
    # with bf, the tensor-core operands of the three backward contractions
    # (da2, da1 and W2) are BF16-rounded as on the GPU; bias sums are not.
    g["W2"] = rnd(da2).T @ c["h1"]
    dh1 = rnd(da2) @ rnd(P["W2"])
    da1 = dh1 * gelu_grad(c["a1"])
    g["W1"] = rnd(da1).T @ c["x"]
    g["b1"] = da1.sum(0)
    flat = np.concatenate([g[name].ravel() for name, _ in SIZES])
    return loss, flat
