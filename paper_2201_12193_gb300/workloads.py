"""Seeded synthetic inputs: initial data projected onto the moment state.

This module holds no arithmetic of the HWENO method.  It only evaluates
initial conditions at Gauss-Legendre points and forms the cell moments of
eq. (1D-moment) / (2D-moment)

    ubar = (1/|I|) int_I u,   vbar = (1/|I|) int_I u (x - x_i)/dx,
    wbar = (1/|I|) int_I u (y - y_j)/dy,

with 8 Gauss-Legendre points per direction per cell.  Both the CUDA path and
the CPU oracle receive the same arrays from here.

Layout of every state: float64 array m[var][moment][j][i] (1D: j has size 1),
conserved variables (rho, rho*mu, E) in 1D Euler, (rho, rho*mu, rho*nu, E) in
2D Euler, (u,) for scalar laws.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

GAMMA = 1.4


@dataclasses.dataclass
class Problem:
    """A grid description plus its initial moments (names follow the C ABI)."""
    name: str
    dim: int
    nx: int
    ny: int
    x0: float
    x1: float
    y0: float
    y1: float
    eq: str                  # "advection" | "burgers" | "euler"
    bc: tuple                # (xlo, xhi, ylo, yhi), "periodic" | "transmissive"
    m: np.ndarray            # initial moments
    adv: tuple = (1.0, 0.0)
    gamma: float = GAMMA
    t_end: float = 0.0
    seed: int | None = None
    meta: dict = dataclasses.field(default_factory=dict)
    fixed: tuple | None = None   # per side: None or dict(a=, b=, c0=, speed=) of fixed ghost states

    @property
    def dx(self):
        return (self.x1 - self.x0) / self.nx

    @property
    def dy(self):
        return (self.y1 - self.y0) / self.ny if self.dim == 2 else 1.0

    @property
    def ncell(self):
        return self.nx * self.ny


def _gl(npts=8):
    x, w = np.polynomial.legendre.leggauss(npts)
    return 0.5 * x, 0.5 * w          # nodes on [-1/2, 1/2], weights summing to 1


def moments_1d(fun, x0, x1, nx, npts=8):
    """fun(x) -> array (nvar, ...) of conserved variables at points x."""
    s, w = _gl(npts)
    dx = (x1 - x0) / nx
    xc = x0 + (np.arange(nx) + 0.5) * dx
    X = xc[:, None] + s[None, :] * dx                 # (nx, q)
    U = np.asarray(fun(X), dtype=np.float64)          # (nvar, nx, q)
    if U.ndim == 2:
        U = U[None]
    ub = np.einsum("vnq,q->vn", U, w)
    vb = np.einsum("vnq,q->vn", U, w * s)
    return np.ascontiguousarray(np.stack([ub, vb], axis=1)[:, :, None, :])


def moments_2d(fun, x0, x1, y0, y1, nx, ny, npts=8, rows=None):
    """fun(X, Y) -> (nvar, ...); returns m[var][3][ny][nx].  Built row-block by
    row-block so that large grids stay within modest host memory."""
    s, w = _gl(npts)
    dx = (x1 - x0) / nx
    dy = (y1 - y0) / ny
    xc = x0 + (np.arange(nx) + 0.5) * dx
    yc = y0 + (np.arange(ny) + 0.5) * dy
    out = None
    step = rows or max(1, min(ny, (1 << 22) // max(1, nx * npts * npts)))
    for j0 in range(0, ny, step):
        j1 = min(ny, j0 + step)
        Y = yc[j0:j1, None, None, None] + s[None, None, None, :] * dy      # (r,1,1,q)
        X = xc[None, :, None, None] + s[None, None, :, None] * dx          # (1,n,q,1)
        U = np.asarray(fun(np.broadcast_to(X, (j1 - j0, nx, npts, npts)),
                           np.broadcast_to(Y, (j1 - j0, nx, npts, npts))), dtype=np.float64)
        if U.ndim == 4:
            U = U[None]
        if out is None:
            out = np.empty((U.shape[0], 3, ny, nx))
        out[:, 0, j0:j1] = np.einsum("vrnab,a,b->vrn", U, w, w)
        out[:, 1, j0:j1] = np.einsum("vrnab,a,b->vrn", U, w * s, w)
        out[:, 2, j0:j1] = np.einsum("vrnab,a,b->vrn", U, w, w * s)
    return np.ascontiguousarray(out)


def prim_to_cons_1d(rho, mu, p, gamma=GAMMA):
    return np.stack([rho, rho * mu, p / (gamma - 1.0) + 0.5 * rho * mu * mu])


def prim_to_cons_2d(rho, mu, nu, p, gamma=GAMMA):
    return np.stack([rho, rho * mu, rho * nu, p / (gamma - 1.0) + 0.5 * rho * (mu * mu + nu * nu)])


# ---------------------------------------------------------------- 1D inputs

def advection_sin_1d(nx=200):
    """u_t + u_x = 0 on [0, 2pi], u0 = sin x, periodic, to t = 2pi."""
    m = moments_1d(lambda x: np.sin(x), 0.0, 2 * math.pi, nx)
    return Problem("advection_sin_1d", 1, nx, 1, 0.0, 2 * math.pi, 0.0, 1.0, "advection",
                   ("periodic",) * 4, m, adv=(1.0, 0.0), t_end=2 * math.pi)


def burgers_1d(nx=200):
    """u_t + (u^2/2)_x = 0 on [0, 2], u0 = 0.5 + sin(pi x), periodic (Example 3.1)."""
    m = moments_1d(lambda x: 0.5 + np.sin(math.pi * x), 0.0, 2.0, nx)
    return Problem("burgers_1d", 1, nx, 1, 0.0, 2.0, 0.0, 1.0, "burgers", ("periodic",) * 4, m,
                   t_end=0.5 / math.pi)


def density_wave_1d(nx=200):
    """Euler, rho = 1 + 0.2 sin(pi x), mu = 1, p = 1 on [0, 2], periodic; exact: translation."""
    def f(x):
        return prim_to_cons_1d(1.0 + 0.2 * np.sin(math.pi * x), np.ones_like(x), np.ones_like(x))
    m = moments_1d(f, 0.0, 2.0, nx)
    return Problem("density_wave_1d", 1, nx, 1, 0.0, 2.0, 0.0, 1.0, "euler", ("periodic",) * 4, m,
                   t_end=2.0)


def riemann_1d(left, right, nx, x0=-0.5, x1=0.5, xs=0.0, name="riemann_1d", t_end=0.16):
    """Two constant states (rho, mu, p) split at xs, transmissive ends."""
    def f(x):
        L = x < xs
        rho = np.where(L, left[0], right[0])
        mu = np.where(L, left[1], right[1])
        p = np.where(L, left[2], right[2])
        return prim_to_cons_1d(rho, mu, p)
    m = moments_1d(f, x0, x1, nx)
    return Problem(name, 1, nx, 1, x0, x1, 0.0, 1.0, "euler", ("transmissive",) * 4, m, t_end=t_end,
                   meta={"left": left, "right": right, "xs": xs})


def lax_1d(nx=200):
    """Lax problem (Example 3.5)."""
    return riemann_1d((0.445, 0.698, 3.528), (0.5, 0.0, 0.571), nx, name="lax_1d", t_end=0.16)


def sod_1d(nx=200):
    return riemann_1d((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), nx, name="sod_1d", t_end=0.2)


def blast_wave_1d(nx=800):
    """Interacting blast waves (Example 3.7) on [0, 1], to t = 0.038: pressure
    1000 / 0.01 / 100 split at 0.1 and 0.9, rho = 1, at rest.  The paper does not
    state the boundary; reflective walls at both ends (the problem's usual
    setting).  Faces at 0.1 and 0.9 are cell faces when nx is a multiple of 10,
    so the moments are exact."""
    def f(x):
        p = np.where(x < 0.1, 1000.0, np.where(x < 0.9, 0.01, 100.0))
        return prim_to_cons_1d(np.ones_like(x), np.zeros_like(x), p)
    m = moments_1d(f, 0.0, 1.0, nx)
    return Problem("blast_wave_1d", 1, nx, 1, 0.0, 1.0, 0.0, 1.0, "euler", ("reflective",) * 4, m, t_end=0.038)


def shu_osher_1d(nx=4000):
    """Shock / density-wave interaction on [-5, 5] (Example 3.6), transmissive ends."""
    def f(x):
        L = x < -4.0
        rho = np.where(L, 3.857143, 1.0 + 0.2 * np.sin(5.0 * x))
        mu = np.where(L, 2.629369, 0.0)
        p = np.where(L, 10.3333, 1.0)
        return prim_to_cons_1d(rho, mu, p)
    m = moments_1d(f, -5.0, 5.0, nx)
    return Problem("shu_osher_1d", 1, nx, 1, -5.0, 5.0, 0.0, 1.0, "euler", ("transmissive",) * 4, m,
                   t_end=1.8)


# ---------------------------------------------------------------- 2D inputs

def advection_2d(n=32, a=1.0, b=0.5):
    """u_t + a u_x + b u_y = 0 on [0, 2pi]^2, u0 = sin(x) sin(y) + 0.5 cos(x + y), periodic."""
    m = moments_2d(lambda X, Y: np.sin(X) * np.sin(Y) + 0.5 * np.cos(X + Y),
                   0.0, 2 * math.pi, 0.0, 2 * math.pi, n, n)
    return Problem("advection_2d", 2, n, n, 0.0, 2 * math.pi, 0.0, 2 * math.pi, "advection",
                   ("periodic",) * 4, m, adv=(a, b), t_end=2 * math.pi)


def burgers_2d(n=40):
    """Example 3.2: u0 = 0.5 + sin(pi (x+y)/2) on [0,4]^2, periodic."""
    m = moments_2d(lambda X, Y: 0.5 + np.sin(math.pi * (X + Y) / 2.0), 0.0, 4.0, 0.0, 4.0, n, n)
    return Problem("burgers_2d", 2, n, n, 0.0, 4.0, 0.0, 4.0, "burgers", ("periodic",) * 4, m,
                   t_end=0.5 / math.pi)


def four_quadrant_states(seed):
    """Seeded quadrant states: rho ~ U[0.1,1.5], mu, nu ~ U[-1,1], p ~ U[0.03,1.5];
    quadrants ordered (x<0.5,y<0.5), (x>0.5,y<0.5), (x<0.5,y>0.5), (x>0.5,y>0.5)."""
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.1, 1.5, 4)
    mu = rng.uniform(-1.0, 1.0, 4)
    nu = rng.uniform(-1.0, 1.0, 4)
    p = rng.uniform(0.03, 1.5, 4)
    return rho, mu, nu, p


def four_quadrant_2d(n=2048, seed=0, ny=None):
    """2D Riemann data on [0,1]^2 split at (0.5, 0.5), transmissive, to t = 0.25.
    When n is even the split lies on cell faces and the moments are exact
    (quadrant state, zero first moments); otherwise they are integrated."""
    ny = ny or n
    rho, mu, nu, p = four_quadrant_states(seed)

    def f(X, Y):
        q = (X > 0.5).astype(np.int64) + 2 * (Y > 0.5).astype(np.int64)
        return prim_to_cons_2d(rho[q], mu[q], nu[q], p[q])
    if n % 2 == 0:
        xc = (np.arange(n) + 0.5) / n
        yc = (np.arange(ny) + 0.5) / n
        q = (xc[None, :] > 0.5).astype(np.int64) + 2 * (yc[:, None] > 0.5).astype(np.int64)
        m = np.zeros((4, 3, ny, n))
        m[:, 0] = prim_to_cons_2d(rho[q], mu[q], nu[q], p[q])
    else:
        m = moments_2d(f, 0.0, 1.0, 0.0, 1.0 * ny / n, n, ny)
    return Problem("four_quadrant_2d", 2, n, ny, 0.0, 1.0, 0.0, 1.0 * ny / n, "euler",
                   ("transmissive",) * 4, m, t_end=0.25, seed=seed,
                   meta={"rho": rho.tolist(), "mu": mu.tolist(), "nu": nu.tolist(), "p": p.tolist()})


def vortex_2d(n=128, seed=0, L=10.0, npts=8):
    """Isentropic vortex of seeded strength U[1,5] and centre uniform in [0,L]^2,
    mean flow (1,1), periodic; the distance to the centre is the periodic
    (minimum-image) one."""
    rng = np.random.default_rng(seed)
    eps = rng.uniform(1.0, 5.0)
    xc, yc = rng.uniform(0.0, L, 2)
    g = GAMMA

    def f(X, Y):
        dx = (X - xc + 0.5 * L) % L - 0.5 * L
        dy = (Y - yc + 0.5 * L) % L - 0.5 * L
        r2 = dx * dx + dy * dy
        e = np.exp(0.5 * (1.0 - r2))
        mu = 1.0 - eps / (2 * math.pi) * e * dy
        nu = 1.0 + eps / (2 * math.pi) * e * dx
        T = 1.0 - (g - 1.0) * eps * eps / (8.0 * g * math.pi ** 2) * e * e
        rho = T ** (1.0 / (g - 1.0))
        return prim_to_cons_2d(rho, mu, nu, rho ** g)
    m = moments_2d(f, 0.0, L, 0.0, L, n, n, npts=npts)
    return Problem("vortex_2d", 2, n, n, 0.0, L, 0.0, L, "euler", ("periodic",) * 4, m, seed=seed,
                   meta={"eps": eps, "xc": xc, "yc": yc})


def walled_blast_2d(n=64, seed=0, ncircles=2, walls=("reflective",) * 4):
    """blast_2d data in a box with the given boundary kinds (xlo, xhi, ylo, yhi)."""
    p = blast_2d(n, seed=seed, ncircles=ncircles)
    p.bc = tuple(walls)
    p.name = "walled_blast_2d"
    return p


def blast_2d(n=4096, seed=0, ncircles=8):
    """Random circles (radius U[0.05,0.2], inside p ~ U[5,100]) in p = 0.1 gas,
    rho = 1, at rest, on [0,1]^2, transmissive."""
    rng = np.random.default_rng(seed)
    cx = rng.uniform(0.0, 1.0, ncircles)
    cy = rng.uniform(0.0, 1.0, ncircles)
    rad = rng.uniform(0.05, 0.2, ncircles)
    pin = rng.uniform(5.0, 100.0, ncircles)

    def f(X, Y):
        p = np.full(X.shape, 0.1)
        for k in range(ncircles):
            inside = (X - cx[k]) ** 2 + (Y - cy[k]) ** 2 < rad[k] ** 2
            p = np.where(inside, np.maximum(p, pin[k]), p)
        z = np.zeros_like(p)
        return prim_to_cons_2d(np.ones_like(p), z, z, p)
    m = moments_2d(f, 0.0, 1.0, 0.0, 1.0, n, n, npts=4)
    return Problem("blast_2d", 2, n, n, 0.0, 1.0, 0.0, 1.0, "euler", ("transmissive",) * 4, m,
                   seed=seed, meta={"cx": cx.tolist(), "cy": cy.tolist(), "r": rad.tolist(),
                                    "p_in": pin.tolist()})


def double_mach_2d(ny=400):
    """Example 3.9, double Mach reflection: [0,4] x [0,1] (4 ny x ny square
    cells), a Mach 10 shock at 60 degrees to the x-axis through (1/6, 0).
    Post-shock (rho, u, v, p) = (8, 8.25 cos 30, -8.25 sin 30, 116.5), pre-shock
    (1.4, 0, 0, 1).  Boundaries: inflow of the post-shock state on the left,
    outflow (transmissive) on the right; on the floor the post-shock state
    before x = 1/6 and a reflective wall after it; on the top the exact shock
    trace: ghost cells (centre height 1 + dy/2) hold the post-shock state left
    of x = 1/6 + (1 + dy/2 + 20 t)/sqrt(3), the pre-shock state right of it.
    Cell moments of the initial discontinuity by 8 x 8 Gauss-Legendre points.
    To t = 0.2."""
    nx = 4 * ny
    s3 = math.sqrt(3.0)
    post = prim_to_cons_2d(8.0, 8.25 * s3 / 2.0, -8.25 * 0.5, 116.5)
    pre = prim_to_cons_2d(1.4, 0.0, 0.0, 1.0)

    def f(X, Y):
        left = X < 1.0 / 6.0 + Y / s3
        return np.stack([np.where(left, post[v], pre[v]) for v in range(4)])
    m = moments_2d(f, 0.0, 4.0, 0.0, 1.0, nx, ny)
    dy = 1.0 / ny
    post_t, pre_t = tuple(float(x) for x in post), tuple(float(x) for x in pre)
    fixed = ({"b": post_t}, None, {"a": post_t, "c0": 1.0 / 6.0},
             {"a": post_t, "b": pre_t, "c0": 1.0 / 6.0 + (1.0 + 0.5 * dy) / s3, "speed": 20.0 / s3})
    return Problem("double_mach_2d", 2, nx, ny, 0.0, 4.0, 0.0, 1.0, "euler",
                   ("inflow", "transmissive", "reflective", "inflow"), m, t_end=0.2, fixed=fixed)


def forward_step_2d(ny=200):
    """Example 3.10, Mach 3 flow over a forward-facing step: [0,3] x [0,1]
    (3 ny x ny square cells), a step of height 0.2 from x = 0.6 on (solid cells
    i >= 0.6 ny, j < 0.2 ny).  Initial and inflow state (rho, u, v, p) =
    (1.4, 3, 0, 1); inflow on the left, outflow (transmissive) on the right,
    reflective walls at the top, the bottom and the step's faces.  To t = 4.
    ny must be a multiple of 5 (the step's corner on a cell corner)."""
    if ny % 5:
        raise ValueError("ny must be a multiple of 5")
    nx = 3 * ny
    state = prim_to_cons_2d(1.4, 3.0, 0.0, 1.0)
    m = np.zeros((4, 3, ny, nx))
    for v in range(4):
        m[v, 0] = state[v]
    fixed = ({"b": tuple(float(x) for x in state)}, None, None, None)
    return Problem("forward_step_2d", 2, nx, ny, 0.0, 3.0, 0.0, 1.0, "euler",
                   ("inflow", "transmissive", "reflective", "reflective"), m, t_end=4.0, fixed=fixed,
                   meta={"solid": (3 * ny // 5, ny // 5)})


def batch_sizes(seed=0, count=256, choices=(64, 128, 256, 512)):
    """Grid sizes of a batch of independent problems, uniform in choices."""
    rng = np.random.default_rng(seed)
    return [int(x) for x in rng.choice(np.asarray(choices), size=count)]


def batch_problems(count=256, seed=0, choices=(64, 128, 256, 512), npts=4):
    """Independent problems of a batch: sizes uniform in choices; even entries
    four-quadrant Riemann data on [0,1]^2 (transmissive), odd entries an isentropic
    vortex on periodic [0,10]^2 (Gauss-Legendre order npts per direction)."""
    sizes = batch_sizes(seed, count, choices)
    out = []
    for k, n in enumerate(sizes):
        if k % 2 == 0:
            out.append(four_quadrant_2d(n, seed=seed * 100003 + k))
        else:
            out.append(vortex_2d(n, seed=seed * 100003 + k, npts=npts))
    return out
