"""CPU FP64 oracle of the moment-based multi-resolution HWENO scheme.

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (the CUDA library and its binding) never does.

The arithmetic lives in ``hweno_oracle.c`` (plain C, one cell at a time, in
the paper's order); this module only compiles it and marshals numpy arrays.
Parity status of each piece is stated in ``hweno_oracle.c`` and in the tests
that pin it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hweno_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

EQ = {"advection": 0, "burgers": 1, "euler": 2}
IND = {"none": 0, "kxrcf": 1, "all": 2, "given": 3, "tvb": 4}
BC = {"periodic": 0, "transmissive": 1, "reflective": 2, "inflow": 3}


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (-O2, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
                               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Cfg(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("eq", ctypes.c_int),
                ("adv_a", ctypes.c_double), ("adv_b", ctypes.c_double), ("gamma", ctypes.c_double),
                ("indicator", ctypes.c_int), ("gbar", ctypes.c_double * 4), ("bc", ctypes.c_int * 4),
                ("tvb_m", ctypes.c_double), ("charwise", ctypes.c_int),
                ("x0", ctypes.c_double), ("y0", ctypes.c_double), ("t", ctypes.c_double),
                ("seg_on", ctypes.c_int * 4), ("seg_c0", ctypes.c_double * 4), ("seg_speed", ctypes.c_double * 4),
                ("fa", (ctypes.c_double * 4) * 4), ("fb", (ctypes.c_double * 4) * 4),
                ("mod_in_L_only", ctypes.c_int), ("sol_i", ctypes.c_int), ("sol_j", ctypes.c_int)]


def make_cfg(dim, nx, ny=1, dx=1.0, dy=1.0, eq="euler", adv=(1.0, 0.0), gamma=1.4,
             indicator="kxrcf", gbar=(1.0, 10.0, 100.0, 1000.0), bc=("periodic",) * 4, tvb_m=0.0,
             charwise=False, x0=0.0, y0=0.0, t=0.0, fixed=None, mod_in_L_only=False, solid=None) -> Cfg:
    """fixed: per side (x-lo, x-hi, y-lo, y-hi) None or a dict with the
    fixed ghost states: "a" inside the segment (centre coordinate along the
    side below c0 + speed * t; no segment when "c0" is absent), "b" elsewhere
    on an "inflow" side.  solid: None or (i0, j1): cells with i >= i0 and
    j < j1 are solid (a forward-facing step; 2D Euler).  The block touches
    the right side (when i0 > 0) and the bottom side (when j1 < ny), which
    therefore may not be periodic: a wrap would meet the block from behind."""
    c = Cfg()
    c.dim, c.nx, c.ny = dim, nx, (ny if dim == 2 else 1)
    c.dx, c.dy = dx, (dy if dim == 2 else 1.0)
    c.eq = EQ[eq] if isinstance(eq, str) else int(eq)
    c.adv_a, c.adv_b = adv
    c.gamma = gamma
    c.indicator = IND[indicator] if isinstance(indicator, str) else int(indicator)
    c.tvb_m = tvb_m
    c.charwise = int(bool(charwise))
    c.x0, c.y0, c.t = x0, y0, t
    c.mod_in_L_only = int(bool(mod_in_L_only))
    if solid is not None:
        c.sol_i, c.sol_j = int(solid[0]), int(solid[1])
        if (c.sol_i > 0 and bc[1] == "periodic") or (c.sol_j < c.ny and bc[2] == "periodic"):
            raise ValueError("solid block: the sides it touches may not be periodic")
    for k, f in enumerate(fixed or [None] * 4):
        if not f:
            continue
        if f.get("c0") is not None:
            c.seg_on[k] = 1
            c.seg_c0[k] = f["c0"]
            c.seg_speed[k] = f.get("speed", 0.0)
        for v in range(4):
            c.fa[k][v] = f.get("a", (0.0,) * 4)[v]
            c.fb[k][v] = f.get("b", (0.0,) * 4)[v]
    for k in range(4):
        c.gbar[k] = gbar[k]
        b = bc[k]
        c.bc[k] = BC[b] if isinstance(b, str) else int(b)
    return c


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            D = ctypes.POINTER(ctypes.c_double)
            U8 = ctypes.POINTER(ctypes.c_uint8)
            I = ctypes.POINTER(ctypes.c_int)
            C = ctypes.POINTER(Cfg)
            _lib.orc_rhs.argtypes = [C, D, D, D, U8, D]
            _lib.orc_step.argtypes = [C, D, ctypes.c_double, U8]
            _lib.orc_max_dt.argtypes = [C, D, ctypes.c_double]
            _lib.orc_max_dt.restype = ctypes.c_double
            _lib.orc_wave_speeds.argtypes = [C, D, ctypes.c_int, ctypes.c_int, D]
            _lib.orc_modification_weights.argtypes = [D]
            _lib.orc_recon_cell.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, D, D, D, D, D]
            _lib.orc_poly.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, D, D, D]
            _lib.orc_level_matrix.argtypes = [ctypes.c_int, ctypes.c_int, I, I, I, I, I, I, I, D]
            _lib.orc_num_flux.argtypes = [C, D, D, ctypes.c_int, D]
            _lib.orc_phys_flux.argtypes = [C, D, ctypes.c_int, D]
            _lib.orc_kxrcf_aleph.argtypes = [C, D, ctypes.c_int, ctypes.c_int]
            _lib.orc_kxrcf_aleph.restype = ctypes.c_double
            _lib.orc_totals.argtypes = [C, D, D]
            _lib.orc_set_beta_source.argtypes = [ctypes.c_int]
            _lib.orc_euler1d_eig.argtypes = [ctypes.c_double, D, D, D]
        return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _u8(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def nvars(cfg: Cfg) -> int:
    return 1 if cfg.eq != 2 else (3 if cfg.dim == 1 else 4)


def state_shape(cfg: Cfg):
    return (nvars(cfg), 2 if cfg.dim == 1 else 3, cfg.ny if cfg.dim == 2 else 1, cfg.nx)


def rhs(cfg: Cfg, U: np.ndarray, decisions=None):
    """L(U) with the troubled-cell steps. Returns (Umod, L, mask, aleph, status).
    With indicator "given", decisions[cell] is 0 (smooth), 1 (troubled) or 2
    (KXRCF decides after the given troubled cells are modified)."""
    U = np.ascontiguousarray(U, dtype=np.float64).reshape(state_shape(cfg))
    Um = np.empty_like(U)
    L = np.empty_like(U)
    ncell = cfg.nx * (cfg.ny if cfg.dim == 2 else 1)
    mask = np.zeros(ncell, np.uint8)
    if decisions is not None:
        mask[:] = np.asarray(decisions, np.uint8).reshape(-1)
    aleph = np.zeros(ncell, np.float64)
    rc = lib().orc_rhs(ctypes.byref(cfg), _dp(U), _dp(Um), _dp(L), _u8(mask), _dp(aleph))
    return Um, L, mask, aleph, rc


def step(cfg: Cfg, m: np.ndarray, dt: float):
    """One SSP-RK3 step. Returns (new state, masks[3, ncell], status)."""
    m = np.array(m, dtype=np.float64, order="C").reshape(state_shape(cfg))
    ncell = cfg.nx * (cfg.ny if cfg.dim == 2 else 1)
    masks = np.zeros((3, ncell), np.uint8)
    rc = lib().orc_step(ctypes.byref(cfg), _dp(m), float(dt), _u8(masks))
    return m, masks, rc


def euler1d_eig(gamma: float, u) -> tuple[np.ndarray, np.ndarray]:
    """Right (columns) and left (rows) eigenvectors of the 1D Euler flux
    Jacobian at the conserved state u, as the characteristic option uses them."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    R = np.empty((3, 3))
    L = np.empty((3, 3))
    lib().orc_euler1d_eig(float(gamma), _dp(u), _dp(R), _dp(L))
    return R, L


def max_dt(cfg: Cfg, m: np.ndarray, cfl: float = 0.6) -> float:
    m = np.ascontiguousarray(m, dtype=np.float64)
    return lib().orc_max_dt(ctypes.byref(cfg), _dp(m), float(cfl))


def wave_speeds(cfg: Cfg, m: np.ndarray, jlo: int, jhi: int):
    """(max a_x, max a_y) of the CFL rule over rows [jlo, jhi)."""
    m = np.ascontiguousarray(m, dtype=np.float64)
    out = np.zeros(2)
    lib().orc_wave_speeds(ctypes.byref(cfg), _dp(m), int(jlo), int(jhi), _dp(out))
    return float(out[0]), float(out[1])


def totals(cfg: Cfg, m: np.ndarray) -> np.ndarray:
    m = np.ascontiguousarray(m, dtype=np.float64)
    out = np.zeros(nvars(cfg))
    lib().orc_totals(ctypes.byref(cfg), _dp(m), _dp(out))
    return out


def run(cfg: Cfg, m: np.ndarray, t_end: float, cfl: float = 0.6, dt_fn=None, max_steps=10**7):
    """Advance to t_end with the CFL rule (or dt_fn(dx)), clipping the last step."""
    t = 0.0
    nsteps = 0
    while t < t_end - 1e-14 * max(1.0, t_end) and nsteps < max_steps:
        dt = dt_fn() if dt_fn is not None else max_dt(cfg, m, cfl)
        dt = min(dt, t_end - t)
        m, _, rc = step(cfg, m, dt)
        if rc != 0:
            raise RuntimeError(f"oracle step failed with status {rc} at t={t}")
        t += dt
        nsteps += 1
    return m, nsteps


def modification_weights() -> np.ndarray:
    out = np.zeros(5)
    lib().orc_modification_weights(_dp(out))
    return out


def recon_cell(dim: int, data, gbar=(1.0, 10.0, 100.0, 1000.0), dx=1.0, dy=1.0):
    data = np.ascontiguousarray(data, dtype=np.float64)
    g = np.ascontiguousarray(gbar, dtype=np.float64)
    vals = np.zeros(4 if dim == 1 else 16)
    beta = np.zeros(4)
    omega = np.zeros(4)
    lib().orc_recon_cell(dim, dx, dy, _dp(g), _dp(data), _dp(vals), _dp(beta), _dp(omega))
    return vals, beta, omega


def poly(dim: int, level: int, data, kind: str = "q", gbar=(1.0, 10.0, 100.0, 1000.0)) -> np.ndarray:
    """Monomial coefficients c[a, b] (xi^a eta^b) of q_level (kind "q"), of p_level
    (kind "p"), or of the linear-weight polynomial sum_l gamma_l4 p_l (kind "lin")."""
    data = np.ascontiguousarray(data, dtype=np.float64)
    g = np.ascontiguousarray(gbar, dtype=np.float64)
    out = np.zeros(36)
    lib().orc_poly(dim, level, {"q": 0, "lin": 1, "p": 2}[kind], _dp(g), _dp(data), _dp(out))
    return out.reshape(6, 6)


def level_matrix(dim: int, level: int):
    """(M, monomials[(a,b)], conditions[(kind, ox, oy)]) of the level's solve."""
    nm = ctypes.c_int()
    nc = ctypes.c_int()
    ma = (ctypes.c_int * 21)()
    mb = (ctypes.c_int * 21)()
    ck = (ctypes.c_int * 23)()
    cx = (ctypes.c_int * 23)()
    cy = (ctypes.c_int * 23)()
    M = np.zeros(21 * 23)
    lib().orc_level_matrix(dim, level, ctypes.byref(nm), ctypes.byref(nc), ma, mb, ck, cx, cy, _dp(M))
    n, m = nm.value, nc.value
    return (M[: n * m].reshape(n, m), [(ma[k], mb[k]) for k in range(n)],
            [(ck[r], cx[r], cy[r]) for r in range(m)])


def num_flux(cfg: Cfg, uL, uR, direction: int = 0) -> np.ndarray:
    uL = np.ascontiguousarray(uL, dtype=np.float64)
    uR = np.ascontiguousarray(uR, dtype=np.float64)
    F = np.zeros(nvars(cfg))
    lib().orc_num_flux(ctypes.byref(cfg), _dp(uL), _dp(uR), direction, _dp(F))
    return F


def kxrcf_aleph(cfg: Cfg, G, i: int, j: int = 0) -> float:
    """The KXRCF value of cell (i, j) from given point values G[j][i][var][k][l]
    (2D; 1D: G[i][var][k], the 4 Gauss-Lobatto points of a cell)."""
    G = np.ascontiguousarray(G, dtype=np.float64)
    if cfg.dim == 2:
        want = (cfg.ny, cfg.nx, nvars(cfg), 4, 4)
        flat = G.reshape(-1)
    else:
        want = (cfg.nx, nvars(cfg), 4)
        flat = np.zeros((cfg.nx, nvars(cfg), 16))
        flat[:, :, :4] = G
        flat = flat.reshape(-1)
    if G.shape != want:
        raise ValueError(f"G must have shape {want}")
    return float(lib().orc_kxrcf_aleph(ctypes.byref(cfg), _dp(flat), int(i), int(j)))


def phys_flux(cfg: Cfg, u, direction: int = 0) -> np.ndarray:
    u = np.ascontiguousarray(u, dtype=np.float64)
    F = np.zeros(nvars(cfg))
    lib().orc_phys_flux(ctypes.byref(cfg), _dp(u), direction, _dp(F))
    return F


def set_beta_source(from_q: bool) -> None:
    """Diagnostic only: take beta_l from q_l instead of p_l (see hweno_oracle.c)."""
    lib().orc_set_beta_source(1 if from_q else 0)
