"""Thin Python binding of the C ABI in include/hweno.h (argument marshalling only).

Every step of the computation runs in libhweno.so (CUDA, sm_103a).  There is no
CPU fallback: if the library is missing or no GPU is present, the calls fail.
Device buffers may be torch CUDA tensors; host buffers numpy arrays or CPU
tensors.  PyTorch only provides device memory and the stream.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libhweno.so")
_lib = None

ENONPHYSICAL = -3
STATUS = {0: "OK", -1: "EINVAL", -2: "ECUDA", -3: "ENONPHYSICAL", -4: "ETIMEOUT", -5: "ESTATE", -6: "ENOMEM"}
EQ = {"advection": 0, "burgers": 1, "euler": 2}
IND = {"none": 0, "kxrcf": 1, "all": 2, "mlp": 3, "tvb": 4}
BC = {"periodic": 0, "transmissive": 1, "reflective": 2, "inflow": 3}
PREC = {"fp64": 0, "fp32": 1, "df64": 2}


class HwenoError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("x0", ctypes.c_double), ("x1", ctypes.c_double), ("y0", ctypes.c_double), ("y1", ctypes.c_double),
                ("eq", ctypes.c_int), ("adv_a", ctypes.c_double), ("adv_b", ctypes.c_double),
                ("precision", ctypes.c_int), ("indicator", ctypes.c_int), ("gamma_bar", ctypes.c_double * 4),
                ("beta_of_q", ctypes.c_int), ("tvb_m", ctypes.c_double), ("charwise", ctypes.c_int)]


class FixedState(ctypes.Structure):
    _fields_ = [("segment", ctypes.c_int), ("c0", ctypes.c_double), ("speed", ctypes.c_double),
                ("a", ctypes.c_double * 4), ("b", ctypes.c_double * 4)]


class Bc(ctypes.Structure):
    _fields_ = [("xlo", ctypes.c_int), ("xhi", ctypes.c_int), ("ylo", ctypes.c_int), ("yhi", ctypes.c_int)]


def lib():
    """Load libhweno.so (fails loudly when it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library {LIB_PATH} is missing: run paper_2201_12193_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        H = ctypes.c_void_p
        D = ctypes.POINTER(ctypes.c_double)
        L.hweno_create.argtypes = [ctypes.POINTER(Grid), ctypes.POINTER(Bc), ctypes.c_double, ctypes.POINTER(H)]
        L.hweno_destroy.argtypes = [H]
        L.hweno_destroy.restype = None
        L.hweno_set_stream.argtypes = [H, ctypes.c_void_p]
        L.hweno_set_moments.argtypes = [H, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int]
        L.hweno_get_moments.argtypes = [H, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int]
        L.hweno_step.argtypes = [H, ctypes.c_double]
        L.hweno_max_dt.argtypes = [H, ctypes.c_double, D]
        L.hweno_troubled_mask.argtypes = [H, ctypes.c_void_p, ctypes.c_size_t]
        L.hweno_totals.argtypes = [H, D]
        L.hweno_sync.argtypes = [H]
        L.hweno_rhs.argtypes = [H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        L.hweno_profile.argtypes = [H, ctypes.c_int]
        L.hweno_profile_read.argtypes = [H, D, ctypes.POINTER(ctypes.c_int), ctypes.c_int]
        L.hweno_max_dt_noalloc.argtypes = [ctypes.POINTER(Grid), ctypes.c_double, ctypes.c_void_p, ctypes.c_double,
                                           ctypes.c_void_p, ctypes.c_void_p]
        L.hweno_create_batch.argtypes = [ctypes.POINTER(Grid), ctypes.POINTER(Bc), ctypes.c_int, ctypes.c_double,
                                         ctypes.POINTER(H)]
        L.hweno_batch_set_moments.argtypes = [H, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int]
        L.hweno_batch_get_moments.argtypes = [H, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int]
        L.hweno_step_batch.argtypes = [H, ctypes.c_void_p, ctypes.c_double]
        L.hweno_batch_dt.argtypes = [H, D, ctypes.c_int]
        L.hweno_batch_troubled_mask.argtypes = [H, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t]
        L.hweno_batch_set_tile.argtypes = [H, ctypes.c_int]
        L.hweno_batch_set_barrier.argtypes = [H, ctypes.c_longlong, ctypes.c_int]
        L.hweno_batch_uses_graph.argtypes = [H]
        L.hweno_batch_status.argtypes = [H, ctypes.POINTER(ctypes.c_uint), ctypes.c_int]
        L.hweno_alu_probe.argtypes = [ctypes.c_int, ctypes.c_longlong, D, ctypes.c_void_p]
        L.hweno_f32_round.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_longlong, ctypes.c_void_p]
        L.hweno_mlp_nparam.restype = ctypes.c_int
        L.hweno_set_mlp.argtypes = [H, ctypes.c_void_p, ctypes.c_int, ctypes.c_float]
        L.hweno_mlp_fallbacks.argtypes = [H, ctypes.POINTER(ctypes.c_longlong)]
        L.hweno_features.argtypes = [H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
        L.hweno_mlp_forward.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
        L.hweno_mlp_loss_grad.argtypes = [ctypes.c_void_p] * 4 + [ctypes.c_int] + [ctypes.c_void_p] * 3
        L.hweno_mlp_adam.argtypes = [ctypes.c_void_p] * 4 + [ctypes.c_int, ctypes.c_float, ctypes.c_void_p]
        L.hweno_mlp_probe.argtypes = [H, ctypes.c_void_p]
        L.hweno_advance.argtypes = [H, ctypes.c_double, ctypes.c_double, ctypes.c_longlong,
                                    ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong)]
        L.hweno_rerecon_count.argtypes = [H, ctypes.POINTER(ctypes.c_longlong)]
        L.hweno_set_positivity_check.argtypes = [H, ctypes.c_int]
        L.hweno_set_persistence.argtypes = [H, ctypes.c_int]
        L.hweno_set_fused.argtypes = [H, ctypes.c_int]
        L.hweno_set_tma.argtypes = [H, ctypes.c_int]
        L.hweno_set_solid.argtypes = [H, ctypes.c_int, ctypes.c_int]
        L.hweno_set_owned_rows.argtypes = [H, ctypes.c_int, ctypes.c_int]
        L.hweno_stage.argtypes = [H, ctypes.c_int, ctypes.c_double]
        L.hweno_copy_rows.argtypes = [H, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int]
        L.hweno_wave_speeds.argtypes = [H, D]
        L.hweno_set_fixed_state.argtypes = [H, ctypes.c_int, ctypes.POINTER(FixedState)]
        L.hweno_set_time.argtypes = [H, ctypes.c_double]
        L.hweno_get_time.argtypes = [H, D]
        L.hweno_last_error.argtypes = [H]
        L.hweno_last_error.restype = ctypes.c_char_p
        L.hweno_version.restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(x):
    """(address, on_device, element count) of a contiguous numpy array or torch tensor."""
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data, 0, x.size
    if not x.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return x.data_ptr(), int(x.is_cuda), x.numel()


def _f64(x):
    if isinstance(x, np.ndarray):
        if x.dtype != np.float64:
            raise TypeError("moments must be float64")
    elif str(x.dtype) != "torch.float64":
        raise TypeError("moments must be float64")
    return x


class Solver:
    """One problem on the GPU; method names follow the C ABI (hweno_*).

    precision: "fp64" (the scheme as specified), "fp32" (FP32 bulk, FP64 state and
    Runge-Kutta accumulation) or "df64" (double-float pairs); indicator: "kxrcf",
    "none", "all", "tvb" (with tvb_m) or "mlp" (with set_mlp); bc per side:
    "periodic", "transmissive", "reflective" (Euler) or "inflow" (2D Euler FP64,
    states by set_fixed_state); charwise: characteristic-wise reconstruction
    (1D Euler).  A 1D handle runs each Runge-Kutta stage as one fused launch
    unless it is charwise or uses TVB (set_fused(False) selects the four-launch
    pipeline; both give the same states bit for bit)."""

    def __init__(self, dim, nx, ny=1, x0=0.0, x1=1.0, y0=0.0, y1=1.0, eq="euler", adv=(1.0, 0.0),
                 precision="fp64", indicator="kxrcf", gamma_bar=(1.0, 10.0, 100.0, 1000.0), beta_of_q=False,
                 bc=("transmissive",) * 4, gamma=1.4, stream=None, tvb_m=0.0, charwise=False):
        g = Grid()
        g.dim, g.nx, g.ny = dim, nx, (ny if dim == 2 else 1)
        g.x0, g.x1, g.y0, g.y1 = x0, x1, y0, y1
        g.eq = EQ[eq]
        g.adv_a, g.adv_b = adv
        g.precision = PREC[precision]
        g.indicator = IND[indicator]
        for k in range(4):
            g.gamma_bar[k] = gamma_bar[k]
        g.beta_of_q = int(bool(beta_of_q))
        g.tvb_m = float(tvb_m)
        g.charwise = int(bool(charwise))
        b = Bc(*[BC[k] for k in bc])
        h = ctypes.c_void_p()
        st = lib().hweno_create(ctypes.byref(g), ctypes.byref(b), float(gamma), ctypes.byref(h))
        if st != 0:
            raise HwenoError(st, "hweno_create failed (see stderr)")
        self._h = h
        self.grid = g
        self.dim, self.nx, self.ny = dim, nx, g.ny
        self.nvar = 1 if eq != "euler" else (3 if dim == 1 else 4)
        self.nmom = 2 if dim == 1 else 3
        self.shape = (self.nvar, self.nmom, self.ny, self.nx)
        self.count = int(np.prod(self.shape))
        if stream is not None:
            self.set_stream(stream)

    @classmethod
    def from_problem(cls, p, **kw):
        s = cls(p.dim, p.nx, p.ny, p.x0, p.x1, p.y0, p.y1, eq=p.eq, adv=p.adv, bc=p.bc, gamma=p.gamma, **kw)
        for side, f in enumerate(p.fixed or ()):
            if f:
                s.set_fixed_state(side, **f)
        if p.meta.get("solid"):
            s.set_solid(*p.meta["solid"])
        return s

    def set_fixed_state(self, side, a=None, b=None, c0=None, speed=0.0):
        """Fixed ghost states of one side (0 x-lo, 1 x-hi, 2 y-lo, 3 y-hi): a inside
        the segment (centre coordinate along the side below c0 + speed * t; no
        segment when c0 is None), b elsewhere on an "inflow" side."""
        f = FixedState()
        f.segment = int(c0 is not None)
        f.c0 = float(c0 if c0 is not None else 0.0)
        f.speed = float(speed)
        for v in range(4):
            f.a[v] = float(a[v]) if a is not None else 0.0
            f.b[v] = float(b[v]) if b is not None else 0.0
        self._check(lib().hweno_set_fixed_state(self._h, int(side), ctypes.byref(f)))

    def set_time(self, t):
        self._check(lib().hweno_set_time(self._h, float(t)))

    def time(self):
        v = ctypes.c_double()
        self._check(lib().hweno_get_time(self._h, ctypes.byref(v)))
        return v.value

    def _check(self, st):
        if st != 0:
            raise HwenoError(st, lib().hweno_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            lib().hweno_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, a raw cudaStream_t integer, or None (default stream)."""
        s = getattr(stream, "cuda_stream", stream) or 0
        self._check(lib().hweno_set_stream(self._h, ctypes.c_void_p(s)))

    def set_moments(self, m):
        if isinstance(m, np.ndarray):
            m = np.ascontiguousarray(m)
        addr, dev, n = _ptr(_f64(m))
        self._check(lib().hweno_set_moments(self._h, ctypes.c_void_p(addr), n, dev))

    def get_moments(self, out=None):
        """Into out (torch CUDA tensor or host array) or a new numpy array."""
        if out is None:
            out = np.empty(self.shape, np.float64)
        addr, dev, n = _ptr(_f64(out))
        self._check(lib().hweno_get_moments(self._h, ctypes.c_void_p(addr), n, dev))
        return out

    def step(self, dt):
        self._check(lib().hweno_step(self._h, float(dt)))

    def max_dt(self, cfl=0.6):
        dt = ctypes.c_double()
        self._check(lib().hweno_max_dt(self._h, float(cfl), ctypes.byref(dt)))
        return dt.value

    def troubled_mask(self):
        out = np.empty((3, self.ny, self.nx), np.uint8)
        self._check(lib().hweno_troubled_mask(self._h, ctypes.c_void_p(out.ctypes.data), out.size))
        return out

    def totals(self):
        out = (ctypes.c_double * 4)()
        self._check(lib().hweno_totals(self._h, out))
        return np.array(out[: self.nvar])

    def sync(self):
        self._check(lib().hweno_sync(self._h))

    def rhs(self, U, Umod, L, mask, aleph=None):  # noqa: D401
        """Device tensors: U (in), Umod, L, mask (uint8 [ny, nx]), aleph (optional float64 [ny, nx])."""
        for x in (U, Umod, L):
            if _ptr(x)[2] != self.count or not _ptr(x)[1]:
                raise ValueError("U, Umod and L must be CUDA tensors of nvar*nmom*ny*nx float64")
        if _ptr(mask)[2] != self.nx * self.ny or not _ptr(mask)[1]:
            raise ValueError("mask must be a CUDA uint8 tensor of ny*nx")
        ptrs = [_ptr(x)[0] for x in (U, Umod, L, mask)]
        a = _ptr(aleph)[0] if aleph is not None else None
        self._check(lib().hweno_rhs(self._h, *[ctypes.c_void_p(p) for p in ptrs], ctypes.c_void_p(a)))

    def set_mlp(self, params, conf=0.9):
        """Install the learned indicator (handle created with indicator="mlp")."""
        if isinstance(params, np.ndarray):
            params = np.ascontiguousarray(params, dtype=np.float32)
        addr, dev, n = _ptr(params)
        if n != mlp_nparam():
            raise ValueError(f"expected {mlp_nparam()} parameters")
        self._check(lib().hweno_set_mlp(self._h, ctypes.c_void_p(addr), dev, float(conf)))

    def mlp_fallbacks(self):
        v = ctypes.c_longlong()
        self._check(lib().hweno_mlp_fallbacks(self._h, ctypes.byref(v)))
        return v.value

    def mlp_probe(self, prob):
        """prob: CUDA float32 tensor of ny*nx that each later stage fills with the
        network's probabilities, or None to stop."""
        if prob is not None and (_ptr(prob)[2] != self.nx * self.ny or not _ptr(prob)[1]):
            raise ValueError("prob must be a CUDA float32 tensor of ny*nx")
        self._probe = prob
        self._check(lib().hweno_mlp_probe(self._h, ctypes.c_void_p(_ptr(prob)[0] if prob is not None else None)))

    def set_positivity_check(self, on=True):
        """Off: only non-finite values fail a step (rho <= 0 / p <= 0 averages carry on)."""
        self._check(lib().hweno_set_positivity_check(self._h, int(bool(on))))

    def set_solid(self, i0, j1):
        """Solid block: cells with i >= i0 and j < j1 (the forward step); j1 = 0 removes it."""
        self._check(lib().hweno_set_solid(self._h, int(i0), int(j1)))

    def set_owned_rows(self, jlo, jhi):
        """Rows [jlo, jhi) this handle owns (row-slab decomposition)."""
        self._check(lib().hweno_set_owned_rows(self._h, int(jlo), int(jhi)))

    def stage(self, k, dt):
        """Stage k (0, 1, 2) of one SSP-RK3 step."""
        self._check(lib().hweno_stage(self._h, int(k), float(dt)))

    def copy_rows(self, j0, nrows, buf, to_state):
        """Rows [j0, j0 + nrows) of the state the next stage reads, to or from
        buf (CUDA float64 tensor of nvar*nmom*nrows*nx values)."""
        a, dev, n = _ptr(_f64(buf))
        if not dev or n != self.nvar * self.nmom * nrows * self.nx:
            raise ValueError("buf must be a CUDA float64 tensor of nvar*nmom*nrows*nx values")
        self._check(lib().hweno_copy_rows(self._h, int(j0), int(nrows), ctypes.c_void_p(a), int(bool(to_state))))

    def wave_speeds(self):
        """(max a_x, max a_y) over the owned rows."""
        out = (ctypes.c_double * 2)()
        self._check(lib().hweno_wave_speeds(self._h, out))
        return out[0], out[1]

    def set_tma(self, on=True):
        """TMA staging of the FP32-bulk update's interior tiles (off by
        default; bitwise the same results either way)."""
        self._check(lib().hweno_set_tma(self._h, int(bool(on))))

    def set_fused(self, on=True):
        """One fused kernel per Runge-Kutta stage instead of the four-launch
        pipeline (KXRCF, none or all indicator): 2D Euler (off by default) and
        component-wise 1D (on by default, bitwise the pipeline)."""
        self._check(lib().hweno_set_fused(self._h, int(bool(on))))

    def set_persistence(self, persist=True):
        """True (default): the first moments modified in troubled cells (eq. (vi))
        replace the stage input and enter the Runge-Kutta combination; False:
        they serve L only."""
        self._check(lib().hweno_set_persistence(self._h, int(bool(persist))))

    def rerecon_count(self):
        """Cells reconstructed a second time (troubled cells, Step 2.3) since the last call."""
        v = ctypes.c_longlong()
        self._check(lib().hweno_rerecon_count(self._h, ctypes.byref(v)))
        return v.value

    def features(self, U, cells, X):
        """108 features (float32 rows) of cells (int32 CUDA tensor) of state U (CUDA)."""
        self._check(lib().hweno_features(self._h, ctypes.c_void_p(_ptr(U)[0]), ctypes.c_void_p(_ptr(cells)[0]),
                                         int(cells.numel()), ctypes.c_void_p(_ptr(X)[0])))

    KERNEL_KINDS = ("reconstruct", "indicator", "reconstruct_troubled", "update", "learned_indicator", "fused_stage")

    def profile(self, enable=True):
        self._check(lib().hweno_profile(self._h, int(bool(enable))))

    def profile_read(self):
        """{kind: (device ms, launches)} since the last read."""
        k = len(self.KERNEL_KINDS)
        ms = (ctypes.c_double * k)()
        n = (ctypes.c_int * k)()
        self._check(lib().hweno_profile_read(self._h, ms, n, k))
        return {k: (ms[i], n[i]) for i, k in enumerate(self.KERNEL_KINDS)}

    def advance(self, t_end, cfl=0.6, max_steps=10 ** 12):
        """Advance by t_end with the CFL dt formed on the device (graph replays of
        12 steps, no host round trip per step). Returns (time reached, steps)."""
        t = ctypes.c_double()
        n = ctypes.c_longlong()
        self._check(lib().hweno_advance(self._h, float(t_end), float(cfl), int(max_steps), ctypes.byref(t),
                                        ctypes.byref(n)))
        return t.value, n.value

    def run(self, t_end, cfl=0.6, dt=None, max_steps=10 ** 9):
        """Advance to t_end (CFL dt unless dt is given), clipping the last step."""
        t, n = 0.0, 0
        while t < t_end - 1e-14 * max(1.0, t_end) and n < max_steps:
            h = dt if dt is not None else self.max_dt(cfl)
            h = min(h, t_end - t)
            self.step(h)
            t += h
            n += 1
        self.sync()
        return n


def version():
    return lib().hweno_version()


def max_dt_noalloc(grid, gamma, m, cfl, out, stream=None):
    """hweno_max_dt_noalloc: m and out are CUDA float64 tensors on the current
    device (m the state of the grid, nvar*nmom*ny*nx values; out 3 doubles
    receiving max a_x, max a_y, dt); nothing is allocated by the library.
    stream: a torch.cuda.Stream or raw cudaStream_t; None = torch's current
    stream, so the call is ordered after the work that wrote m."""
    import torch

    a, dev, n = _ptr(_f64(m))
    o, odev, on = _ptr(_f64(out))
    if not (dev and odev) or on < 3:
        raise ValueError("m and out must be CUDA float64 tensors (out with 3 elements)")
    cur = torch.cuda.current_device()
    if m.device.index != cur or out.device.index != cur:
        raise ValueError("m and out must live on the current CUDA device")
    nvar = 1 if grid.eq != EQ["euler"] else (3 if grid.dim == 1 else 4)
    need = nvar * (2 if grid.dim == 1 else 3) * grid.nx * (grid.ny if grid.dim == 2 else 1)
    if n < need:
        raise ValueError(f"m holds {n} values; the grid needs {need}")
    if stream is None:
        stream = torch.cuda.current_stream()
    s = getattr(stream, "cuda_stream", stream) or 0
    st = lib().hweno_max_dt_noalloc(ctypes.byref(grid), float(gamma), ctypes.c_void_p(a), float(cfl),
                                    ctypes.c_void_p(o), ctypes.c_void_p(s))
    if st != 0:
        raise HwenoError(st, "hweno_max_dt_noalloc failed (see stderr)")


def alu_probe(precision="fp64", iters=None, stream=None):
    """Measured FMA throughput of the current device in FLOP/s ("fp64" or "fp32")."""
    if iters is None:
        iters = 40000 if precision == "fp64" else 2000000
    out = ctypes.c_double()
    st = lib().hweno_alu_probe({"fp64": 0, "fp32": 1}[precision], int(iters), ctypes.byref(out), _stream(stream))
    if st != 0:
        raise HwenoError(st, "hweno_alu_probe failed")
    return out.value


def f32_round(x, out, stream=None):
    """The kernels' double -> float rounding of CUDA float64 tensor x into float32 tensor out."""
    a, dev, n = _ptr(_f64(x))
    o, odev, on = _ptr(out)
    if not (dev and odev) or on != n or str(out.dtype) != "torch.float32":
        raise ValueError("x (float64) and out (float32) must be CUDA tensors of the same size")
    st = lib().hweno_f32_round(ctypes.c_void_p(a), ctypes.c_void_p(o), n, _stream(stream))
    if st != 0:
        raise HwenoError(st, "hweno_f32_round failed")


def mlp_nparam():
    return lib().hweno_mlp_nparam()


def _dev(x):
    a, dev, n = _ptr(x)
    if not dev:
        raise ValueError("expected a CUDA tensor")
    return ctypes.c_void_p(a if n else None)


def _stream(stream):
    return ctypes.c_void_p(getattr(stream, "cuda_stream", stream) or 0)


def mlp_forward(params, X, prob, stream=None):
    st = lib().hweno_mlp_forward(_dev(params), _dev(X), int(X.shape[0]), _dev(prob), _stream(stream))
    if st != 0:
        raise HwenoError(st, "hweno_mlp_forward failed")


def mlp_loss_grad(params, X, y, w, grad, loss, stream=None):
    st = lib().hweno_mlp_loss_grad(_dev(params), _dev(X), _dev(y), _dev(w) if w is not None else None,
                                   int(X.shape[0]), _dev(grad), _dev(loss), _stream(stream))
    if st != 0:
        raise HwenoError(st, "hweno_mlp_loss_grad failed")


def mlp_adam(params, grad, m1, m2, step, lr, stream=None):
    st = lib().hweno_mlp_adam(_dev(params), _dev(grad), _dev(m1), _dev(m2), int(step), float(lr), _stream(stream))
    if st != 0:
        raise HwenoError(st, "hweno_mlp_adam failed")


def _grid_struct(dim, nx, ny, x0, x1, y0, y1, eq, adv=(0.0, 0.0), precision="fp64", indicator="kxrcf",
                 gamma_bar=(1.0, 10.0, 100.0, 1000.0), beta_of_q=False):
    g = Grid()
    g.dim, g.nx, g.ny = dim, nx, ny
    g.x0, g.x1, g.y0, g.y1 = x0, x1, y0, y1
    g.eq = EQ[eq]
    g.adv_a, g.adv_b = adv
    g.precision = PREC[precision]
    g.indicator = IND[indicator]
    for k in range(4):
        g.gamma_bar[k] = gamma_bar[k]
    g.beta_of_q = int(bool(beta_of_q))
    return g


class BatchSolver:
    """Independent 2D Euler problems advanced together (hweno_create_batch)."""

    def __init__(self, problems, precision="fp64", indicator="kxrcf", gamma_bar=(1.0, 10.0, 100.0, 1000.0),
                 beta_of_q=False, gamma=1.4, stream=None):
        n = len(problems)
        grids = (Grid * n)()
        bcs = (Bc * n)()
        for k, p in enumerate(problems):
            grids[k] = _grid_struct(2, p.nx, p.ny, p.x0, p.x1, p.y0, p.y1, "euler", precision=precision,
                                    indicator=indicator, gamma_bar=gamma_bar, beta_of_q=beta_of_q)
            bcs[k] = Bc(*[BC[b] for b in p.bc])
        h = ctypes.c_void_p()
        st = lib().hweno_create_batch(grids, bcs, n, float(gamma), ctypes.byref(h))
        if st != 0:
            raise HwenoError(st, "hweno_create_batch failed (see stderr)")
        self._h = h
        self.n = n
        self.shapes = [(4, 3, p.ny, p.nx) for p in problems]
        if stream is not None:
            s = getattr(stream, "cuda_stream", stream) or 0
            self._check(lib().hweno_set_stream(self._h, ctypes.c_void_p(s)))

    def _check(self, st):
        if st != 0:
            raise HwenoError(st, lib().hweno_last_error(self._h).decode())

    def set_positivity_check(self, on=True):
        self._check(lib().hweno_set_positivity_check(self._h, int(bool(on))))

    def set_persistence(self, persist=True):
        self._check(lib().hweno_set_persistence(self._h, int(bool(persist))))

    def close(self):
        if getattr(self, "_h", None):
            lib().hweno_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_moments(self, k, m):
        if isinstance(m, np.ndarray):
            m = np.ascontiguousarray(m)
        addr, dev, n = _ptr(_f64(m))
        self._check(lib().hweno_batch_set_moments(self._h, k, ctypes.c_void_p(addr), n, dev))

    def get_moments(self, k, out=None):
        if out is None:
            out = np.empty(self.shapes[k], np.float64)
        addr, dev, n = _ptr(_f64(out))
        self._check(lib().hweno_batch_get_moments(self._h, k, ctypes.c_void_p(addr), n, dev))
        return out

    def step(self, dt=None, cfl=0.6):
        """dt: None (per-problem CFL dt) or a CUDA float64 tensor of n dts."""
        p = 0
        if dt is not None:
            p, dev, cnt = _ptr(_f64(dt))
            if not dev or cnt != self.n:
                raise ValueError("dt must be a CUDA float64 tensor with one entry per problem")
        self._check(lib().hweno_step_batch(self._h, ctypes.c_void_p(p), float(cfl)))

    def dts(self):
        out = np.empty(self.n, np.float64)
        self._check(lib().hweno_batch_dt(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), self.n))
        return out

    def troubled_mask(self, k):
        out = np.empty((3,) + self.shapes[k][2:], np.uint8)
        self._check(lib().hweno_batch_troubled_mask(self._h, k, ctypes.c_void_p(out.ctypes.data), out.size))
        return out

    def set_tile(self, variant):
        self._check(lib().hweno_batch_set_tile(self._h, int(variant)))

    def set_barrier(self, spin_limit=1 << 26, extra_arrivals=0):
        """Bound of the grid barrier's waits; extra_arrivals > 0 makes every wait
        run out (the timeout path: the next synchronising call raises ETIMEOUT)."""
        self._check(lib().hweno_batch_set_barrier(self._h, int(spin_limit), int(extra_arrivals)))

    def uses_graph(self):
        return lib().hweno_batch_uses_graph(self._h) == 1

    def failed_problems(self):
        """Indices of the problems that made the last reported step non-physical."""
        bits = (ctypes.c_uint * self.n)()
        self._check(lib().hweno_batch_status(self._h, bits, self.n))
        return [k for k in range(self.n) if bits[k]]

    def sync(self):
        self._check(lib().hweno_sync(self._h))
