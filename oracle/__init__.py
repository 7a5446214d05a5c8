"""FP64 CPU oracle for the damped acoustic wave equation -- TEST INFRASTRUCTURE.

This package wraps ``fdw_oracle.c`` (plain C, double precision) with ctypes and
numpy.  It is the independent reference the CUDA library is checked against:
only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  It shares no code with the CUDA library.

Each function follows a passage of arXiv 1609.03361 (Devito); the C file names
the section, equation or listing next to each routine.

Conventions: 2D fields are ``[nx][nz]`` and 3D fields ``[nx][ny][nz]`` (last
axis contiguous) on the *computational* grid, i.e. the physical shape plus
``nbl`` absorbing-layer points on every side.  Point coordinates are
``[npts][ndim]`` arrays in metres relative to the physical origin.  Units:
velocity km/s (= m/ms), spacing m, time ms, ``m = 1/v**2``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fdw_oracle.c")
_LIB = os.path.join(_HERE, "_liboracle.so")
_lock = threading.Lock()
_lib = None


class OracleError(RuntimeError):
    pass


_ERRORS = {1: "bad argument", 2: "bad space order", 3: "point outside the physical domain",
           4: "out of memory"}


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_liboracle.so`` (gcc, -O2, OpenMP)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Setup(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("shape", ctypes.c_int64 * 3),
                ("spacing", ctypes.c_double * 3), ("space_order", ctypes.c_int),
                ("nbl", ctypes.c_int), ("dt", ctypes.c_double), ("nt", ctypes.c_int)]


_D = ctypes.POINTER(ctypes.c_double)
_I64 = ctypes.POINTER(ctypes.c_int64)
_SP = ctypes.POINTER(_Setup)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.orc_fd_weights.argtypes = [ctypes.c_int, _D]
            lib.orc_stability_sum.argtypes = [ctypes.c_int]
            lib.orc_stability_sum.restype = ctypes.c_double
            lib.orc_dt_max.argtypes = [ctypes.c_int, _D, ctypes.c_int, ctypes.c_double]
            lib.orc_dt_max.restype = ctypes.c_double
            lib.orc_extend_model.argtypes = [_SP, _D, _D]
            lib.orc_fold_model.argtypes = [_SP, _D, _D]
            lib.orc_damping.argtypes = [_SP, ctypes.c_double, _D]
            lib.orc_interp.argtypes = [_SP, ctypes.c_int, _D, _I64, _D]
            lib.orc_forward.argtypes = [_SP, _D, _D, ctypes.c_int, _D, _D, ctypes.c_int, _D, _D, _D, _D]
            lib.orc_adjoint.argtypes = [_SP, _D, _D, ctypes.c_int, _D, _D, ctypes.c_int, _D, _D, _D]
            lib.orc_gradient.argtypes = [_SP, _D, _D, ctypes.c_int, _D, _D, ctypes.c_int, _D, _D, _D]
            lib.orc_points.argtypes = [_SP]
            lib.orc_points.restype = ctypes.c_int64
            lib.orc_diffusion.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_int, _D]
            _lib = lib
    return _lib


def _dp(a):
    if a is None:
        return None
    return a.ctypes.data_as(_D)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _check(rc):
    if rc != 0:
        raise OracleError(_ERRORS.get(rc, f"error {rc}"))


class Setup:
    """Grid and time axis of one problem (physical shape, spacing, order, layer, dt, nt)."""

    def __init__(self, shape, spacing, space_order, nbl, dt, nt):
        self.shape = tuple(int(s) for s in shape)
        self.ndim = len(self.shape)
        if self.ndim not in (2, 3):
            raise ValueError("ndim must be 2 or 3")
        sp = spacing if np.ndim(spacing) else [spacing] * self.ndim
        self.spacing = tuple(float(h) for h in sp)
        self.space_order = int(space_order)
        self.nbl = int(nbl)
        self.dt = float(dt)
        self.nt = int(nt)

    @property
    def comp_shape(self):
        return tuple(n + 2 * self.nbl for n in self.shape)

    def _c(self):
        s = _Setup()
        s.ndim = self.ndim
        for a in range(3):
            s.shape[a] = self.shape[a] if a < self.ndim else 1
            s.spacing[a] = self.spacing[a] if a < self.ndim else 1.0
        s.space_order = self.space_order
        s.nbl = self.nbl
        s.dt = self.dt
        s.nt = self.nt
        return s


def fd_weights(p: int) -> np.ndarray:
    """Closed-form central 2nd-derivative weights c_0..c_r for order p (Sec. 3.1)."""
    c = np.zeros(9)
    _check(_load().orc_fd_weights(int(p), _dp(c)))
    return c[: p // 2 + 1].copy()


def stability_sum(p: int) -> float:
    return float(_load().orc_stability_sum(int(p)))


def dt_max(ndim: int, spacing, p: int, vmax: float) -> float:
    sp = _f64(spacing if np.ndim(spacing) else [spacing] * ndim)
    return float(_load().orc_dt_max(int(ndim), _dp(sp), int(p), float(vmax)))


def extend_model(setup: Setup, m_phys) -> np.ndarray:
    """Physical-shape model -> computational grid by edge repetition."""
    m_phys = _f64(m_phys, setup.shape)
    out = np.empty(setup.comp_shape)
    s = setup._c()
    _check(_load().orc_extend_model(ctypes.byref(s), _dp(m_phys), _dp(out)))
    return out


def fold_model(setup: Setup, g_comp) -> np.ndarray:
    """Adjoint of ``extend_model``: a computational-grid field (the gradient
    with respect to the extended model) summed onto the physical model."""
    g_comp = _f64(g_comp, setup.comp_shape)
    out = np.empty(setup.shape)
    s = setup._c()
    _check(_load().orc_fold_model(ctypes.byref(s), _dp(g_comp), _dp(out)))
    return out


def damping(setup: Setup, vmax: float) -> np.ndarray:
    """Quadratic absorbing-layer damping field eta on the computational grid."""
    out = np.empty(setup.comp_shape)
    s = setup._c()
    _check(_load().orc_damping(ctypes.byref(s), float(vmax), _dp(out)))
    return out


def interp(setup: Setup, coords):
    """Flat corner indices [npts][2^ndim] and multilinear weights (Sec. 5.2)."""
    coords = _f64(coords).reshape(-1, setup.ndim)
    n = coords.shape[0]
    nc = 1 << setup.ndim
    idx = np.zeros((n, nc), dtype=np.int64)
    w = np.zeros((n, nc))
    s = setup._c()
    _check(_load().orc_interp(ctypes.byref(s), n, _dp(coords), idx.ctypes.data_as(_I64), _dp(w)))
    return idx, w


def forward(setup: Setup, m, eta, src, q, rec, history=False, final=False):
    """Forward modelling (Sec. 5.1 Listing 6 + Sec. 5.2).  Returns traces [nt][nrec]
    (and the history [nt][*comp_shape] and/or the last field when asked)."""
    m = _f64(m, setup.comp_shape)
    eta = _f64(eta, setup.comp_shape)
    src = _f64(src).reshape(-1, setup.ndim)
    rec = _f64(rec).reshape(-1, setup.ndim)
    ns, nr = src.shape[0], rec.shape[0]
    q = _f64(q).reshape(setup.nt, ns)
    out = np.zeros((setup.nt, nr))
    hist = np.zeros((setup.nt,) + setup.comp_shape) if history else None
    fin = np.zeros(setup.comp_shape) if final else None
    s = setup._c()
    _check(_load().orc_forward(ctypes.byref(s), _dp(m), _dp(eta), ns, _dp(src), _dp(q), nr,
                               _dp(rec), _dp(out), _dp(hist), _dp(fin)))
    res = [out]
    if history:
        res.append(hist)
    if final:
        res.append(fin)
    return res[0] if len(res) == 1 else tuple(res)


def adjoint(setup: Setup, m, eta, rec, d, src, history=False):
    """Adjoint modelling (Sec. 5.1 Listing 7): data [nt][nrec] -> source-side
    traces [nt][nsrc] (and the adjoint field history when asked)."""
    m = _f64(m, setup.comp_shape)
    eta = _f64(eta, setup.comp_shape)
    src = _f64(src).reshape(-1, setup.ndim)
    rec = _f64(rec).reshape(-1, setup.ndim)
    ns, nr = src.shape[0], rec.shape[0]
    d = _f64(d).reshape(setup.nt, nr)
    out = np.zeros((setup.nt, ns))
    hist = np.zeros((setup.nt,) + setup.comp_shape) if history else None
    s = setup._c()
    _check(_load().orc_adjoint(ctypes.byref(s), _dp(m), _dp(eta), nr, _dp(rec), _dp(d), ns,
                               _dp(src), _dp(out), _dp(hist)))
    return (out, hist) if history else out


def gradient(setup: Setup, m, eta, src, q, rec, resid):
    """Exact discrete gradient w.r.t. m (computational grid) of sum <resid, P_r u>."""
    m = _f64(m, setup.comp_shape)
    eta = _f64(eta, setup.comp_shape)
    src = _f64(src).reshape(-1, setup.ndim)
    rec = _f64(rec).reshape(-1, setup.ndim)
    ns, nr = src.shape[0], rec.shape[0]
    q = _f64(q).reshape(setup.nt, ns)
    resid = _f64(resid).reshape(setup.nt, nr)
    g = np.zeros(setup.comp_shape)
    s = setup._c()
    _check(_load().orc_gradient(ctypes.byref(s), _dp(m), _dp(eta), ns, _dp(src), _dp(q), nr,
                                _dp(rec), _dp(resid), _dp(g)))
    return g


def diffusion(u0, dx, dy, alpha, dt, steps):
    """Forward-Euler 2D diffusion (Sec. 4, Eq. 1), interior points only."""
    u = np.array(u0, dtype=np.float64, order="C", copy=True)
    nx, ny = u.shape
    _check(_load().orc_diffusion(nx, ny, float(dx), float(dy), float(alpha), float(dt),
                                 int(steps), _dp(u)))
    return u
