"""Thin Python binding of libfdwave (``include/fdwave.h``).

The functions ``fdw_*`` below carry the C names and only marshal arguments:
numpy arrays and torch tensors become plain pointers (host or device), torch's
current CUDA stream becomes the ``cudaStream_t``.  Every step of the
computation runs in the CUDA library; when the library is not built or cannot
be loaded every call raises ``FdwError`` (there is no CPU fallback).

``Solver`` bundles one context with convenient array handling and
``FWIGradient`` exposes forward modelling and the FWI gradient as a
``torch.autograd.Function``.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("FDW_LIB_PATH") or os.path.join(_HERE, "libfdwave.so")

FDW_OK = 0
FDW_F32, FDW_F16, FDW_BF16 = 0, 1, 2
FDW_LAYOUT_PHYSICAL, FDW_LAYOUT_COMPUTATIONAL = 0, 1
STATUS = {0: "FDW_OK", 1: "FDW_ERR_ARG", 2: "FDW_ERR_SHAPE", 3: "FDW_ERR_ORDER", 4: "FDW_ERR_CFL",
          5: "FDW_ERR_OUT_OF_DOMAIN", 6: "FDW_ERR_OOM", 7: "FDW_ERR_CUDA", 8: "FDW_ERR_TIMEOUT",
          9: "FDW_ERR_STATE"}
_DTYPES = {"f32": FDW_F32, "fp32": FDW_F32, "float32": FDW_F32, "f16": FDW_F16, "fp16": FDW_F16,
           "float16": FDW_F16, "bf16": FDW_BF16, "bfloat16": FDW_BF16}
_LAYOUTS = {"physical": FDW_LAYOUT_PHYSICAL, "computational": FDW_LAYOUT_COMPUTATIONAL}


class FdwError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        super().__init__(f"{STATUS.get(status, status)}: {msg}")


_lock = threading.Lock()
_lib = None

_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_PP = ctypes.POINTER(ctypes.c_void_p)

# (name, restype, argtypes)
_SIGS = [
    ("fdw_version", _I, []),
    ("fdw_status_string", ctypes.c_char_p, [_I]),
    ("fdw_fd_weights", _I, [_I, ctypes.POINTER(_D)]),
    ("fdw_dt_max", _D, [_I, ctypes.POINTER(_D), _I, _D]),
    ("fdw_create", _I, [ctypes.POINTER(_P), _I, ctypes.POINTER(ctypes.c_int64),
                        ctypes.POINTER(_D), _I, _I, _D, _I, _D, _I]),
    ("fdw_destroy", None, [_P]),
    ("fdw_last_error", ctypes.c_char_p, [_P]),
    ("fdw_set_model", _I, [_P, _P, _I, _I, _P]),
    ("fdw_set_damping", _I, [_P, _P, _P]),
    ("fdw_set_sources", _I, [_P, _I, _P]),
    ("fdw_set_receivers", _I, [_P, _I, _P]),
    ("fdw_forward", _I, [_P, _P, _P, _P]),
    ("fdw_forward_ckpt", _I, [_P, _P, _P, _I, _I, _P]),
    ("fdw_adjoint", _I, [_P, _P, _P, _P]),
    ("fdw_gradient", _I, [_P, _P, _P, _P, _I, _P]),
    ("fdw_get_wavefield", _I, [_P, _I, _P, _P]),
    ("fdw_sync", _I, [_P]),
    ("fdw_autotune", _I, [_P, _I]),
    ("fdw_set_tiling", _I, [_P, _I, _I, _I]),
    ("fdw_get_tiling", _I, [_P, ctypes.POINTER(_I)]),
    ("fdw_set_persistent", _I, [_P, _I]),
    ("fdw_set_time_blocking", _I, [_P, _I, _I, _I, _I]),
    ("fdw_get_time_blocking", _I, [_P, ctypes.POINTER(_I)]),
    ("fdw_batch_create", _I, [ctypes.POINTER(_P), _I, _PP]),
    ("fdw_batch_destroy", None, [_P]),
    ("fdw_batch_last_error", ctypes.c_char_p, [_P]),
    ("fdw_batch_forward", _I, [_P, _PP, _PP, _P]),
    ("fdw_batch_forward_ckpt", _I, [_P, _PP, _PP, _I, _I, _P]),
    ("fdw_batch_gradient", _I, [_P, _PP, _PP, _PP, _I, _P]),
    ("fdw_batch_autotune", _I, [_P, _I]),
    ("fdw_batch_get_tiling", _I, [_P, ctypes.POINTER(_I)]),
    ("fdw_forward_static", _I, [_I, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(_D), _I, _I,
                                _D, _I, _D, _P, _I, _P, _P, _I, _P, _P, _P]),
    ("fdw_diffusion2d", _I, [_P, _P, ctypes.c_int64, ctypes.c_int64, _D, _D, _D, _D, _I, _I, _P]),
    ("fdw_set_checkpoint_budget", _I, [_P, _I]),
    ("fdw_create_slab", _I, [ctypes.POINTER(_P), _I, ctypes.POINTER(ctypes.c_int64),
                             ctypes.POINTER(_D), _I, _I, _D, _I, _D, _I, ctypes.c_int64,
                             ctypes.c_int64]),
    ("fdw_step", _I, [_P, _I, _P, _P, _P]),
    ("fdw_halo_planes", _I, [_P, _I, _PP, _PP, _PP, _PP, ctypes.POINTER(ctypes.c_int64)]),
    ("fdw_exchange_ghosts", _I, [_P, _P, _I, _P]),
    ("fdw_halo_copy", _I, [_P, _I, _I, _P, _P, _P]),
    ("fdw_checkpoint_schedule", _I, [_I, _I, ctypes.POINTER(_I), _I]),
]


def lib():
    """Load libfdwave.so (built in-tree); raise FdwError when it is missing."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise FdwError(7, f"{LIB_PATH} is not built (python -m paper_1609_03361_gb300.build)")
            try:
                L = ctypes.CDLL(LIB_PATH)
            except OSError as e:
                raise FdwError(7, f"cannot load {LIB_PATH}: {e}") from e
            for name, res, args in _SIGS:
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def declared_symbols():
    return [s[0] for s in _SIGS]


# ------------------------------------------------------------------ marshalling

def _torch():
    import torch
    return torch


def _is_tensor(x):
    return type(x).__module__.startswith("torch") and hasattr(x, "data_ptr")


def _ptr(x, keep, dtype=np.float32):
    """Plain pointer to the data of a numpy array / torch tensor / int / None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if _is_tensor(x):
        torch = _torch()
        want = {np.float32: torch.float32, np.float64: torch.float64}[dtype]
        if x.dtype != want or not x.is_contiguous():
            x = x.to(want).contiguous()
        keep.append(x)
        return x.data_ptr()
    a = np.ascontiguousarray(x, dtype=dtype)
    keep.append(a)
    return a.ctypes.data


def _stream(stream, device):
    if stream is None:
        try:
            torch = _torch()
            if torch.cuda.is_available():
                return torch.cuda.current_stream(device).cuda_stream
        except Exception:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(st, ctx=None, batch=None):
    if st != FDW_OK:
        msg = ""
        if ctx:
            msg = (lib().fdw_last_error(ctx) or b"").decode()
        elif batch:
            msg = (lib().fdw_batch_last_error(batch) or b"").decode()
        raise FdwError(st, msg)


# ------------------------------------------------------------------ C names

def fdw_version():
    return lib().fdw_version()


def fdw_fd_weights(space_order):
    c = (ctypes.c_double * 9)()
    _check(lib().fdw_fd_weights(int(space_order), c))
    return np.array(c[: space_order // 2 + 1])


def fdw_dt_max(ndim, spacing, space_order, vmax):
    sp = np.broadcast_to(np.asarray(spacing, dtype=np.float64), (ndim,)).copy()
    return lib().fdw_dt_max(int(ndim), sp.ctypes.data_as(ctypes.POINTER(_D)), int(space_order),
                            float(vmax))


def fdw_create(shape, spacing, space_order, nbl, dt, nt, vmax, device=0):
    ndim = len(shape)
    sh = (ctypes.c_int64 * ndim)(*[int(s) for s in shape])
    sp = np.broadcast_to(np.asarray(spacing, dtype=np.float64), (ndim,)).copy()
    out = _P()
    _check(lib().fdw_create(ctypes.byref(out), ndim, sh, sp.ctypes.data_as(ctypes.POINTER(_D)),
                            int(space_order), int(nbl), float(dt), int(nt), float(vmax),
                            int(device)))
    return out.value


def fdw_create_slab(shape, spacing, space_order, nbl, dt, nt, vmax, device, x_begin, x_end):
    ndim = len(shape)
    sh = (ctypes.c_int64 * ndim)(*[int(s) for s in shape])
    sp = np.broadcast_to(np.asarray(spacing, dtype=np.float64), (ndim,)).copy()
    out = _P()
    _check(lib().fdw_create_slab(ctypes.byref(out), ndim, sh, sp.ctypes.data_as(ctypes.POINTER(_D)),
                                 int(space_order), int(nbl), float(dt), int(nt), float(vmax),
                                 int(device), int(x_begin), int(x_end)))
    return out.value


def fdw_step(ctx, n, q, rec, stream=None, device=0):
    keep = []
    _check(lib().fdw_step(ctx, int(n), _ptr(q, keep), _ptr(rec, keep), _stream(stream, device)),
           ctx)


def fdw_halo_planes(ctx, n):
    """(send_lo, send_hi, recv_lo, recv_hi, count): device addresses and float
    count of the ghost-plane blocks of a slab after step n."""
    ptrs = [_P() for _ in range(4)]
    cnt = ctypes.c_int64()
    _check(lib().fdw_halo_planes(ctx, int(n), *[ctypes.byref(p) for p in ptrs], ctypes.byref(cnt)),
           ctx)
    return tuple(p.value for p in ptrs) + (cnt.value,)


def fdw_exchange_ghosts(lower, upper, n, stream=None, device=0):
    _check(lib().fdw_exchange_ghosts(lower, upper, int(n), _stream(stream, device)), upper)


def fdw_halo_copy(ctx, n, direction, lo, hi, stream=None, device=0):
    keep = []
    _check(lib().fdw_halo_copy(ctx, int(n), int(direction), _ptr(lo, keep), _ptr(hi, keep),
                               _stream(stream, device)), ctx)


def fdw_destroy(ctx):
    if ctx:
        lib().fdw_destroy(ctx)


def fdw_set_model(ctx, m, layout=FDW_LAYOUT_PHYSICAL, m_dtype=FDW_F32, stream=None, device=0):
    keep = []
    _check(lib().fdw_set_model(ctx, _ptr(m, keep), int(layout), int(m_dtype),
                               _stream(stream, device)), ctx)


def fdw_set_damping(ctx, eta, stream=None, device=0):
    keep = []
    _check(lib().fdw_set_damping(ctx, _ptr(eta, keep), _stream(stream, device)), ctx)


def fdw_set_sources(ctx, xyz):
    keep = []
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    _check(lib().fdw_set_sources(ctx, xyz.shape[0] if xyz.size else 0, _ptr(xyz, keep, np.float64)),
           ctx)


def fdw_set_receivers(ctx, xyz):
    keep = []
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    _check(lib().fdw_set_receivers(ctx, xyz.shape[0] if xyz.size else 0,
                                   _ptr(xyz, keep, np.float64)), ctx)


def fdw_forward(ctx, q, rec, stream=None, device=0):
    keep = []
    _check(lib().fdw_forward(ctx, _ptr(q, keep), _ptr(rec, keep), _stream(stream, device)), ctx)


def fdw_forward_ckpt(ctx, q, rec, ckpt_every, snap_dtype=FDW_F16, stream=None, device=0):
    keep = []
    _check(lib().fdw_forward_ckpt(ctx, _ptr(q, keep), _ptr(rec, keep), int(ckpt_every),
                                  int(snap_dtype), _stream(stream, device)), ctx)


def fdw_adjoint(ctx, d, qadj, stream=None, device=0):
    keep = []
    _check(lib().fdw_adjoint(ctx, _ptr(d, keep), _ptr(qadj, keep), _stream(stream, device)), ctx)


def fdw_gradient(ctx, resid, resid_sub, grad, grad_layout=FDW_LAYOUT_COMPUTATIONAL, stream=None,
                 device=0):
    keep = []
    _check(lib().fdw_gradient(ctx, _ptr(resid, keep), _ptr(resid_sub, keep), _ptr(grad, keep),
                              int(grad_layout), _stream(stream, device)), ctx)


def fdw_get_wavefield(ctx, which, out, stream=None, device=0):
    keep = []
    _check(lib().fdw_get_wavefield(ctx, int(which), _ptr(out, keep), _stream(stream, device)), ctx)


def fdw_sync(ctx):
    _check(lib().fdw_sync(ctx), ctx)


def fdw_autotune(ctx, steps=10):
    _check(lib().fdw_autotune(ctx, int(steps)), ctx)


def fdw_set_tiling(ctx, tile=-1, xchunk=0, stages=0):
    _check(lib().fdw_set_tiling(ctx, int(tile), int(xchunk), int(stages)), ctx)


def fdw_set_persistent(ctx, on=True):
    _check(lib().fdw_set_persistent(ctx, 1 if on else 0), ctx)


def fdw_set_time_blocking(ctx, steps_per_pass, variant=-1, xchunk=0, stages=0):
    _check(lib().fdw_set_time_blocking(ctx, int(steps_per_pass), int(variant), int(xchunk),
                                       int(stages)), ctx)


def fdw_get_time_blocking(ctx):
    out = (ctypes.c_int * 5)()
    _check(lib().fdw_get_time_blocking(ctx, out), ctx)
    return dict(zip(("steps", "variant", "xchunk", "stages", "units"), list(out)))


def fdw_set_checkpoint_budget(ctx, max_pairs):
    _check(lib().fdw_set_checkpoint_budget(ctx, int(max_pairs)), ctx)


def fdw_checkpoint_schedule(nseg, nslots):
    """Binomial checkpoint schedule as a list of (op, arg): 1 advance to
    segment arg, 2 store in slot arg, 3 restore slot arg (-1: zero state),
    4 reverse segment arg."""
    n = lib().fdw_checkpoint_schedule(int(nseg), int(nslots), None, 0)
    if n < 0:
        raise FdwError(1, "bad schedule arguments")
    buf = (ctypes.c_int * (2 * max(n, 1)))()
    m = lib().fdw_checkpoint_schedule(int(nseg), int(nslots), buf, n)
    assert m == n
    return [(buf[2 * i], buf[2 * i + 1]) for i in range(n)]


def fdw_get_tiling(ctx):
    out = (ctypes.c_int * 5)()
    _check(lib().fdw_get_tiling(ctx, out), ctx)
    return dict(zip(("tile", "xchunk", "stages", "ctas", "units"), list(out)))


def _ptr_array(xs, keep, dtype=np.float32):
    arr = (ctypes.c_void_p * len(xs))(*[_ptr(x, keep, dtype) for x in xs])
    keep.append(arr)
    return arr


def fdw_batch_create(ctxs):
    arr = (ctypes.c_void_p * len(ctxs))(*ctxs)
    out = _P()
    _check(lib().fdw_batch_create(ctypes.byref(out), len(ctxs), arr))
    return out.value


def fdw_batch_destroy(b):
    if b:
        lib().fdw_batch_destroy(b)


def fdw_batch_forward(b, qs, recs, stream=None, device=0):
    keep = []
    _check(lib().fdw_batch_forward(b, _ptr_array(qs, keep), _ptr_array(recs, keep),
                                   _stream(stream, device)), batch=b)


def fdw_batch_forward_ckpt(b, qs, recs, ckpt_every, snap_dtype=FDW_F16, stream=None, device=0):
    keep = []
    _check(lib().fdw_batch_forward_ckpt(b, _ptr_array(qs, keep), _ptr_array(recs, keep),
                                        int(ckpt_every), int(snap_dtype),
                                        _stream(stream, device)), batch=b)


def fdw_batch_gradient(b, resids, subs, grads, grad_layout=FDW_LAYOUT_COMPUTATIONAL, stream=None,
                       device=0):
    keep = []
    sub = _ptr_array(subs, keep) if subs is not None else None
    _check(lib().fdw_batch_gradient(b, _ptr_array(resids, keep), sub, _ptr_array(grads, keep),
                                    int(grad_layout), _stream(stream, device)), batch=b)


def fdw_batch_autotune(b, steps=10):
    _check(lib().fdw_batch_autotune(b, int(steps)), batch=b)


def fdw_batch_get_tiling(b):
    out = (ctypes.c_int * 5)()
    _check(lib().fdw_batch_get_tiling(b, out), batch=b)
    return dict(zip(("tile", "xchunk", "stages", "ctas", "units"), list(out)))


def fdw_forward_static(shape, spacing, space_order, nbl, dt, nt, vmax, m, src_xyz, q, rec_xyz,
                       rec, stream=None, device=0):
    """Allocation-free forward modelling of a small problem (see include/fdwave.h).

    m (physical shape), q [nt][nsrc] and rec [nt][nrec] must be contiguous
    float32 CUDA tensors on ``device``: the call writes the traces into ``rec``
    itself, so no converted copy is made; coordinates are host arrays."""
    torch = _torch()
    ndim = len(shape)
    src = np.ascontiguousarray(src_xyz, dtype=np.float64).reshape(-1, ndim)
    rcv = np.ascontiguousarray(rec_xyz, dtype=np.float64).reshape(-1, ndim)
    dev = torch.device("cuda", device) if isinstance(device, int) else torch.device(device)
    want = {"m": (m, int(np.prod([int(v) for v in shape]))), "q": (q, int(nt) * src.shape[0]),
            "rec": (rec, int(nt) * rcv.shape[0])}
    for name, (t, n) in want.items():
        if not (_is_tensor(t) and t.is_cuda and t.device == dev and t.dtype == torch.float32
                and t.is_contiguous()):
            raise FdwError(1, f"{name} must be a contiguous float32 CUDA tensor on {dev}")
        if t.numel() != n:
            raise FdwError(1, f"{name} has {t.numel()} elements, expected {n}")
    sh = (ctypes.c_int64 * ndim)(*[int(v) for v in shape])
    sp = np.broadcast_to(np.asarray(spacing, dtype=np.float64), (ndim,)).copy()
    _check(lib().fdw_forward_static(ndim, sh, sp.ctypes.data_as(ctypes.POINTER(_D)),
                                    int(space_order), int(nbl), float(dt), int(nt), float(vmax),
                                    m.data_ptr(), src.shape[0],
                                    src.ctypes.data if src.size else None, q.data_ptr(),
                                    rcv.shape[0], rcv.ctypes.data if rcv.size else None,
                                    rec.data_ptr(), _stream(stream, dev)))


def fdw_diffusion2d(u, tmp, dx, dy, alpha, dt, steps, steps_per_pass=0, stream=None):
    """2D diffusion of Sec. 4 in place on ``u`` (see include/fdwave.h): ``u`` and
    ``tmp`` are contiguous float32 CUDA tensors of shape (nx, ny); ``tmp`` is
    scratch (allocated here when None)."""
    torch = _torch()
    if not (_is_tensor(u) and u.is_cuda and u.dtype == torch.float32 and u.is_contiguous()
            and u.dim() == 2):
        raise FdwError(1, "u must be a contiguous 2-D float32 CUDA tensor (updated in place)")
    if tmp is None:
        tmp = torch.empty_like(u)
    if tmp.shape != u.shape or tmp.dtype != u.dtype or not tmp.is_contiguous() or not tmp.is_cuda:
        raise FdwError(1, "tmp must match u")
    nx, ny = u.shape
    _check(lib().fdw_diffusion2d(u.data_ptr(), tmp.data_ptr(), int(nx), int(ny), float(dx),
                                 float(dy), float(alpha), float(dt), int(steps),
                                 int(steps_per_pass), _stream(stream, u.device)))
    return u


# ------------------------------------------------------------------ objects

class Solver:
    """One shot on one GPU.  Arrays may be numpy (host) or torch tensors (host or
    CUDA); outputs are allocated like the first array argument of the call."""

    def __init__(self, shape, spacing, space_order, nbl, dt, nt, vmax, device=0, slab=None):
        """slab = (x_begin, x_end): only those computational x planes (fdw_create_slab)."""
        self.shape = tuple(int(s) for s in shape)
        self.ndim = len(self.shape)
        self.spacing = tuple(np.broadcast_to(np.asarray(spacing, dtype=np.float64),
                                             (self.ndim,)).tolist())
        self.space_order, self.nbl, self.dt, self.nt = int(space_order), int(nbl), float(dt), int(nt)
        self.vmax, self.device = float(vmax), int(device)
        self.slab = None if slab is None else (int(slab[0]), int(slab[1]))
        if self.slab is None:
            self.ctx = fdw_create(self.shape, self.spacing, space_order, nbl, dt, nt, vmax, device)
        else:
            self.ctx = fdw_create_slab(self.shape, self.spacing, space_order, nbl, dt, nt, vmax,
                                       device, *self.slab)
        self.nsrc = 0
        self.nrec = 0

    def close(self):
        if getattr(self, "ctx", None):
            fdw_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def comp_shape(self):
        """Shape of the computational arrays of this context (for a slab: its
        own planes plus r ghost planes on either side, in x)."""
        full = tuple(n + 2 * self.nbl for n in self.shape)
        if self.slab is None:
            return full
        r = self.space_order // 2
        return (self.slab[1] - self.slab[0] + 2 * r,) + full[1:]

    def _like(self, ref, shape):
        if _is_tensor(ref):
            torch = _torch()
            return torch.empty(shape, dtype=torch.float32, device=ref.device)
        return np.empty(shape, dtype=np.float32)

    def set_model(self, m, layout="physical", dtype="f32", stream=None):
        fdw_set_model(self.ctx, m, _LAYOUTS[layout], _DTYPES[dtype], stream, self.device)

    def set_damping(self, eta, stream=None):
        fdw_set_damping(self.ctx, eta, stream, self.device)

    def set_sources(self, xyz):
        xyz = np.asarray(xyz, dtype=np.float64).reshape(-1, self.ndim)
        fdw_set_sources(self.ctx, xyz)
        self.nsrc = xyz.shape[0]

    def set_receivers(self, xyz):
        xyz = np.asarray(xyz, dtype=np.float64).reshape(-1, self.ndim)
        fdw_set_receivers(self.ctx, xyz)
        self.nrec = xyz.shape[0]

    def forward(self, q, rec=None, stream=None):
        if rec is None:
            rec = self._like(q, (self.nt, self.nrec))
        fdw_forward(self.ctx, q, rec, stream, self.device)
        return rec

    def forward_ckpt(self, q, ckpt_every, snap_dtype="f16", rec=None, stream=None):
        if rec is None:
            rec = self._like(q, (self.nt, self.nrec))
        fdw_forward_ckpt(self.ctx, q, rec, ckpt_every, _DTYPES[snap_dtype], stream, self.device)
        return rec

    def adjoint(self, d, qadj=None, stream=None):
        if qadj is None:
            qadj = self._like(d, (self.nt, self.nsrc))
        fdw_adjoint(self.ctx, d, qadj, stream, self.device)
        return qadj

    def gradient(self, resid, resid_sub=None, layout="computational", grad=None, stream=None):
        if grad is None:
            shape = self.comp_shape if layout == "computational" else self.shape
            grad = self._like(resid, shape)
        fdw_gradient(self.ctx, resid, resid_sub, grad, _LAYOUTS[layout], stream, self.device)
        return grad

    def wavefield(self, which=0, out=None, like=None, stream=None):
        if out is None:
            out = self._like(like, self.comp_shape)
        fdw_get_wavefield(self.ctx, which, out, stream, self.device)
        return out

    def sync(self):
        fdw_sync(self.ctx)

    def autotune(self, steps=10):
        fdw_autotune(self.ctx, steps)

    def step(self, n, q, rec, stream=None):
        """One time step (device arrays q [nt][nsrc], rec [nt][nrec])."""
        fdw_step(self.ctx, n, q, rec, stream, self.device)

    def halo_planes(self, n):
        return fdw_halo_planes(self.ctx, n)

    def set_checkpoint_budget(self, max_pairs):
        fdw_set_checkpoint_budget(self.ctx, max_pairs)

    def set_tiling(self, tile=-1, xchunk=0, stages=0):
        fdw_set_tiling(self.ctx, tile, xchunk, stages)

    def tiling(self):
        return fdw_get_tiling(self.ctx)

    def set_persistent(self, on=True):
        """Plain forward runs as one persistent launch over all time steps."""
        fdw_set_persistent(self.ctx, on)

    def set_time_blocking(self, steps_per_pass, variant=-1, xchunk=0, stages=0):
        """Plain forward runs advance two time steps per launch (steps_per_pass=2)."""
        fdw_set_time_blocking(self.ctx, steps_per_pass, variant, xchunk, stages)

    def time_blocking(self):
        return fdw_get_time_blocking(self.ctx)


class Batch:
    """Several Solvers stepped together (one launch per time step for all)."""

    def __init__(self, solvers):
        self.solvers = list(solvers)
        self.b = fdw_batch_create([s.ctx for s in self.solvers])

    def close(self):
        if getattr(self, "b", None):
            fdw_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def forward(self, qs, recs=None, stream=None):
        if recs is None:
            recs = [s._like(q, (s.nt, s.nrec)) for s, q in zip(self.solvers, qs)]
        fdw_batch_forward(self.b, qs, recs, stream, self.solvers[0].device)
        return recs

    def forward_ckpt(self, qs, ckpt_every, snap_dtype="f16", recs=None, stream=None):
        if recs is None:
            recs = [s._like(q, (s.nt, s.nrec)) for s, q in zip(self.solvers, qs)]
        fdw_batch_forward_ckpt(self.b, qs, recs, ckpt_every, _DTYPES[snap_dtype], stream,
                               self.solvers[0].device)
        return recs

    def gradient(self, resids, subs=None, layout="computational", grads=None, stream=None):
        if grads is None:
            grads = [s._like(r, s.comp_shape if layout == "computational" else s.shape)
                     for s, r in zip(self.solvers, resids)]
        fdw_batch_gradient(self.b, resids, subs, grads, _LAYOUTS[layout], stream,
                           self.solvers[0].device)
        return grads

    def autotune(self, steps=10):
        fdw_batch_autotune(self.b, steps)

    def tiling(self):
        return fdw_batch_get_tiling(self.b)


def _make_fwi_function():
    torch = _torch()

    class FWIGradient(torch.autograd.Function):
        """traces = F(m): forward modelling of one shot as a function of the
        physical squared-slowness model m (CUDA tensor).  The backward pass is
        the adjoint-state gradient with checkpointed recomputation."""

        @staticmethod
        def forward(ctx, m, solver, q, ckpt_every=10, snap_dtype="f16", m_dtype="f32"):
            solver.set_model(m.detach().contiguous(), "physical", m_dtype)
            rec = solver.forward_ckpt(q, ckpt_every, snap_dtype)
            ctx.solver = solver
            return rec

        @staticmethod
        def backward(ctx, grad_rec):
            g = ctx.solver.gradient(grad_rec.contiguous(), None, "physical")
            return g, None, None, None, None, None

    return FWIGradient


_fwi = None


def fwi_traces(m, solver, q, ckpt_every=10, snap_dtype="f16", m_dtype="f32"):
    """Differentiable receiver traces of one shot (see FWIGradient)."""
    global _fwi
    if _fwi is None:
        _fwi = _make_fwi_function()
    return _fwi.apply(m, solver, q, ckpt_every, snap_dtype, m_dtype)
