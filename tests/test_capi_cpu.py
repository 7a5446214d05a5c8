"""C ABI checks that need no GPU: the library loads, exports every symbol that
include/*.h declares, and its host-side logic (stencil weights, stability limit,
argument validation) is correct.  No kernel is launched here."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fw():
    from paper_1609_03361_gb300 import build, fdwave
    build.build()
    return fdwave


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"\b(fdw_[a-z0-9_]+)\s*\(", txt):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol(fw):
    names = _declared()
    assert len(names) >= 25
    L = ctypes.CDLL(fw.LIB_PATH)
    missing = [n for n in sorted(names) if not hasattr(L, n)]
    assert not missing, missing
    # the binding declares exactly the header's functions
    assert set(fw.declared_symbols()) == names


def test_library_links_no_driver(fw):
    # the CUDA driver is reached through the runtime's entry-point query only
    out = os.popen(f"ldd {fw.LIB_PATH}").read()
    assert "libcuda.so" not in out


@pytest.mark.parametrize("p", range(2, 17, 2))
def test_host_weights_match_oracle(fw, p):
    # two independent implementations: Fornberg recursion (library) and the
    # closed form (oracle)
    a = fw.fdw_fd_weights(p)
    b = oracle.fd_weights(p)
    assert np.allclose(a, b, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("ndim,p,h,v", [(2, 4, 10.0, 1.5), (3, 8, 12.5, 2.625), (3, 16, 7.0, 4.5),
                                        (3, 2, (10.0, 12.5, 5.0), 3.0)])
def test_host_dt_max_matches_oracle(fw, ndim, p, h, v):
    assert fw.fdw_dt_max(ndim, h, p, v) == pytest.approx(oracle.dt_max(ndim, h, p, v), rel=1e-12)


def test_argument_validation_before_any_device_work(fw):
    F = fw.FdwError
    with pytest.raises(F) as e:
        fw.fdw_create((10, 10, 10), 10.0, 7, 4, 1.0, 10, 2.0)
    assert e.value.status == 3  # odd order
    with pytest.raises(F) as e:
        fw.fdw_create((10, 10, 10), 10.0, 18, 4, 1.0, 10, 2.0)
    assert e.value.status == 3
    with pytest.raises(F) as e:
        fw.fdw_create((10, 1, 10), 10.0, 4, 4, 1.0, 10, 2.0)
    assert e.value.status == 2  # dimension < 2
    dtm = fw.fdw_dt_max(3, 10.0, 8, 2.0)
    with pytest.raises(F) as e:
        fw.fdw_create((10, 10, 10), 10.0, 8, 4, dtm * 1.001, 10, 2.0)
    assert e.value.status == 4  # above the stability limit
    assert fw.fdw_dt_max(3, 10.0, 5, 2.0) < 0
    assert fw.fdw_dt_max(4, 10.0, 4, 2.0) < 0


def test_status_strings(fw):
    L = fw.lib()
    for st in range(10):
        assert L.fdw_status_string(st)
    assert L.fdw_version() >= 100


def test_diffusion_host_checks(fw):
    # argument checks that return before any device call (the pointers are
    # never dereferenced)
    f = fw.lib().fdw_diffusion2d
    lim = 0.1 ** 4 / (2 * 1.0 * 2 * 0.1 ** 2)  # Eq. 2 for dx = dy = 0.1, alpha = 1
    assert f(16, 32, 10, 10, 0.1, 0.1, 1.0, lim * 1.001, 3, 0, None) == 4   # FDW_ERR_CFL
    assert f(16, 32, 10, 10, 0.1, 0.1, 1.0, lim, 3, 3, None) == 1         # steps_per_pass
    assert f(16, 16, 10, 10, 0.1, 0.1, 1.0, lim, 3, 0, None) == 1         # u == tmp
    assert f(16, 32, 2, 10, 0.1, 0.1, 1.0, lim, 3, 0, None) == 1          # nx < 3
    assert f(16, 32, 10, 10, 0.1, 0.1, -1.0, lim, 3, 0, None) == 1        # alpha <= 0
    assert f(None, 32, 10, 10, 0.1, 0.1, 1.0, lim, 3, 0, None) == 1       # null field


# ---------------------------------------------------------------- allocation-free entry point
# Every check below returns before the library makes any CUDA call: sizes,
# order, stability and point locations are host logic, and a host buffer is
# refused (FDW_ERR_ARG) instead of reaching a kernel as a device address.

def _static(fw, shape, p, nbl, dt, nt, vmax, m, src, q, rec_xyz, rec):
    import ctypes
    ndim = len(shape)
    sh = (ctypes.c_int64 * ndim)(*shape)
    sp = (ctypes.c_double * ndim)(*([10.0] * ndim))
    src = np.ascontiguousarray(src, dtype=np.float64).reshape(-1, ndim)
    rcv = np.ascontiguousarray(rec_xyz, dtype=np.float64).reshape(-1, ndim)
    return fw.lib().fdw_forward_static(
        ndim, sh, sp, p, nbl, dt, nt, vmax, m.ctypes.data, src.shape[0],
        src.ctypes.data if src.size else None, q.ctypes.data, rcv.shape[0],
        rcv.ctypes.data if rcv.size else None, rec.ctypes.data, None)


def test_static_forward_host_checks(fw):
    shape, p, nbl, nt, vmax = (20, 18, 22), 8, 4, 10, 2.0
    dt = 0.9 * fw.fdw_dt_max(3, 10.0, p, vmax)
    m = np.ones(shape, np.float32)
    q = np.zeros((nt, 1), np.float32)
    src = [[50.0, 50.0, 50.0]]
    rec1 = [[60.0, 60.0, 60.0]]
    out = np.zeros((nt, 1), np.float32)
    # more receivers than the static tables hold (4096): FDW_ERR_SHAPE
    many = np.tile(np.array(rec1), (4097, 1))
    assert _static(fw, shape, p, nbl, dt, nt, vmax, m, src, q, many,
                   np.zeros((nt, 4097), np.float32)) == 2
    # a grid beyond 4096 computational points per axis: FDW_ERR_SHAPE
    assert _static(fw, (5000, 4), 4, 0, dt, nt, vmax, m, [[1.0, 1.0]], q, [[2.0, 2.0]], out) == 2
    # odd order, dt above the stability limit
    assert _static(fw, shape, 7, nbl, dt, nt, vmax, m, src, q, rec1, out) == 3
    assert _static(fw, shape, p, nbl, 1.01 * fw.fdw_dt_max(3, 10.0, p, vmax), nt, vmax, m, src, q,
                   rec1, out) == 4
    # a source or a receiver outside [0, (N-1) h]: FDW_ERR_OUT_OF_DOMAIN
    assert _static(fw, shape, p, nbl, dt, nt, vmax, m, [[50.0, 171.0, 50.0]], q, rec1, out) == 5
    assert _static(fw, shape, p, nbl, dt, nt, vmax, m, src, q, [[-0.5, 60.0, 60.0]], out) == 5
    # every check passes but m, q and rec are host buffers: FDW_ERR_ARG
    assert _static(fw, shape, p, nbl, dt, nt, vmax, m, src, q, rec1, out) == 1
