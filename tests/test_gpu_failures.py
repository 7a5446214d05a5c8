"""Host-side failure paths of a context: points outside the domain, calls out
of order and a failed device allocation.  Each failure is made on the host
(no kernel faults or hangs): the call returns its status before any device
work, and the context computes correct traces afterwards.  A context needs a
device, so these run on the GPU; the checks that need none are in
test_capi_cpu.py."""
import os

import numpy as np
import pytest

from problems import Problem, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-4
OUT_OF_DOMAIN, OOM, STATE = 5, 6, 9


@pytest.fixture(scope="module")
def fw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1609_03361_gb300 import build, fdwave
    build.build()
    fdwave.lib()
    return fdwave


class _FailAllocations:
    """Every device allocation of the library fails while inside the block
    (the library's FDW_TEST_FAIL_ALLOC hook; no allocator call is made)."""

    def __enter__(self):
        os.environ["FDW_TEST_FAIL_ALLOC"] = "1"

    def __exit__(self, *exc):
        os.environ.pop("FDW_TEST_FAIL_ALLOC", None)


def _problem():
    return Problem((24, 21, 26), 10.0, 8, 5, 50, nsrc=2, nrec=6, seed=17)


def test_points_outside_the_domain(fw):
    pb = _problem()
    s = pb.solver(fw)
    top = np.array([(n - 1) * pb.h for n in pb.shape])
    for bad in ([-1e-9, 10.0, 10.0], [10.0, top[1] + 1e-6, 10.0], [10.0, 10.0, np.nan]):
        with pytest.raises(fw.FdwError) as e:
            s.set_sources(np.vstack([pb.src, bad]))
        assert e.value.status == OUT_OF_DOMAIN
        with pytest.raises(fw.FdwError) as e:
            s.set_receivers(np.vstack([pb.rec, bad]))
        assert e.value.status == OUT_OF_DOMAIN
    # the last accepted points stay in force
    s.nsrc, s.nrec = pb.src.shape[0], pb.rec.shape[0]
    rec = s.forward(pb.q32)
    s.sync()
    s.close()
    assert rel_l2(rec, pb.oracle_forward()) < TOL


def test_calls_out_of_order(fw):
    pb = _problem()
    s = fw.Solver(pb.shape, pb.h, pb.p, pb.nbl, pb.dt, pb.nt, pb.vmax)
    s.set_sources(pb.src)
    s.set_receivers(pb.rec)
    with pytest.raises(fw.FdwError) as e:
        s.forward(pb.q32)                      # no model yet
    assert e.value.status == STATE
    with pytest.raises(fw.FdwError) as e:
        s.adjoint(np.zeros((pb.nt, 6), np.float32))
    assert e.value.status == STATE
    s.set_model(pb.m32)
    with pytest.raises(fw.FdwError) as e:
        s.gradient(np.zeros((pb.nt, 6), np.float32))   # no checkpointed forward
    assert e.value.status == STATE
    rec = s.forward(pb.q32)
    with pytest.raises(fw.FdwError) as e:
        s.gradient(np.zeros((pb.nt, 6), np.float32))   # a plain forward keeps no checkpoints
    assert e.value.status == STATE
    s.sync()
    s.close()
    assert rel_l2(rec, pb.oracle_forward()) < TOL


def test_failed_allocations_leave_the_context_usable(fw):
    pb = _problem()
    # creation itself
    with _FailAllocations():
        with pytest.raises(fw.FdwError) as e:
            fw.Solver(pb.shape, pb.h, pb.p, pb.nbl, pb.dt, pb.nt, pb.vmax)
    assert e.value.status == OOM
    s = fw.Solver(pb.shape, pb.h, pb.p, pb.nbl, pb.dt, pb.nt, pb.vmax)
    s.set_model(pb.m32)
    s.set_sources(pb.src)
    s.set_receivers(pb.rec)
    # the plan (unit tables, descriptors, tickets) of the first forward
    with _FailAllocations():
        with pytest.raises(fw.FdwError) as e:
            s.forward(pb.q32)
    assert e.value.status == OOM
    ref = pb.oracle_forward()
    rec = s.forward(pb.q32)
    assert rel_l2(rec, ref) < TOL
    # new receivers: the device point tables
    with _FailAllocations():
        with pytest.raises(fw.FdwError) as e:
            s.set_receivers(pb.rec[::-1].copy())
    assert e.value.status == OOM
    assert np.array_equal(s.forward(pb.q32), rec)   # the old receivers stay in force
    # the checkpoint store of a checkpointed forward, then the gradient
    with _FailAllocations():
        with pytest.raises(fw.FdwError) as e:
            s.forward_ckpt(pb.q32, 7, "f32")
    assert e.value.status == OOM
    resid = np.random.default_rng(2).standard_normal((pb.nt, 6)).astype(np.float32)
    s.forward_ckpt(pb.q32, 7, "f32")
    g = s.gradient(resid)
    # a model storage type change: the model buffer is reallocated
    with _FailAllocations():
        with pytest.raises(fw.FdwError) as e:
            s.set_model(pb.m32, "physical", "f16")
    assert e.value.status == OOM
    with pytest.raises(fw.FdwError) as e:
        s.forward(pb.q32)                      # no model stored any more
    assert e.value.status == STATE
    s.set_model(pb.m32)
    assert np.array_equal(s.forward(pb.q32), rec)
    s.sync()
    s.close()
    assert rel_l2(g, pb.oracle_gradient(resid)) < TOL


def test_tiling_arguments(fw):
    """Tile indices and pipeline depths outside their ranges are refused
    before any launch: every tile needs r + 2 stages except tile 9, whose
    stages each hold one plane's reads and pipeline from two; the context then
    runs at a valid tiling."""
    ARG = 1
    pb = _problem()
    s = pb.solver(fw)
    for bad in [(10, 0, 0), (-2, 0, 0), (9, 0, 1), (7, 0, 5), (4, 0, 1), (4, -1, 0)]:
        with pytest.raises(fw.FdwError) as e:
            s.set_tiling(*bad)
        assert e.value.status == ARG, bad
    s.set_tiling(9, 0, 2)
    rec = s.forward(pb.q32)
    s.sync()
    assert s.tiling()["stages"] == 2
    assert rel_l2(rec, pb.oracle_forward()) < TOL
    s.close()
