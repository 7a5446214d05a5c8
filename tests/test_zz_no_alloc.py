"""The allocation-free forward entry point (fdw_forward_static).

It serves callers that cannot call cudaMalloc; it keeps its scratch in a
static device array of the library.  It runs the same step kernel on the same
host tables as fdw_forward, so with the same tiling (tile 0 in 3D, tile 3 in
2D, x chunks of 64 planes, r + 3 stages) its traces are bit for bit those of
fdw_forward, and both are within the FP32 tolerance of the FP64 oracle.

This file is collected last on purpose: a failure here comes after every
other test has run.  It works alone in a fresh process and after the other
tests (the static array is rewritten by every call)."""
import numpy as np
import pytest

from problems import Problem, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module")
def fw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1609_03361_gb300 import build, fdwave
    build.build()
    fdwave.lib()
    return fdwave


def _static_tiling(pb):
    return (0 if pb.ndim == 3 else 3, 64, pb.p // 2 + 3)


def _runtime(fw, pb):
    s = pb.solver(fw, tiling=_static_tiling(pb))
    rec = s.forward(pb.q32)
    s.sync()
    s.close()
    return rec


def _static(fw, pb, fill=float("nan")):
    dev = torch.device("cuda", 0)
    m = torch.from_numpy(pb.m32).to(dev)
    q = torch.from_numpy(pb.q32).to(dev)
    rec = torch.full((pb.nt, pb.rec.shape[0]), fill, device=dev)
    fw.fdw_forward_static(pb.shape, pb.h, pb.p, pb.nbl, pb.dt, pb.nt, pb.vmax, m, pb.src, q,
                          pb.rec, rec)
    return rec.cpu().numpy()


@pytest.mark.parametrize("shape,p,nbl,nt", [((30, 27, 33), 8, 6, 80), ((61, 57), 4, 6, 80),
                                            ((30, 27, 33), 16, 6, 60), ((61, 57), 2, 20, 200)])
def test_static_forward_matches_forward_and_oracle_twice(fw, shape, p, nbl, nt):
    pb = Problem(shape, 10.0, p, nbl, nt, nsrc=2, nrec=9, seed=77 + p)
    ref = _runtime(fw, pb)
    oref = pb.oracle_forward()
    for _ in range(2):   # the second call finds the previous call's contents
        got = _static(fw, pb)
        assert np.isfinite(got).all()
        assert np.array_equal(got, ref)
        assert rel_l2(got, oref) < TOL
        assert np.abs(got - oref).max() <= TOL * np.abs(oref).max()


def test_static_forward_degenerate_cases(fw):
    # one time sample: u^0 = 0 is recorded
    pb = Problem((20, 21, 22), 10.0, 4, 3, 1, nsrc=1, nrec=3, seed=1)
    got = _static(fw, pb)
    assert got.shape == (1, 3) and np.count_nonzero(got) == 0
    # no sources: every trace stays zero
    pb = Problem((20, 21, 22), 10.0, 4, 3, 30, nsrc=0, nrec=4, seed=1)
    assert np.count_nonzero(_static(fw, pb)) == 0
    # no receivers: the call runs and records nothing
    pb = Problem((20, 21, 22), 10.0, 4, 3, 30, nsrc=1, nrec=0, seed=1)
    assert _static(fw, pb).shape == (30, 0)


def test_static_forward_rejects_large_grids_and_bad_tensors(fw):
    dev = torch.device("cuda", 0)
    m = torch.ones((200, 200, 200), device=dev)
    q = torch.zeros((4, 1), device=dev)
    rec = torch.zeros((4, 1), device=dev)
    with pytest.raises(fw.FdwError) as e:
        fw.fdw_forward_static((200, 200, 200), 10.0, 4, 10, 0.1, 4, 1.0, m, [[50.0, 50.0, 50.0]],
                              q, [[60.0, 60.0, 60.0]], rec)
    assert e.value.status == 2
    pb = Problem((20, 21, 22), 10.0, 4, 3, 30, nsrc=1, nrec=3, seed=1)
    m = torch.from_numpy(pb.m32).to(dev)
    q = torch.from_numpy(pb.q32).to(dev)
    for bad in (torch.zeros((30, 3)), torch.zeros((30, 3), device=dev, dtype=torch.float64),
                torch.zeros((3, 30), device=dev).t(), torch.zeros((29, 3), device=dev)):
        with pytest.raises(fw.FdwError) as e:
            fw.fdw_forward_static(pb.shape, pb.h, pb.p, pb.nbl, pb.dt, pb.nt, pb.vmax, m, pb.src,
                                  q, pb.rec, bad)
        assert e.value.status == 1


def test_contexts_keep_working_around_static_calls(fw):
    """A static call configures the step kernel it shares with the contexts
    (tile 3 is the default 2D tile): the contexts' later forward runs and
    single steps must still launch and match the oracle."""
    pb = Problem((61, 57), 10.0, 4, 20, 120, nsrc=1, nrec=11, seed=3)
    oref = pb.oracle_forward()
    s = pb.solver(fw, tiling=(3, 0, 8))   # deeper pipeline than the static call's r + 3
    first = s.forward(pb.q32)
    assert rel_l2(first, oref) < TOL
    assert rel_l2(_static(fw, pb), oref) < TOL
    again = s.forward(pb.q32)
    s.sync()
    assert np.array_equal(again, first)
    dev = torch.device("cuda", 0)
    q = torch.from_numpy(pb.q32).to(dev)
    rec = torch.zeros((pb.nt, 11), device=dev)
    for n in range(pb.nt):
        s.step(n, q, rec)
    s.sync()
    s.close()
    assert np.array_equal(rec.cpu().numpy(), first)
