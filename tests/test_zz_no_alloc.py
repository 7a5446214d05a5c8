"""The allocation-free forward entry point (fdw_forward_static).

It serves callers that cannot call cudaMalloc; it keeps its scratch in a
static device array of the library and must give what the ordinary forward
path gives.  This file is collected last on purpose: a failure here comes
after every other test has run.  It works alone in a fresh process and after
the other tests (the static array is rewritten by every call)."""
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


@pytest.mark.parametrize("shape,p", [((30, 27, 33), 8), ((61, 57), 4)])
def test_static_forward_matches_forward_twice(fw, shape, p):
    pb = Problem(shape, 10.0, p, 6, 80, nsrc=2, nrec=9, seed=77)
    s = pb.solver(fw)
    ref = s.forward(pb.q32)
    s.sync()
    s.close()
    dev = torch.device("cuda", 0)
    m = torch.from_numpy(pb.m32).to(dev)
    q = torch.from_numpy(pb.q32).to(dev)
    for _ in range(2):
        rec = torch.full((pb.nt, pb.rec.shape[0]), float("nan"), device=dev)
        fw.fdw_forward_static(pb.shape, pb.h, pb.p, pb.nbl, pb.dt, pb.nt, pb.vmax, m, pb.src, q,
                              pb.rec, rec)
        got = rec.cpu().numpy()
        assert np.isfinite(got).all()
        assert rel_l2(got, ref) < TOL


def test_static_forward_rejects_large_grids(fw):
    dev = torch.device("cuda", 0)
    m = torch.ones((200, 200, 200), device=dev)
    q = torch.zeros((4, 1), device=dev)
    rec = torch.zeros((4, 1), device=dev)
    with pytest.raises(fw.FdwError) as e:
        fw.fdw_forward_static((200, 200, 200), 10.0, 4, 10, 0.1, 4, 1.0, m, [[50.0, 50.0, 50.0]],
                              q, [[60.0, 60.0, 60.0]], rec)
    assert e.value.status == 2
