"""Failure detection on the GPU without a fault: every wait of the step kernel
is bounded.  With the test hook FDW_TEST_STALL (direct launches only) the
producer issues no loads, every consumer wait runs out of its clock budget
(about 2 s), the kernel records the error and returns; fdw_sync reports
FDW_ERR_TIMEOUT and the context stays usable."""
import numpy as np
import pytest

from problems import Problem, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1609_03361_gb300 import build, fdwave
    build.build()
    fdwave.lib()
    return fdwave


def test_bounded_wait_reports_timeout_and_context_survives(fw, monkeypatch):
    pb = Problem((20, 22, 24), 10.0, 4, 4, 2, nsrc=1, nrec=3, seed=5)
    s = pb.solver(fw)
    monkeypatch.setenv("FDW_NO_GRAPH", "1")
    monkeypatch.setenv("FDW_TEST_STALL", "1")
    s.forward(pb.q32)
    with pytest.raises(fw.FdwError) as e:
        s.sync()
    assert e.value.status == 8  # FDW_ERR_TIMEOUT
    monkeypatch.delenv("FDW_TEST_STALL")
    rec = s.forward(pb.q32)
    s.sync()
    s.close()
    assert rel_l2(rec, pb.oracle_forward()) < 1e-4
