"""Gradient under a checkpoint budget (binomial schedule) through the C ABI.

With FP32 checkpoints every recomputed forward state is a bit-exact copy of
the one the unlimited budget restores, and the adjoint steps run in the same
order, so the gradient must be identical bit for bit; with FP16 checkpoints
it must stay within the FP16 snapshot tolerance of the FP64 oracle."""
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


def _grad(fw, pb, k, stype, budget, resid):
    s = pb.solver(fw)
    s.set_checkpoint_budget(budget)
    rec = s.forward_ckpt(pb.q32, k, stype)
    g = s.gradient(resid)
    s.sync()
    s.close()
    return rec, g


@pytest.fixture(scope="module")
def case():
    pb = Problem((27, 24, 30), 10.0, 8, 6, 95, nsrc=2, nrec=9, seed=71)
    resid = np.random.default_rng(12).standard_normal((pb.nt, 9)).astype(np.float32)
    return pb, resid


@pytest.mark.parametrize("k,budget", [(7, 1), (7, 2), (7, 5), (10, 3), (1, 4), (3, 1)])
def test_budget_gradient_is_bitwise_unlimited(fw, case, k, budget):
    pb, resid = case
    rec0, g0 = _grad(fw, pb, k, "f32", 0, resid)
    rec1, g1 = _grad(fw, pb, k, "f32", budget, resid)
    assert np.array_equal(rec1, rec0)
    assert np.array_equal(g1, g0)


def test_budget_gradient_fp16_matches_oracle(fw, case):
    pb, resid = case
    _, g = _grad(fw, pb, 6, "f16", 2, resid)
    assert rel_l2(g, pb.oracle_gradient(resid)) < 1e-2


def test_budget_repeated_and_changed(fw, case):
    pb, resid = case
    _, g0 = _grad(fw, pb, 7, "f32", 0, resid)
    s = pb.solver(fw)
    s.set_checkpoint_budget(2)
    s.forward_ckpt(pb.q32, 7, "f32")
    a = s.gradient(resid)
    with pytest.raises(fw.FdwError):
        s.gradient(resid)          # the schedule consumed the checkpoints
    s.forward_ckpt(pb.q32, 7, "f32")
    b = s.gradient(resid)
    s.forward_ckpt(pb.q32, 7, "f32")
    s.set_checkpoint_budget(4)
    with pytest.raises(fw.FdwError):
        s.gradient(resid)          # the stored pairs follow the old budget
    s.forward_ckpt(pb.q32, 7, "f32")
    c = s.gradient(resid)
    s.set_checkpoint_budget(0)     # back to one pair per segment: repeatable
    s.forward_ckpt(pb.q32, 7, "f32")
    d = s.gradient(resid)
    e = s.gradient(resid)
    s.sync()
    s.close()
    for g in (a, b, c, d, e):
        assert np.array_equal(g, g0)


def test_batched_budget_gradient(fw):
    shapes = [(21, 20, 19), (24, 17, 22)]
    pbs = [Problem(sh, 12.5, 4, 5, 50, nsrc=1, nrec=5, seed=80 + i) for i, sh in enumerate(shapes)]
    dt = min(pb.dt for pb in pbs)
    vmax = max(pb.vmax for pb in pbs)
    import oracle
    for pb in pbs:
        pb.dt, pb.vmax = dt, vmax
        pb.setup = oracle.Setup(pb.shape, pb.h, pb.p, pb.nbl, dt, pb.nt)
    rng = np.random.default_rng(3)
    res = [rng.standard_normal((pb.nt, 5)).astype(np.float32) for pb in pbs]
    solvers = [pb.solver(fw) for pb in pbs]
    for s in solvers:
        s.set_checkpoint_budget(2)
    b = fw.Batch(solvers)
    b.forward_ckpt([pb.q32 for pb in pbs], 6, "f32")
    grads = b.gradient(res)
    for s in solvers:
        s.sync()
    b.close()
    for s in solvers:
        s.close()
    for pb, g, r in zip(pbs, grads, res):
        _, g0 = _grad(fw, pb, 6, "f32", 0, r)
        assert np.array_equal(g, g0)
