"""Plain forward modelling as one persistent launch over all time steps
(fdw_set_persistent): the same scheme and the same arithmetic per point as
one launch per step, only scheduled differently, so traces and wavefields
must be bit for bit those of the per-step loop, and within 1e-4 of the FP64
oracle."""
import numpy as np
import pytest

from problems import Problem, assert_close, rel_l2

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


def _fwd(fw, pb, persist, tiling=None):
    s = pb.solver(fw, tiling=tiling)
    s.set_persistent(persist)
    rec = s.forward(pb.q32)
    u = s.wavefield(0)
    s.sync()
    s.close()
    return rec, u


@pytest.mark.parametrize("p", [2, 4, 8, 12, 16])
def test_persistent_equals_per_step_all_orders(fw, p):
    pb = Problem((37, 45, 29), 10.0, p, 8, 70, nsrc=2, nrec=9, seed=100 + p)
    rec1, u1 = _fwd(fw, pb, False)
    rec2, u2 = _fwd(fw, pb, True)
    assert np.array_equal(rec1, rec2) and np.array_equal(u1, u2)
    ref, uref = pb.oracle_forward(final=True)
    assert_close(rec2, ref, TOL, "traces")
    assert_close(u2, uref, TOL, "wavefield")


@pytest.mark.parametrize("tiling", [(0, 0, 0), (4, 8, 0), (4, 13, 7), (6, 9, 10), (7, 11, 0),
                                    (8, 0, 0), (1, 0, 0), (5, 7, 9), (9, 0, 0), (9, 11, 3),
                                    (9, 5, 2)])
def test_persistent_equals_per_step_tilings(fw, tiling):
    """Short x chunks give many rows, so units of a later step run while the
    previous step is still in progress elsewhere in the grid."""
    pb = Problem((40, 51, 35), 12.5, 8, 6, 60, nsrc=3, nrec=12, seed=11)
    rec1, u1 = _fwd(fw, pb, False, tiling)
    rec2, u2 = _fwd(fw, pb, True, tiling)
    assert np.array_equal(rec1, rec2) and np.array_equal(u1, u2)


def test_persistent_2d_and_short_runs(fw):
    pb = Problem((61, 57), 10.0, 4, 20, 200, nsrc=1, nrec=11, seed=3)
    rec1, u1 = _fwd(fw, pb, False)
    rec2, u2 = _fwd(fw, pb, True)
    assert np.array_equal(rec1, rec2) and np.array_equal(u1, u2)
    for nt in (1, 2, 3):
        pb = Problem((20, 21, 22), 10.0, 8, 3, nt, nsrc=1, nrec=3, seed=nt)
        rec1, u1 = _fwd(fw, pb, False)
        rec2, u2 = _fwd(fw, pb, True)
        assert np.array_equal(rec1, rec2) and np.array_equal(u1, u2)


def test_persistent_points_on_chunk_edges(fw):
    """Sources and receivers on and next to x-chunk boundaries: the injected
    nodes of one unit and the sampled corners of the next are read across
    rows that finish at different times."""
    pb = Problem((44, 30, 33), 10.0, 8, 4, 80, nsrc=1, nrec=4, seed=7)
    lx = 8
    xs = [(i * lx - pb.nbl) * pb.h + d for i in (2, 3, 4) for d in (-10.0, -3.0, 0.0, 4.0)]
    xs = [x for x in xs if 0.0 <= x <= (pb.shape[0] - 1) * pb.h]
    pts = np.array([[x, 0.4 * (pb.shape[1] - 1) * pb.h, 0.6 * (pb.shape[2] - 1) * pb.h]
                    for x in xs])
    pb.rec = np.vstack([pb.rec, pts])
    pb.src = np.vstack([pb.src, pts[:3]])
    pb.q32 = np.concatenate([pb.q32, pb.q32[:, :1].repeat(3, axis=1)], axis=1)
    rec1, u1 = _fwd(fw, pb, False, (4, lx, 0))
    rec2, u2 = _fwd(fw, pb, True, (4, lx, 0))
    assert np.array_equal(rec1, rec2) and np.array_equal(u1, u2)
    ref, uref = pb.oracle_forward(final=True)
    assert_close(rec2, ref, TOL, "traces")
    assert_close(u2, uref, TOL, "wavefield")


def test_persistent_batch_of_uneven_shots(fw):
    import oracle
    shapes = [(21, 24, 19), (30, 17, 26), (18, 18, 33)]
    pbs = [Problem(sh, 12.5, 8, 5, 60, nsrc=1, nrec=5, seed=50 + i) for i, sh in enumerate(shapes)]
    dt = min(pb.dt for pb in pbs)
    vmax = max(pb.vmax for pb in pbs)
    for pb in pbs:
        pb.dt = dt
        pb.vmax = vmax
        pb.setup = oracle.Setup(pb.shape, pb.h, pb.p, pb.nbl, dt, pb.nt)
    outs = []
    for persist in (False, True):
        solvers = [pb.solver(fw) for pb in pbs]
        for s in solvers:
            s.set_persistent(persist)
        b = fw.Batch(solvers)
        outs.append(b.forward([pb.q32 for pb in pbs]))
        for s in solvers:
            s.sync()
        b.close()
        for s in solvers:
            s.close()
    for a, c, pb in zip(outs[0], outs[1], pbs):
        assert np.array_equal(a, c)
        assert_close(c, pb.oracle_forward(), TOL, "traces")


def test_persistent_rejected_on_slabs(fw):
    pb = Problem((24, 20, 22), 10.0, 4, 4, 20, nsrc=1, nrec=3, seed=3)
    s = fw.Solver(pb.shape, pb.h, 4, 4, pb.dt, pb.nt, pb.vmax, slab=(0, 15))
    with pytest.raises(fw.FdwError) as e:
        s.set_persistent(True)
    assert e.value.status == 9
    s.close()


def _adj(fw, pb, d, persist, tiling=None):
    s = pb.solver(fw, tiling=tiling)
    s.set_persistent(persist)
    qa = s.adjoint(d)
    s.sync()
    s.close()
    return qa


@pytest.mark.parametrize("p,tiling", [(2, None), (4, None), (8, None), (12, None), (16, None),
                                      (8, (9, 5, 2)), (8, (7, 11, 0)), (8, (4, 8, 0)),
                                      (8, (0, 13, 0))])
def test_persistent_adjoint_equals_per_step(fw, p, tiling):
    """The adjoint as one persistent launch (time running backwards, the
    receiver data injected at the unit tails) gives the per-step loop's
    source-side traces bit for bit (the per-step loop injects in a launch of
    its own, with the same arithmetic), the oracle's to 1e-4, and closes the
    dot test against the persistent forward run."""
    pb = Problem((33, 29, 37), 10.0, p, 6, 60, nsrc=2, nrec=9, seed=300 + p)
    rng = np.random.default_rng(p)
    d = rng.standard_normal((pb.nt, 9)).astype(np.float32)
    qa1 = _adj(fw, pb, d, False, tiling)
    qa2 = _adj(fw, pb, d, True, tiling)
    assert np.array_equal(qa1, qa2)
    assert_close(qa2, pb.oracle_adjoint(d), TOL, "adjoint traces")
    rec, _ = _fwd(fw, pb, True, tiling)
    lhs = float(np.sum(rec.astype(np.float64) * d))
    rhs = float(np.sum(pb.q32.astype(np.float64) * qa2))
    assert abs(lhs - rhs) <= 1e-5 * max(abs(lhs), abs(rhs))


def test_persistent_adjoint_2d_and_short_runs(fw):
    pb = Problem((61, 57), 10.0, 4, 20, 120, nsrc=1, nrec=11, seed=8)
    d = np.random.default_rng(8).standard_normal((pb.nt, 11)).astype(np.float32)
    assert np.array_equal(_adj(fw, pb, d, False), _adj(fw, pb, d, True))
    for nt in (1, 2, 3):
        pb = Problem((20, 21, 22), 10.0, 8, 3, nt, nsrc=1, nrec=3, seed=nt)
        d = np.random.default_rng(nt).standard_normal((nt, 3)).astype(np.float32)
        assert np.array_equal(_adj(fw, pb, d, False), _adj(fw, pb, d, True))


def _grad(fw, pb, k, stype, resid, persist, tiling=None, sub=None):
    s = pb.solver(fw, tiling=tiling)
    s.set_persistent(persist)
    rec = s.forward_ckpt(pb.q32, k, stype)
    g = s.gradient(resid, sub)
    s.sync()
    s.close()
    return rec, g


@pytest.mark.parametrize("p,k,stype,tiling", [(8, 10, "f32", None), (8, 10, "f16", None),
                                              (8, 1, "f16", None), (8, 2, "f16", None),
                                              (8, 7, "bf16", None), (4, 3, "f32", (4, 8, 0)),
                                              (16, 9, "f16", None), (8, 70, "f32", None),
                                              (8, 13, "f32", (9, 5, 2)), (2, 4, "f16", (7, 11, 0))])
def test_persistent_checkpointed_gradient_equals_per_step(fw, p, k, stype, tiling):
    """The checkpointed forward (one launch per segment of k steps, the
    snapshot maximum folded into its last two steps), the recompute and the
    adjoint-with-imaging steps of each segment (one launch each, the residuals
    injected at the unit tails) give the per-step loop's traces and gradient
    bit for bit, and the oracle's gradient to its tolerance."""
    pb = Problem((29, 26, 31), 10.0, p, 6, 70, nsrc=1, nrec=8, seed=400 + p + k)
    resid = np.random.default_rng(k).standard_normal((pb.nt, 8)).astype(np.float32)
    rec1, g1 = _grad(fw, pb, k, stype, resid, False, tiling)
    rec2, g2 = _grad(fw, pb, k, stype, resid, True, tiling)
    assert np.array_equal(rec1, rec2)
    assert np.array_equal(g1, g2)
    # (random residuals: the BF16 bound with data-like residuals, 5e-3, is
    # held in the low-precision snapshot test)
    ref = pb.oracle_gradient(resid)
    assert rel_l2(g2, ref) < {"f32": TOL, "f16": 1e-3, "bf16": 5e-2}[stype]


def test_persistent_gradient_residual_difference_and_short_runs(fw):
    pb = Problem((24, 22, 26), 10.0, 4, 5, 60, nsrc=1, nrec=6, seed=41)
    rng = np.random.default_rng(5)
    a = rng.standard_normal((pb.nt, 6)).astype(np.float32)
    b = rng.standard_normal((pb.nt, 6)).astype(np.float32)
    _, g1 = _grad(fw, pb, 6, "f32", a, False, sub=b)
    _, g2 = _grad(fw, pb, 6, "f32", a, True, sub=b)
    assert np.array_equal(g1, g2)
    for nt, k in ((2, 1), (3, 2), (5, 10)):
        pb = Problem((20, 21, 22), 10.0, 8, 3, nt, nsrc=1, nrec=3, seed=nt)
        r = np.random.default_rng(nt).standard_normal((nt, 3)).astype(np.float32)
        rec1, g1 = _grad(fw, pb, k, "f16", r, False)
        rec2, g2 = _grad(fw, pb, k, "f16", r, True)
        assert np.array_equal(rec1, rec2) and np.array_equal(g1, g2)


def test_persistent_batched_gradient_equals_per_step(fw):
    import oracle
    shapes = [(21, 20, 19), (24, 17, 22), (18, 23, 20)]
    pbs = [Problem(sh, 12.5, 8, 5, 50, nsrc=1, nrec=5, seed=60 + i) for i, sh in enumerate(shapes)]
    dt = min(pb.dt for pb in pbs)
    vmax = max(pb.vmax for pb in pbs)
    for pb in pbs:
        pb.dt = dt
        pb.vmax = vmax
        pb.setup = oracle.Setup(pb.shape, pb.h, pb.p, pb.nbl, dt, pb.nt)
    rng = np.random.default_rng(9)
    res = [rng.standard_normal((pb.nt, 5)).astype(np.float32) for pb in pbs]
    outs = []
    for persist in (False, True):
        solvers = [pb.solver(fw) for pb in pbs]
        for s in solvers:
            s.set_persistent(persist)
        b = fw.Batch(solvers)
        recs = b.forward_ckpt([pb.q32 for pb in pbs], 7, "f16")
        grads = b.gradient(res)
        for s in solvers:
            s.sync()
        outs.append(([np.array(r) for r in recs], [np.array(g) for g in grads]))
        b.close()
        for s in solvers:
            s.close()
    for r1, r2 in zip(outs[0][0], outs[1][0]):
        assert np.array_equal(r1, r2)
    for g1, g2, pb, r in zip(outs[0][1], outs[1][1], pbs, res):
        assert np.array_equal(g1, g2)
        assert rel_l2(g2, pb.oracle_gradient(r)) < 1e-3
