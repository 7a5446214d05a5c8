"""Two time steps per launch (temporal blocking of the forward scheme) against
the FP64 oracle and against the one-step loop.

The two-step kernel recomputes the first step on a halo of r rows / planes
around each output tile (16 or 32 rows at order 2, 12 or 28 at order 4, by 56
points) and adds the sources that fall in that halo itself, so sources and receivers are placed on
and across tile and x-chunk boundaries.  Tolerances: relative L2 <= 1e-4
against the oracle (the FP32 accuracy target); against the one-step GPU loop,
which evaluates each point with the same arithmetic, relative L2 <= 1e-6.
"""
import numpy as np
import pytest

from problems import Problem, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-4
TOL_GPU = 1e-6


@pytest.fixture(scope="module")
def fw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1609_03361_gb300 import build, fdwave
    build.build()
    fdwave.lib()
    return fdwave


def _boundary_points(pb, ty, xchunk, rng):
    """Points on and next to output-tile edges (y multiples of ty, z = 56)
    and x-chunk edges, in physical coordinates."""
    h, nbl = pb.h, pb.nbl
    top = np.array([(n - 1) * h for n in pb.shape])
    pts = []
    for k in range(1, 4):
        for off in (-1.0, -0.5, 0.0, 0.25, 1.0):
            x = ((k * xchunk if xchunk else 20) - nbl + off) * h
            y = (k * ty - nbl + off) * h
            z = (56 - nbl + off) * h
            pts.append([x, y, z])
            pts.append([rng.uniform(0, top[0]), y, rng.uniform(0, top[2])])
    return np.clip(np.array(pts), 0.0, top)


def _run(fw, pb, steps, variant=-1, xchunk=0, mtype="f32"):
    s = pb.solver(fw, mtype=mtype)
    if steps == 2:
        s.set_time_blocking(2, variant, xchunk)
    rec = s.forward(pb.q32)
    u = s.wavefield(0)
    info = s.time_blocking()
    s.sync()
    s.close()
    return rec, u, info


TILE_ROWS = {(2, 0): 16, (4, 0): 12, (2, 1): 32, (4, 1): 28}


@pytest.mark.parametrize("p", [2, 4])
@pytest.mark.parametrize("variant,xchunk,nt", [(0, 0, 61), (1, 0, 60), (0, 9, 60), (1, 13, 61)])
def test_two_step_matches_oracle_and_one_step(fw, p, variant, xchunk, nt):
    pb = Problem((37, 45, 70), 10.0, p, 8, nt, nsrc=2, nrec=9, seed=p + 3 * variant)
    rng = np.random.default_rng(p)
    ty = TILE_ROWS[(p, variant)]
    extra = _boundary_points(pb, ty, xchunk, rng)
    pb.rec = np.vstack([pb.rec, extra])
    pb.src = np.vstack([pb.src, extra[::5]])
    nsrc = pb.src.shape[0]
    pb.q32 = np.stack([pb.q32[:, i % 2] * (1 + 0.1 * i) for i in range(nsrc)], axis=1)
    rec1, u1, info1 = _run(fw, pb, 1)
    rec2, u2, info2 = _run(fw, pb, 2, variant, xchunk)
    assert info1["steps"] == 1
    assert info2["steps"] == 2 and info2["variant"] == variant and info2["units"] > 1
    if xchunk:
        assert info2["xchunk"] == xchunk
    ref, uref = pb.oracle_forward(final=True)
    assert np.abs(ref).max() > 0
    assert rel_l2(rec2, ref) < TOL
    assert rel_l2(u2, uref) < TOL
    assert rel_l2(rec2, rec1) < TOL_GPU
    assert rel_l2(u2, u1) < TOL_GPU


@pytest.mark.parametrize("mtype", ["f16", "bf16"])
def test_two_step_low_precision_model(fw, mtype):
    pb = Problem((40, 33, 61), 12.5, 4, 6, 50, nsrc=2, nrec=10, seed=21)
    rec1, u1, _ = _run(fw, pb, 1, mtype=mtype)
    rec2, u2, _ = _run(fw, pb, 2, 0, 0, mtype=mtype)
    assert np.abs(rec1).max() > 0
    assert rel_l2(rec2, rec1) < TOL_GPU
    assert rel_l2(u2, u1) < TOL_GPU


@pytest.mark.parametrize("nt", [1, 2, 3, 4, 5])
def test_two_step_short_runs(fw, nt):
    pb = Problem((20, 22, 64), 10.0, 2, 4, nt, nsrc=1, nrec=5, seed=nt, ongrid=True)
    rec1, u1, _ = _run(fw, pb, 1)
    rec2, u2, _ = _run(fw, pb, 2)
    assert rel_l2(rec2, rec1) < TOL_GPU or np.abs(rec1).max() == 0
    assert np.allclose(rec2, rec1, atol=1e-6 * max(np.abs(rec1).max(), 1e-30))
    assert np.allclose(u2, u1, atol=1e-6 * max(np.abs(u1).max(), 1e-30))


def test_two_step_batched(fw):
    pbs = [Problem(sh, 10.0, 4, 5, 41, nsrc=1, nrec=7, seed=i)
           for i, sh in enumerate([(30, 26, 60), (24, 40, 33), (35, 31, 47)])]
    dt = min(pb.dt for pb in pbs)
    vmax = max(pb.vmax for pb in pbs)
    solvers, singles = [], []
    for pb in pbs:
        pb.dt = dt
        s = fw.Solver(pb.shape, pb.h, pb.p, pb.nbl, dt, pb.nt, vmax)
        s.set_model(pb.m32)
        s.set_sources(pb.src)
        s.set_receivers(pb.rec)
        singles.append(s.forward(pb.q32))
        s.set_time_blocking(2)
        solvers.append(s)
    b = fw.Batch(solvers)
    recs = b.forward([pb.q32 for pb in pbs])
    for r, ref in zip(recs, singles):
        assert np.abs(ref).max() > 0
        assert rel_l2(r, ref) < TOL_GPU
    b.close()
    for s in solvers:
        s.close()


def test_two_step_device_arrays_and_repeat(fw):
    pb = Problem((33, 29, 58), 10.0, 4, 6, 40, nsrc=1, nrec=6, seed=4)
    s = pb.solver(fw)
    s.set_time_blocking(2, 1)
    q = torch.from_numpy(pb.q32).cuda()
    a = s.forward(q).cpu().numpy()
    b = s.forward(q).cpu().numpy()
    s.sync()
    s.close()
    assert np.array_equal(a, b)           # deterministic: no atomics
    ref = pb.oracle_forward()
    assert rel_l2(a, ref) < TOL


def test_two_step_rejected_and_fallbacks(fw):
    pb = Problem((24, 20, 30), 10.0, 6, 4, 20, nsrc=1, nrec=3, seed=3)
    s = pb.solver(fw)
    with pytest.raises(fw.FdwError):
        s.set_time_blocking(2)            # order 6: no two-step kernel
    with pytest.raises(fw.FdwError):
        s.set_time_blocking(3)
    s.close()
    p4 = Problem((24, 20, 30), 10.0, 4, 4, 20, nsrc=1, nrec=3, seed=3)
    s = p4.solver(fw)
    with pytest.raises(fw.FdwError):
        s.set_time_blocking(2, 0, 0, 4)   # fewer than 2r + 1 stages
    s.close()
    p2 = Problem((40, 41), 10.0, 4, 4, 20, nsrc=1, nrec=3, seed=3)
    s = p2.solver(fw)
    with pytest.raises(fw.FdwError):
        s.set_time_blocking(2)            # 2D grid
    s.close()
    s = fw.Solver(pb.shape, pb.h, 4, 4, pb.dt, pb.nt, pb.vmax, slab=(0, 15))
    with pytest.raises(fw.FdwError):
        s.set_time_blocking(2)            # slab context
    s.close()
    # a damping field: the forward runs one step per launch, same traces
    p3 = Problem((26, 24, 60), 10.0, 4, 5, 30, nsrc=1, nrec=4, seed=8)
    eta = np.full(tuple(n + 2 * p3.nbl for n in p3.shape), 0.01, np.float32)
    outs = []
    for steps in (1, 2):
        s = p3.solver(fw)
        s.set_damping(eta)
        if steps == 2:
            s.set_time_blocking(2)
            s.set_model(p3.m32)
            s.set_damping(eta)
        outs.append(s.forward(p3.q32))
        s.sync()
        s.close()
    assert np.array_equal(outs[0], outs[1])


def test_two_step_full_grid_so4_first_steps(fw):
    """The 256^3 physical grid (336^3 computational) at space order 4 in the
    launch configuration the bench times, against the one-step loop."""
    from paper_1609_03361_gb300 import workloads as W
    w = W.config_3d(256, 12.5, 4, 12)
    w.dt = W.choose_dt(fw.fdw_dt_max(3, 12.5, 4, w.vmax))
    dev = torch.device("cuda", 0)
    m = torch.from_numpy(w.m.astype(np.float32)).to(dev)
    q = torch.from_numpy(w.wavelet().astype(np.float32)[:, None]).to(dev)
    outs = []
    for steps in (1, 2):
        s = fw.Solver(w.shape, w.spacing, w.space_order, w.nbl, w.dt, w.nt, w.vmax)
        if steps == 2:
            s.set_time_blocking(2)
        s.set_model(m)
        s.set_sources(w.src)
        s.set_receivers(w.rec)
        rec = s.forward(q).cpu().numpy()
        u = s.wavefield(0, like=q).cpu().numpy()
        s.sync()
        s.close()
        outs.append((rec, u))
    assert np.abs(outs[0][0]).max() > 0
    assert rel_l2(outs[1][0], outs[0][0]) < TOL_GPU
    assert rel_l2(outs[1][1], outs[0][1]) < TOL_GPU
