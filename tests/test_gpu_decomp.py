"""Single-shot domain decomposition on one GPU: the grid cut into 2-4 x slabs
held by one process, ghost planes exchanged after every step.  Each slab runs
the whole-grid step's arithmetic on its planes, so the summed traces and the
slabs' own planes of the last wavefield must equal the whole-grid run bit for
bit; sources and receivers sit on and across slab boundaries.  The summed
traces and the wavefield reassembled from the slabs are also compared with the
FP64 oracle (relative L2 and point-wise, 1e-4)."""
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


def _whole(fw, pb):
    s = pb.solver(fw)
    rec = s.forward(torch.from_numpy(pb.q32).cuda())
    u = s.wavefield(0, like=rec)
    s.sync()
    s.close()
    return rec.cpu().numpy(), u.cpu().numpy()


def _boundary_points(pb, ranges, h):
    """Points at and across the slab boundaries (physical coordinates)."""
    pts = []
    for _, e in ranges[:-1]:
        xb = (e - pb.nbl) * h               # the boundary plane
        for dx in (-1.5 * h, -0.5 * h, 0.0, 0.3 * h, 1.0 * h):
            x = min(max(xb + dx, 0.0), (pb.shape[0] - 1) * h)
            pts.append([x] + [0.37 * (n - 1) * h for n in pb.shape[1:]])
    return np.array(pts)


@pytest.mark.parametrize("shape,p,parts", [((40, 36, 44), 8, 2), ((40, 36, 44), 8, 3),
                                           ((33, 20, 25), 4, 4), ((61, 57), 4, 2),
                                           ((30, 26, 28), 16, 2)])
def test_slabs_equal_whole_grid(fw, shape, p, parts):
    from paper_1609_03361_gb300.decomp import SlabForward, slab_ranges
    h = 10.0
    nbl = 6
    pb = Problem(shape, h, p, nbl, 60, nsrc=2, nrec=9, seed=parts * 7 + p)
    ranges = slab_ranges(shape[0] + 2 * nbl, parts, p // 2)
    extra = _boundary_points(pb, ranges, h)
    pb.rec = np.vstack([pb.rec, extra])
    pb.src = np.vstack([pb.src, extra[:2]])
    pb.q32 = np.concatenate([pb.q32, pb.q32[:, :2]], axis=1)
    rec_w, u_w = _whole(fw, pb)

    sf = SlabForward(pb.shape, h, p, nbl, pb.dt, pb.nt, pb.vmax, parts)
    assert sf.ranges == ranges
    sf.set_model(pb.m32)
    sf.set_sources(pb.src)
    sf.set_receivers(pb.rec)
    q = torch.from_numpy(pb.q32).cuda()
    recs = [torch.zeros((pb.nt, pb.rec.shape[0]), device="cuda") for _ in range(parts)]
    sf.forward([q] * parts, recs)
    torch.cuda.synchronize()
    total = sum(r.cpu().numpy().astype(np.float64) for r in recs)
    assert np.array_equal(total.astype(np.float32), rec_w)
    # every receiver recorded by exactly one slab
    nonzero = sum((np.abs(r.cpu().numpy()).sum(0) > 0).astype(int) for r in recs)
    assert np.all(nonzero[np.abs(rec_w).sum(0) > 0] == 1)
    r = p // 2
    u_slabs = np.empty_like(u_w)
    for s, (b, e) in zip(sf.slabs, ranges):
        u = s.wavefield(0, like=q).cpu().numpy()
        assert u.shape[0] == e - b + 2 * r
        assert np.array_equal(u[r:r + e - b], u_w[b:e])
        u_slabs[b:e] = u[r:r + e - b]
    sf.close()
    # the decomposed run against the FP64 oracle on the whole grid
    ref, uref = pb.oracle_forward(final=True)
    assert np.abs(ref).max() > 0
    for got, want in ((total, ref), (u_slabs, uref)):
        assert rel_l2(got, want) < 1e-4
        assert np.abs(got - want).max() <= 1e-4 * np.abs(want).max()


def test_slab_rejects_whole_loops(fw):
    pb = Problem((24, 20, 22), 10.0, 4, 4, 20, nsrc=1, nrec=3, seed=3)
    s = fw.Solver(pb.shape, pb.h, 4, 4, pb.dt, pb.nt, pb.vmax, slab=(0, 15))
    s.set_model(pb.m32)
    s.set_sources(pb.src)
    s.set_receivers(pb.rec)
    with pytest.raises(fw.FdwError):
        s.forward(pb.q32)
    with pytest.raises(fw.FdwError):
        fw.Batch([s])
    with pytest.raises(fw.FdwError):
        fw.Solver(pb.shape, pb.h, 4, 4, pb.dt, pb.nt, pb.vmax, slab=(10, 11))  # < r planes
    with pytest.raises(fw.FdwError):
        s.step(0, pb.q32, np.zeros((pb.nt, 3), np.float32))          # host arrays
    s.close()


def test_step_by_step_equals_forward(fw):
    pb = Problem((30, 28, 26), 10.0, 8, 5, 40, nsrc=1, nrec=7, seed=9)
    rec_w, u_w = _whole(fw, pb)
    s = pb.solver(fw)
    q = torch.from_numpy(pb.q32).cuda()
    rec = torch.zeros((pb.nt, 7), device="cuda")
    for n in range(pb.nt):
        s.step(n, q, rec)
    u = s.wavefield(0, like=q).cpu().numpy()
    s.sync()
    s.close()
    assert np.array_equal(rec.cpu().numpy(), rec_w)
    assert np.array_equal(u, u_w)
