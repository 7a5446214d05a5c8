"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerance: relative L2 <= 1e-4 for FP32 traces, wavefields and gradients
(the accuracy target for the FP32 path); the FP32 adjoint identity to 1e-5.
Sizes span several tiles in y and z with ragged tails and several x chunks.
"""
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


def _fwd(fw, pb, **kw):
    s = pb.solver(fw, **kw)
    rec = s.forward(pb.q32)
    u = s.wavefield(0)
    s.sync()
    s.close()
    return rec, u


@pytest.mark.parametrize("p", [2, 4, 6, 8, 10, 12, 14, 16])
def test_forward_3d_all_orders(fw, p):
    pb = Problem((37, 45, 29), 10.0, p, 8, 70, nsrc=2, nrec=9, seed=p)
    rec, u = _fwd(fw, pb)
    ref, uref = pb.oracle_forward(final=True)
    assert_close(rec, ref, TOL, "traces")
    assert_close(u, uref, TOL, "wavefield")


@pytest.mark.parametrize("p", [2, 4, 6, 8, 10, 12, 14, 16])
@pytest.mark.parametrize("tile", [7, 8, 9])
def test_forward_3d_tensor_memory_queue_all_orders(fw, p, tile):
    """Tiles 7, 8 and 9 keep the x queue in tensor memory: the same arithmetic
    as tiles 4, 6 and 4 (tile 9 forms two pair sums per instruction, each
    rounded as the scalar add), so bit for bit their results, and the
    oracle's to 1e-4."""
    pb = Problem((37, 45, 29), 10.0, p, 8, 70, nsrc=2, nrec=9, seed=p)
    rec, u = _fwd(fw, pb, tiling=(tile, 0, 0))
    ref, uref = pb.oracle_forward(final=True)
    assert_close(rec, ref, TOL, "traces")
    assert_close(u, uref, TOL, "wavefield")
    rec4, u4 = _fwd(fw, pb, tiling=({7: 4, 8: 6, 9: 4}[tile], 0, 0))
    assert np.array_equal(rec, rec4) and np.array_equal(u, u4)


@pytest.mark.parametrize("tiling", [(0, 0, 0), (1, 0, 0), (2, 0, 0), (4, 0, 0), (5, 0, 0),
                                    (0, 5, 0), (2, 3, 6), (1, 13, 0), (4, 64, 7), (0, 1, 0),
                                    (5, 7, 9), (6, 0, 0), (6, 9, 10), (7, 0, 0), (7, 1, 6),
                                    (7, 13, 9), (8, 0, 0), (8, 9, 10), (9, 0, 0), (9, 1, 2),
                                    (9, 13, 3), (9, 9, 7), (9, 64, 5)])
def test_forward_3d_tilings(fw, tiling):
    pb = Problem((40, 51, 35), 12.5, 8, 6, 60, nsrc=3, nrec=12, seed=11)
    rec, u = _fwd(fw, pb, tiling=tiling)
    ref, uref = pb.oracle_forward(final=True)
    assert_close(rec, ref, TOL, "traces")
    assert_close(u, uref, TOL, "wavefield")


def test_tilings_agree_bitwise(fw):
    """Every tiling computes each point with the same arithmetic."""
    pb = Problem((30, 33, 41), 10.0, 8, 5, 50, nsrc=2, nrec=8, seed=5)
    base_rec, base_u = _fwd(fw, pb, tiling=(0, 0, 0))
    for t in [(1, 0, 0), (2, 7, 0), (0, 2, 6), (1, 64, 9), (4, 3, 0), (5, 11, 7), (6, 13, 8),
              (7, 0, 0), (7, 5, 6), (8, 13, 8), (9, 0, 0), (9, 5, 2), (9, 13, 5)]:
        rec, u = _fwd(fw, pb, tiling=t)
        assert np.array_equal(rec, base_rec), t
        assert np.array_equal(u, base_u), t


@pytest.mark.parametrize("p", [2, 4, 8, 16])
def test_forward_2d(fw, p):
    pb = Problem((61, 57), 10.0, p, 20, 200, nsrc=1, nrec=11, seed=3)
    rec, u = _fwd(fw, pb)
    ref, uref = pb.oracle_forward(final=True)
    assert_close(rec, ref, TOL, "traces")
    assert_close(u, uref, TOL, "wavefield")


def test_forward_ongrid_and_edge_points(fw):
    pb = Problem((25, 22, 27), 10.0, 4, 4, 60, nsrc=2, nrec=5, seed=8, ongrid=True)
    top = np.array([(n - 1) * 10.0 for n in pb.shape])
    pb.rec = np.vstack([pb.rec, top, np.zeros(3), [top[0], 0.0, 105.0], [55.0, 210.0, 260.0]])
    rec, _ = _fwd(fw, pb)
    ref = pb.oracle_forward()
    assert rel_l2(rec, ref) < TOL


@pytest.mark.parametrize("mtype", ["f16", "bf16"])
def test_forward_low_precision_model(fw, mtype):
    """The model stored in 16 bits (as s = 1/m): parity with the oracle run on
    the same rounded model; the drift against the FP32 model is bounded.  The
    16-bit model tiles change the stage layout, so tile 9 (centre tiles after
    the model tile) must give tile 4's traces bit for bit."""
    pb = Problem((33, 30, 37), 12.5, 8, 6, 80, nsrc=1, nrec=8, seed=2)
    rec, _ = _fwd(fw, pb, mtype=mtype)
    rec9, _ = _fwd(fw, pb, mtype=mtype, tiling=(9, 0, 3))
    rec4, _ = _fwd(fw, pb, mtype=mtype, tiling=(4, 0, 0))
    assert np.array_equal(rec9, rec4)
    mt = torch.float16 if mtype == "f16" else torch.bfloat16
    # the library stores s = 1/m in 16 bits
    s_rounded = torch.from_numpy(1.0 / pb.m32).to(mt).to(torch.float64).numpy()
    m_rounded = 1.0 / s_rounded
    ref = pb.oracle_forward(m32=m_rounded)
    assert rel_l2(rec, ref) < TOL
    drift = rel_l2(rec, pb.oracle_forward())
    assert drift < (2e-2 if mtype == "f16" else 1e-1)


def test_device_and_host_arrays_agree(fw):
    pb = Problem((26, 29, 31), 10.0, 6, 5, 50, nsrc=1, nrec=7, seed=4)
    s = pb.solver(fw)
    rec_h = s.forward(pb.q32)
    rec_d = s.forward(torch.from_numpy(pb.q32).cuda()).cpu().numpy()
    s.sync()
    assert np.array_equal(rec_h, rec_d)
    s.close()


def test_degenerate_cases(fw):
    # no sources: everything stays zero; no receivers: the call still runs
    pb = Problem((20, 21, 22), 10.0, 4, 3, 30, nsrc=0, nrec=4, seed=1)
    rec, u = _fwd(fw, pb)
    assert np.count_nonzero(rec) == 0 and np.count_nonzero(u) == 0
    pb = Problem((20, 21, 22), 10.0, 4, 3, 30, nsrc=1, nrec=0, seed=1)
    s = pb.solver(fw)
    s.forward(pb.q32, rec=np.zeros((30, 0), np.float32))
    u = s.wavefield(0)
    s.sync()
    uref = pb.oracle_forward(final=True)[1]
    assert rel_l2(u, uref) < TOL
    # one time sample: u^0 = 0 is recorded
    pb = Problem((20, 21, 22), 10.0, 4, 3, 1, nsrc=1, nrec=3, seed=1)
    rec, _ = _fwd(fw, pb)
    assert rec.shape == (1, 3) and np.count_nonzero(rec) == 0


@pytest.mark.parametrize("ndim,p,tiling", [(3, 4, None), (3, 8, None), (3, 16, None), (2, 8, None),
                                           (3, 8, (7, 0, 0)), (3, 16, (8, 0, 0)),
                                           (3, 8, (9, 0, 0)), (3, 12, (9, 7, 3))])
def test_adjoint_parity_and_dot_test(fw, ndim, p, tiling):
    shape = (31, 27, 35) if ndim == 3 else (50, 45)
    pb = Problem(shape, 10.0, p, 6, 70, nsrc=2, nrec=7, seed=21 + p)
    rng = np.random.default_rng(p)
    d = rng.standard_normal((pb.nt, 7)).astype(np.float32)
    s = pb.solver(fw, tiling=tiling)
    qa = s.adjoint(d)
    Fq = s.forward(pb.q32)
    s.sync()
    s.close()
    ref = pb.oracle_adjoint(d)
    assert rel_l2(qa, ref) < TOL
    a = np.sum(Fq.astype(np.float64) * d)
    b = np.sum(pb.q32.astype(np.float64) * qa)
    assert abs(a - b) / abs(a) < 1e-5


@pytest.mark.parametrize("k,tiling", [(1, None), (4, None), (9, None), (70, None), (4, (7, 0, 0)),
                                      (9, (8, 11, 0)), (4, (9, 0, 0)), (9, (9, 11, 3))])
def test_gradient_fp32_checkpoints(fw, k, tiling):
    pb = Problem((29, 26, 31), 10.0, 8, 6, 70, nsrc=1, nrec=8, seed=31)
    rng = np.random.default_rng(3)
    resid = rng.standard_normal((pb.nt, 8)).astype(np.float32)
    s = pb.solver(fw, tiling=tiling)
    s.forward_ckpt(pb.q32, k, "f32")
    g = s.gradient(resid)
    s.sync()
    s.close()
    ref = pb.oracle_gradient(resid)
    assert rel_l2(g, ref) < TOL


# FP16 snapshots (11-bit significand, one float32 scale per snapshot) keep the
# gradient within 1e-3 of the FP64 oracle's exact gradient.  BF16 snapshots
# (8-bit significand: 2^-9 relative rounding of every stored value) do not
# reach 1e-3; their bound here is 5e-3.  k = 1 takes the separate max pass of
# the snapshot scale; k >= 2 folds the maximum into the two steps that
# produce each pair.
@pytest.mark.parametrize("stype,tol,k", [("f16", 1e-3, 10), ("bf16", 5e-3, 10), ("f16", 1e-3, 1),
                                         ("f16", 1e-3, 2), ("bf16", 5e-3, 3)])
def test_gradient_low_precision_snapshots(fw, stype, tol, k):
    pb = Problem((29, 26, 31), 10.0, 8, 6, 90, nsrc=1, nrec=8, seed=32)
    resid = pb.oracle_forward().astype(np.float32)
    s = pb.solver(fw)
    s.forward_ckpt(pb.q32, k, stype)
    g = s.gradient(resid)
    s.sync()
    s.close()
    ref = pb.oracle_gradient(resid)
    err = rel_l2(g, ref)
    assert err < tol, f"{stype} k={k}: gradient rel L2 {err:.3e} vs the FP64 oracle"


def test_gradient_residual_difference_and_physical_layout(fw):
    pb = Problem((24, 22, 26), 10.0, 4, 5, 60, nsrc=1, nrec=6, seed=41)
    rng = np.random.default_rng(5)
    a = rng.standard_normal((pb.nt, 6)).astype(np.float32)
    b = rng.standard_normal((pb.nt, 6)).astype(np.float32)
    s = pb.solver(fw)
    s.forward_ckpt(pb.q32, 6, "f32")
    g_phys = s.gradient(a, b, layout="physical")
    g_comp = s.gradient(a - b, None, layout="computational")
    s.sync()
    s.close()
    ref = pb.oracle_gradient(a.astype(np.float64) - b)
    assert rel_l2(g_comp, ref) < TOL
    # the physical-layout gradient is the oracle's computational gradient
    # folded onto the physical model (the adjoint of the model extension)
    import oracle
    fold = oracle.fold_model(pb.setup, ref)
    assert rel_l2(g_phys, fold) < TOL


def test_batched_forward_matches_single(fw):
    shapes = [(21, 24, 19), (30, 17, 26), (18, 18, 33)]
    pbs = [Problem(sh, 12.5, 8, 5, 60, nsrc=1, nrec=5, seed=50 + i) for i, sh in enumerate(shapes)]
    dt = min(pb.dt for pb in pbs)
    vmax = max(pb.vmax for pb in pbs)
    import oracle
    for pb in pbs:
        pb.dt = dt
        pb.vmax = vmax
        pb.setup = oracle.Setup(pb.shape, pb.h, pb.p, pb.nbl, dt, pb.nt)
    solvers = [pb.solver(fw) for pb in pbs]
    b = fw.Batch(solvers)
    recs = b.forward([pb.q32 for pb in pbs])
    for s in solvers:
        s.sync()
    for pb, rec in zip(pbs, recs):
        assert rel_l2(rec, pb.oracle_forward()) < TOL
        single = pb.solver(fw, tiling=(b.tiling()["tile"], b.tiling()["xchunk"], b.tiling()["stages"]))
        r1 = single.forward(pb.q32)
        single.sync()
        assert np.array_equal(r1, rec)
        single.close()
    b.close()
    for s in solvers:
        s.close()


def test_batched_gradient_matches_oracle(fw):
    shapes = [(21, 20, 19), (24, 17, 22)]
    pbs = [Problem(sh, 12.5, 4, 5, 50, nsrc=1, nrec=5, seed=60 + i) for i, sh in enumerate(shapes)]
    dt = min(pb.dt for pb in pbs)
    vmax = max(pb.vmax for pb in pbs)
    import oracle
    for pb in pbs:
        pb.dt = dt
        pb.vmax = vmax
        pb.setup = oracle.Setup(pb.shape, pb.h, pb.p, pb.nbl, dt, pb.nt)
    solvers = [pb.solver(fw) for pb in pbs]
    b = fw.Batch(solvers)
    rng = np.random.default_rng(9)
    res = [rng.standard_normal((pb.nt, 5)).astype(np.float32) for pb in pbs]
    b.forward_ckpt([pb.q32 for pb in pbs], 7, "f32")
    grads = b.gradient(res)
    for s in solvers:
        s.sync()
    for pb, g, r in zip(pbs, grads, res):
        assert rel_l2(g, pb.oracle_gradient(r)) < TOL
    b.close()
    for s in solvers:
        s.close()


def test_autotune_keeps_results(fw):
    pb = Problem((34, 30, 28), 10.0, 8, 6, 40, nsrc=1, nrec=6, seed=70)
    s = pb.solver(fw)
    s.autotune(3)
    t = s.tiling()
    assert t["tile"] in (0, 1, 2, 4, 5, 6, 7, 8) and t["stages"] >= 6
    rec = s.forward(pb.q32)
    s.sync()
    s.close()
    assert rel_l2(rec, pb.oracle_forward()) < TOL


def test_config_2d_101_so4_500_steps(fw):
    """The 2D workload exactly: 101^2 at 10 m, SO4, 40-point layer, 1.5 km/s,
    10 Hz Ricker at the centre, 101 on-grid receivers at 20 m depth, 500 steps."""
    import oracle
    from paper_1609_03361_gb300 import workloads as W
    w = W.config_2d_small()
    w.dt = W.choose_dt(oracle.dt_max(2, w.spacing, w.space_order, w.vmax))
    s = fw.Solver(w.shape, w.spacing, w.space_order, w.nbl, w.dt, w.nt, w.vmax)
    s.set_model(w.m.astype(np.float32))
    s.set_sources(w.src)
    s.set_receivers(w.rec)
    q = w.wavelet().astype(np.float32)[:, None]
    rec = s.forward(q)
    s.sync()
    s.close()
    st = oracle.Setup(w.shape, w.spacing, w.space_order, w.nbl, w.dt, w.nt)
    M = oracle.extend_model(st, w.m.astype(np.float32).astype(np.float64))
    ref = oracle.forward(st, M, oracle.damping(st, w.vmax), w.src, q.astype(np.float64), w.rec)
    assert rel_l2(rec, ref) < TOL


@pytest.fixture(scope="module")
def full_grid_case():
    """The 256^3 SO8 workload on its full 336^3 computational grid over its
    first 150 steps (the 15 Hz wavelet peaks at step 34; by step 150 the front
    has crossed x-chunk and tile boundaries and entered the damping layer
    above the source), with the oracle's traces and last field (the oracle
    needs about 0.1 s per step on this grid on 16 cores)."""
    import oracle
    from paper_1609_03361_gb300 import workloads as W
    nt = 150
    w = W.config_3d(256, 12.5, 8, nt)
    w.dt = W.choose_dt(oracle.dt_max(3, w.spacing, w.space_order, w.vmax))
    q = w.wavelet().astype(np.float32)[:, None]
    st = oracle.Setup(w.shape, w.spacing, w.space_order, w.nbl, w.dt, nt)
    M = oracle.extend_model(st, w.m.astype(np.float32).astype(np.float64))
    ref, uref = oracle.forward(st, M, oracle.damping(st, w.vmax), w.src, q.astype(np.float64),
                               w.rec, final=True)
    return w, q, ref, uref


# the autotuner's choice (as in the bench) and tilings the bench's tuner has
# picked on the GB300 (tile 4 with x chunks of 80 and 64, 7 stages; tile 9
# with x chunks of 128 or 192, 5 stages); the persist cases run every step
# in one persistent launch
@pytest.mark.parametrize("tiling,persist", [(None, False), ((4, 80, 7), False),
                                            ((4, 64, 7), False), ((7, 80, 7), False),
                                            ((4, 80, 7), True), ((9, 128, 5), True),
                                            ((9, 192, 5), True)])
def test_config_3d_256_so8_full_grid_first_steps(fw, full_grid_case, tiling, persist):
    w, q32, ref, uref = full_grid_case
    dev = torch.device("cuda", 0)
    s = fw.Solver(w.shape, w.spacing, w.space_order, w.nbl, w.dt, w.nt, w.vmax)
    if tiling is not None:
        s.set_tiling(*tiling)
    s.set_persistent(persist)
    s.set_model(torch.from_numpy(w.m.astype(np.float32)).to(dev))
    s.set_sources(w.src)
    s.set_receivers(w.rec)
    q = torch.from_numpy(q32).to(dev)
    if tiling is None:
        s.autotune(2)
    rec = s.forward(q).cpu().numpy()
    u = s.wavefield(0, like=q).cpu().numpy()
    s.sync()
    s.close()
    assert_close(rec, ref, TOL, "traces")
    assert_close(u, uref, TOL, "wavefield")
    # the front reached the layer above the source (depth index < nbl)
    assert np.abs(uref[:, :, : w.nbl]).max() > 1e-3 * np.abs(uref).max()


def test_batched_config_full_grids_first_steps(fw):
    """The 64-shot batched workload (cubes of 96^3..192^3 physical plus the
    layer, SO8) launched as one batch over its first 16 steps; the smallest
    and the largest shot are compared with the FP64 oracle on their full
    grids, and every shot's traces must be finite."""
    import oracle
    from paper_1609_03361_gb300 import workloads as W
    nt = 16
    shots = W.batched_shots(nshots=64, nt=nt)
    vmax = max(w.vmax for w in shots)
    dt = W.choose_dt(oracle.dt_max(3, shots[0].spacing, 8, vmax))
    dev = torch.device("cuda", 0)
    solvers, qs = [], []
    for w in shots:
        w.dt = dt
        s = fw.Solver(w.shape, w.spacing, 8, w.nbl, dt, nt, vmax)
        s.set_model(torch.from_numpy(w.m.astype(np.float32)).to(dev))
        s.set_sources(w.src)
        s.set_receivers(w.rec)
        solvers.append(s)
        qs.append(torch.from_numpy(w.wavelet().astype(np.float32)[:, None]).to(dev))
    b = fw.Batch(solvers)
    recs = [r.cpu().numpy() for r in b.forward(qs)]
    for s in solvers:
        s.sync()
    b.close()
    for s in solvers:
        s.close()
    assert all(np.isfinite(r).all() for r in recs)
    sides = [w.shape[0] for w in shots]
    for i in {int(np.argmin(sides)), int(np.argmax(sides))}:
        w = shots[i]
        st = oracle.Setup(w.shape, w.spacing, 8, w.nbl, dt, nt)
        M = oracle.extend_model(st, w.m.astype(np.float32).astype(np.float64))
        ref = oracle.forward(st, M, oracle.damping(st, vmax), w.src,
                             qs[i].cpu().numpy().astype(np.float64), w.rec)
        assert np.abs(ref).max() > 0
        assert rel_l2(recs[i], ref) < TOL


@pytest.mark.parametrize("shape,p,nbl", [((2, 2, 2), 16, 0), ((3, 2, 5), 8, 1), ((2, 3), 16, 0),
                                         ((5, 4, 3), 2, 0)])
def test_tiny_grids(fw, shape, p, nbl):
    """Grids smaller than the stencil and the tile: every neighbour beyond the
    grid is the zero halo."""
    pb = Problem(shape, 10.0, p, nbl, 12, nsrc=1, nrec=2, seed=len(shape) + p)
    rec, u = _fwd(fw, pb)
    ref, uref = pb.oracle_forward(final=True)
    assert rel_l2(rec, ref) < TOL
    assert rel_l2(u, uref) < TOL


def test_single_step(fw):
    pb = Problem((20, 18, 22), 10.0, 8, 4, 2, nsrc=2, nrec=5, seed=4)
    rec, u = _fwd(fw, pb)
    ref, uref = pb.oracle_forward(final=True)
    assert rel_l2(u, uref) < TOL
    assert np.allclose(rec, ref, rtol=1e-4, atol=1e-4 * np.abs(ref).max())


def test_config_3d_512_so16_full_grid_first_steps(fw):
    """The 512^3 SO16 workload on its full 592^3 computational grid (830 MB a
    field) over its first 40 steps, FP32 model, against the oracle: every
    trace and the last field, relative L2 and point-wise."""
    import oracle
    from paper_1609_03361_gb300 import workloads as W
    nt = 40
    w = W.config_3d(512, 12.5, 16, nt)
    w.dt = W.choose_dt(oracle.dt_max(3, w.spacing, 16, w.vmax))
    dev = torch.device("cuda", 0)
    s = fw.Solver(w.shape, w.spacing, 16, w.nbl, w.dt, nt, w.vmax)
    s.set_model(torch.from_numpy(w.m.astype(np.float32)).to(dev))
    s.set_sources(w.src)
    s.set_receivers(w.rec)
    q32 = w.wavelet().astype(np.float32)[:, None]
    rec = s.forward(torch.from_numpy(q32).to(dev)).cpu().numpy()
    u = s.wavefield(0, like=torch.from_numpy(q32).to(dev)).cpu().numpy()
    s.sync()
    s.close()
    st = oracle.Setup(w.shape, w.spacing, 16, w.nbl, w.dt, nt)
    M = oracle.extend_model(st, w.m.astype(np.float32).astype(np.float64))
    ref, uref = oracle.forward(st, M, oracle.damping(st, w.vmax), w.src, q32.astype(np.float64),
                               w.rec, final=True)
    assert_close(u, uref, TOL, "wavefield")
    assert_close(rec, ref, TOL, "traces")


@pytest.mark.parametrize("p,k,stype", [(4, 5, "f32"), (8, 10, "f32"), (8, 7, "f16"), (12, 4, "f32"),
                                       (16, 9, "f16")])
def test_gradient_tile9_equals_tile4(fw, p, k, stype):
    """Tile 9's gradient step stages the forward-field and accumulator tiles
    with the plane's other reads and forms the pair sums two at a time: the
    arithmetic of tile 4's gradient step, so its gradient bit for bit."""
    pb = Problem((29, 26, 31), 10.0, p, 6, 60, nsrc=1, nrec=8, seed=500 + p)
    resid = np.random.default_rng(p).standard_normal((pb.nt, 8)).astype(np.float32)
    out = []
    for tiling in [(4, 0, 0), (9, 0, 0), (9, 5, 2)]:
        s = pb.solver(fw, tiling=tiling)
        s.forward_ckpt(pb.q32, k, stype)
        out.append(s.gradient(resid))
        s.sync()
        s.close()
    assert np.array_equal(out[0], out[1]) and np.array_equal(out[0], out[2])
    if stype == "f32":
        assert rel_l2(out[1], pb.oracle_gradient(resid)) < TOL
