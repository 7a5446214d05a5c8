"""2D diffusion of Sec. 4 through the C ABI against the FP64 oracle.

Tolerance: the scheme at or below the Eq. 2 limit is a convex combination of
a point and its four neighbours, so rounding errors do not grow: each float32
step adds at most a few units in the last place of max|u|.  The bound used is
(steps + 1) * 8 * 2^-24 * max|u0| on the largest pointwise difference, with
the oracle fed the same float32-rounded initial field.  Results for different
numbers of fused steps per pass must agree bit for bit (every point sees the
same operations in the same order)."""
import numpy as np
import pytest

import oracle
from paper_1609_03361_gb300 import workloads as W

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


def _bound(u0, steps):
    return (steps + 1) * 8 * 2.0 ** -24 * float(np.abs(u0).max())


def _gpu(fw, u0, dx, dy, alpha, dt, steps, spp):
    u = torch.from_numpy(u0.astype(np.float32)).cuda()
    fw.fdw_diffusion2d(u, None, dx, dy, alpha, dt, steps, spp)
    torch.cuda.synchronize()
    return u.cpu().numpy()


@pytest.mark.parametrize("shape", [(3, 3), (5, 130), (67, 45), (40, 257), (129, 500)])
@pytest.mark.parametrize("spp", [1, 2, 4, 8])
def test_diffusion_matches_oracle(fw, shape, spp):
    nx, ny = shape
    u0 = W.diffusion_field(nx, ny, seed=nx * 1000 + ny).astype(np.float32)
    dx, dy, alpha = 0.01, 0.013, 0.7
    dt = 0.9 * W.diffusion_dt(dx, dy, alpha)
    steps = 37
    got = _gpu(fw, u0, dx, dy, alpha, dt, steps, spp)
    ref = oracle.diffusion(u0.astype(np.float64), dx, dy, alpha, dt, steps)
    assert np.abs(got - ref).max() <= _bound(u0, steps)
    # boundary rows and columns keep their initial values exactly
    assert np.array_equal(got[0], u0[0]) and np.array_equal(got[-1], u0[-1])
    assert np.array_equal(got[:, 0], u0[:, 0]) and np.array_equal(got[:, -1], u0[:, -1])


def test_fused_passes_are_bitwise_equal(fw):
    u0 = W.diffusion_field(301, 389, seed=5).astype(np.float32)
    dx = dy = 0.001
    dt = W.diffusion_dt(dx, dy)
    outs = [_gpu(fw, u0, dx, dy, 1.0, dt, 53, spp) for spp in (1, 2, 4, 8)]
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])


def test_zero_steps_and_odd_step_counts(fw):
    u0 = W.diffusion_field(50, 70, seed=2).astype(np.float32)
    dx = dy = 0.02
    dt = W.diffusion_dt(dx, dy)
    assert np.array_equal(_gpu(fw, u0, dx, dy, 1.0, dt, 0, 4), u0)
    for steps in (1, 3, 9, 15):
        got = _gpu(fw, u0, dx, dy, 1.0, dt, steps, 8)
        ref = oracle.diffusion(u0.astype(np.float64), dx, dy, 1.0, dt, steps)
        assert np.abs(got - ref).max() <= _bound(u0, steps)


def test_paper_example_1000_squared_500_steps(fw):
    """The benchmark configuration of Sec. 4: a 1000 x 1000 grid of spacing
    0.001, alpha = 1, dt at the Eq. 2 limit (neighbour weights 1/4, no centre
    term), 500 time steps."""
    u0 = W.diffusion_field(1000, 1000, seed=0).astype(np.float32)
    dx = dy = 0.001
    dt = W.diffusion_dt(dx, dy)
    got = _gpu(fw, u0, dx, dy, 1.0, dt, 500, 0)
    ref = oracle.diffusion(u0.astype(np.float64), dx, dy, 1.0, dt, 500)
    assert np.abs(got - ref).max() <= _bound(u0, 500)


def test_argument_errors(fw):
    u = torch.zeros((20, 20), device="cuda")
    dt = W.diffusion_dt(0.1, 0.1)
    with pytest.raises(fw.FdwError) as e:
        fw.fdw_diffusion2d(u, None, 0.1, 0.1, 1.0, dt * 1.01, 5)
    assert e.value.status == 4  # FDW_ERR_CFL
    with pytest.raises(fw.FdwError):
        fw.fdw_diffusion2d(u, None, 0.1, 0.1, 1.0, dt, 5, steps_per_pass=3)
    with pytest.raises(fw.FdwError):
        fw.fdw_diffusion2d(u, u, 0.1, 0.1, 1.0, dt, 5)
    with pytest.raises(fw.FdwError):
        fw.fdw_diffusion2d(u.cpu(), None, 0.1, 0.1, 1.0, dt, 5)
    small = torch.zeros((2, 20), device="cuda")
    with pytest.raises(fw.FdwError):
        fw.fdw_diffusion2d(small, None, 0.1, 0.1, 1.0, dt, 5)
