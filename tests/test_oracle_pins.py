"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test names what it pins: values the paper prints (tests/golden/, with
citations), Fornberg's recursion in exact arithmetic, convergence orders on
manufactured solutions, the 2D Green's function, the adjoint identity of
Sec. 5.3 (Eq. 4), finite-difference checks of the gradient, the energy
identity of the leapfrog scheme, and interpolation identities.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from helpers import central_second_derivative, grid_coords, np_laplacian, rel_l2
from paper_1609_03361_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


# --------------------------------------------------------------------------
# Stencil weights
# --------------------------------------------------------------------------

def test_so2_weights_match_paper():
    g = _golden("paper_so2_dx2.json")
    c = oracle.fd_weights(2)
    w = dict(zip(g["offsets"], g["weights_times_h2"]))
    assert c[0] == w[0] and c[1] == w[1] == w[-1]


@pytest.mark.parametrize("p", range(2, 17, 2))
def test_closed_form_weights_match_fornberg_recursion(p):
    exact = central_second_derivative(p)
    c = oracle.fd_weights(p)
    assert len(c) == p // 2 + 1
    for k, (got, ref) in enumerate(zip(c, exact)):
        assert abs(got - float(ref)) <= 1e-15 * max(1.0, abs(float(ref))), (p, k, got, ref)


def test_fornberg_rationals_spot_values():
    # Independent check of the test-side recursion itself on classic values.
    assert central_second_derivative(4) == [Fraction(-5, 2), Fraction(4, 3), Fraction(-1, 12)]
    c16 = central_second_derivative(16)
    assert c16[0] == Fraction(-1077749, 352800) and c16[8] == Fraction(-1, 411840)


def test_wave_so2_2d_expansion_matches_paper():
    """Sec. 3.1 prints the SO2 2D expansion of m*u.dt2 = u.laplace: 3-point dt2
    and a 5-point Laplacian (-4 centre, 1 per neighbour, over h^2).  An impulse
    injected at step 0 must spread after one more step exactly that way."""
    g = _golden("paper_wave_so2_2d.json")
    lw = g["laplace_weights_times_h2"]
    n, h, v, dt = 9, 10.0, 1.5, 1.0
    s = oracle.Setup((n, n), h, 2, 0, dt, 3)
    m = 1.0 / v ** 2
    M = np.full((n, n), m)
    eta = np.zeros((n, n))
    c = (n // 2) * h
    q = np.array([[1.0], [0.0], [0.0]])
    _, hist = oracle.forward(s, M, eta, [[c, c]], q, [[c, c]], history=True)
    a = dt * dt / m
    i = n // 2
    assert hist[1][i, i] == pytest.approx(a, rel=1e-15)
    assert np.count_nonzero(hist[1]) == 1
    u2 = hist[2]
    k = dt * dt / (m * h * h)
    # dt2 row (t+s: 1, t: -2, t-s: 1) with u^0 = 0 gives u^2 = 2 u^1 + (s^2/m) lap u^1.
    assert g["dt2_weights_times_s2"] == {"t-s": 1, "t": -2, "t+s": 1}
    assert u2[i, i] == pytest.approx(2 * a + k * lw["centre"] * a, rel=1e-14)
    for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
        assert u2[i + di, i + dj] == pytest.approx(k * 1 * a, rel=1e-14)
    assert lw["x-h"] == lw["x+h"] == lw["y-h"] == lw["y+h"] == 1
    assert u2[i + 1, i + 1] == 0.0 and u2[i + 2, i] == 0.0


# --------------------------------------------------------------------------
# Stability limit
# --------------------------------------------------------------------------

@pytest.mark.parametrize("p", [2, 4, 8, 16])
def test_stability_sum_is_symbol_maximum(p):
    """S equals max over wavenumbers of |symbol| of the 1-D stencil (Fornberg weights)."""
    c = [float(x) for x in central_second_derivative(p)]
    th = np.linspace(0, math.pi, 20001)
    sym = c[0] + 2 * sum(c[j] * np.cos(j * th) for j in range(1, len(c)))
    assert oracle.stability_sum(p) == pytest.approx(np.max(np.abs(sym)), rel=1e-12)


def test_stability_table_values():
    # dt_max * v / h for uniform grids (2D, 3D) at p = 4, 8, 16.
    table = {4: (0.6124, 0.5000), 8: (0.5546, 0.4529), 16: (0.5189, 0.4237)}
    for p, (d2, d3) in table.items():
        assert oracle.dt_max(2, 1.0, p, 1.0) == pytest.approx(d2, abs=1e-4)
        assert oracle.dt_max(3, 1.0, p, 1.0) == pytest.approx(d3, abs=1e-4)


@pytest.mark.parametrize("p", [4, 8])
def test_cfl_limit_separates_growth(p):
    """Just below dt_max the undamped scheme stays bounded; just above it a
    Nyquist mode grows without bound."""
    n, h, v = 24, 10.0, 2.0
    dtm = oracle.dt_max(2, h, p, v)
    rng = np.random.default_rng(3)
    q = np.zeros((400, 1))
    q[:5, 0] = rng.standard_normal(5)
    res = []
    for f in (0.995, 1.02):
        s = oracle.Setup((n, n), h, p, 0, f * dtm, 400)
        M = np.full((n, n), 1 / v ** 2)
        tr = oracle.forward(s, M, np.zeros((n, n)), [[115.0, 115.0]], q, [[115.0, 115.0]])
        res.append(np.abs(tr[-50:]).max() / np.abs(tr[:50]).max())
    assert res[0] < 10.0
    assert res[1] > 1e3


# --------------------------------------------------------------------------
# Convergence on manufactured solutions
# --------------------------------------------------------------------------

def _gaussian_problem(h, p, dt, nt, T, Tpp, L=1000.0, sig=60.0, v=1.5):
    """u = g(x) T(t), g a Gaussian centred in the domain (negligible at the
    edges), forced at every node by m g T'' - lap(g) T (continuum Laplacian)."""
    n = int(round(L / h)) + 1
    s = oracle.Setup((n, n), h, p, 0, dt, nt)
    X = grid_coords((n, n), (h, h))
    r2 = ((X - L / 2) ** 2).sum(1)
    g = np.exp(-r2 / sig ** 2)
    lap = g * (4 * r2 / sig ** 4 - 4 / sig ** 2)
    m = 1.0 / v ** 2
    t = np.arange(nt) * dt
    q = m * g[None, :] * Tpp(t)[:, None] - lap[None, :] * T(t)[:, None]
    _, fin = oracle.forward(s, np.full((n, n), m), np.zeros((n, n)), X, q, X[:1], final=True)
    exact = (g * T(t[-1])).reshape(n, n)
    return np.abs(fin - exact).max() / np.abs(exact).max()


@pytest.mark.parametrize("p", [2, 4, 8])
def test_spatial_convergence_order(p):
    """T(t) = t (t + dt) has an exact central second difference, so the only
    error is the order-p Laplacian: halving h must divide it by about 2^p."""
    dt, nt = 0.5, 41
    T = lambda t: t * (t + dt)
    Tpp = lambda t: 2.0 + 0.0 * t
    e = [_gaussian_problem(h, p, dt, nt, T, Tpp) for h in (20.0, 10.0, 5.0)]
    order = math.log2(e[1] / e[2])
    assert p - 0.3 < order < p + 0.5, (p, e)


def test_temporal_convergence_order():
    """With p = 16 the spatial error is negligible; halving dt must divide the
    error by about 4 (second order in time)."""
    w = 2 * math.pi * 0.01
    errs = []
    for dt in (2.0, 1.0, 0.5):
        T = lambda t, dt=dt: t * (t + dt) * np.cos(w * t)
        Tpp = lambda t, dt=dt: (2 * np.cos(w * t) - 2 * w * (2 * t + dt) * np.sin(w * t)
                                - w * w * t * (t + dt) * np.cos(w * t))
        nt = int(round(120.0 / dt)) + 1
        errs.append(_gaussian_problem(10.0, 16, dt, nt, T, Tpp))
    order = math.log2(errs[1] / errs[2])
    assert 1.9 < order < 2.1, errs


# --------------------------------------------------------------------------
# 2D Green's function
# --------------------------------------------------------------------------

def test_green_function_2d():
    """m u_tt - lap u = h^2 delta(x) q(t) in 2D has the solution
    u(r, t) = h^2/(2 pi) int_0^{acosh(t v / r)} q(t - (r/v) cosh th) dth
    (q = 0 for t < 0).  SO8 at 10 points per shortest wavelength, traces
    before any layer reflection can return: agreement within 1.5%."""
    from scipy.integrate import quad
    h, p, v, f, L, nbl = 5.0, 8, 1.5, 10.0, 1000.0, 40
    n = int(round(L / h)) + 1
    dt = W.choose_dt(oracle.dt_max(2, h, p, v))
    nt = int(560.0 / dt) + 1
    s = oracle.Setup((n, n), h, p, nbl, dt, nt)
    M = oracle.extend_model(s, np.full((n, n), 1 / v ** 2))
    eta = oracle.damping(s, v)
    c = L / 2
    rec = np.array([[c + 150.0, c], [c, c + 250.0], [c + 200.0, c + 200.0]])
    q = W.ricker(f, dt, nt)[:, None]
    tr = oracle.forward(s, M, eta, [[c, c]], q, rec)
    fr = f * 1e-3
    t0 = 1 / fr

    def rick(tt):
        a = (math.pi * fr * (tt - t0)) ** 2
        return (1 - 2 * a) * math.exp(-a)

    t = np.arange(nt) * dt
    for j, (x, z) in enumerate(rec):
        r = math.hypot(x - c, z - c)
        ref = np.zeros(nt)
        for i, ti in enumerate(t):
            if ti * v > r:
                val, _ = quad(lambda th: rick(ti - (r / v) * math.cosh(th)), 0,
                              math.acosh(ti * v / r), limit=200)
                ref[i] = h * h / (2 * math.pi) * val
        assert rel_l2(tr[:, j], ref) < 0.015, j


# --------------------------------------------------------------------------
# Adjoint identity (Sec. 5.3, Eq. 4)
# --------------------------------------------------------------------------

def _two_layer(shape):
    v = np.full(shape, 1.5)
    v[..., shape[-1] // 2:] = 2.5
    return v


@pytest.mark.parametrize("ndim,p", [(2, 2), (2, 4), (2, 8), (2, 12), (2, 16), (3, 4), (3, 8)])
def test_adjoint_dot_product(ndim, p):
    """<F q, d> = <q, F^T d> for the forward map q -> receiver traces, with
    damping, a two-layer model and off-grid points; FP64 to 1e-12 (the paper's
    Table 1 reaches ~6e-9 relative in 3D)."""
    shape = (30, 26) if ndim == 2 else (14, 12, 16)
    h = 10.0
    v = _two_layer(shape)
    dt = 0.8 * oracle.dt_max(ndim, h, p, v.max())
    nt = 120 if ndim == 2 else 60
    s = oracle.Setup(shape, h, p, 6, dt, nt)
    M = oracle.extend_model(s, 1 / v ** 2)
    eta = oracle.damping(s, v.max())
    rng = np.random.default_rng(7)
    top = np.array([(n - 1) * h for n in shape])
    src = rng.uniform(0, 1, (3, ndim)) * top
    rec = rng.uniform(0, 1, (5, ndim)) * top
    q = rng.standard_normal((nt, 3))
    d = rng.standard_normal((nt, 5))
    Fq = oracle.forward(s, M, eta, src, q, rec)
    FTd = oracle.adjoint(s, M, eta, rec, d, src)
    a, b = np.sum(Fq * d), np.sum(q * FTd)
    assert abs(a - b) <= 1e-12 * abs(a), (a, b)
    table = _golden("paper_adjoint_table.json")
    worst = max(abs(r[4] / r[2]) for r in table["rows"])
    assert abs(a - b) / abs(a) < worst


# --------------------------------------------------------------------------
# Gradient: finite differences and Taylor test
# --------------------------------------------------------------------------

def _grad_setup(ndim=2):
    shape = (24, 20) if ndim == 2 else (10, 10, 12)
    h, p = 10.0, 4
    v = _two_layer(shape)
    vmax = v.max() * 1.05
    dt = 0.8 * oracle.dt_max(ndim, h, p, vmax)
    nt = 150 if ndim == 2 else 70
    s = oracle.Setup(shape, h, p, 5, dt, nt)
    M = oracle.extend_model(s, 1 / v ** 2)
    eta = oracle.damping(s, vmax)
    top = np.array([(n - 1) * h for n in shape])
    src = np.array([top * 0.37])
    rng = np.random.default_rng(11)
    rec = rng.uniform(0, 1, (6, ndim)) * top
    q = W.ricker(25.0, dt, nt)[:, None]
    v_true = v * (1 + 0.05 * rng.standard_normal(shape))
    d = oracle.forward(s, oracle.extend_model(s, 1 / v_true ** 2), eta, src, q, rec)
    return s, M, eta, src, q, rec, d


def _J(s, M, eta, src, q, rec, d):
    r = oracle.forward(s, M, eta, src, q, rec) - d
    return 0.5 * np.sum(r * r), r


@pytest.mark.parametrize("ndim", [2, 3])
def test_gradient_matches_central_differences(ndim):
    s, M, eta, src, q, rec, d = _grad_setup(ndim)
    J0, r = _J(s, M, eta, src, q, rec, d)
    g = oracle.gradient(s, M, eta, src, q, rec, r)
    rng = np.random.default_rng(5)
    for _ in range(5):
        dm = rng.standard_normal(M.shape) * M.mean()
        eps = 1e-4
        Jp, _ = _J(s, M + eps * dm, eta, src, q, rec, d)
        Jm, _ = _J(s, M - eps * dm, eta, src, q, rec, d)
        fd = (Jp - Jm) / (2 * eps)
        an = np.sum(g * dm)
        assert abs(fd - an) <= 1e-6 * abs(fd), (fd, an)


def test_gradient_taylor_second_order():
    s, M, eta, src, q, rec, d = _grad_setup(2)
    J0, r = _J(s, M, eta, src, q, rec, d)
    g = oracle.gradient(s, M, eta, src, q, rec, r)
    dm = np.random.default_rng(9).standard_normal(M.shape) * M.mean()
    gd = np.sum(g * dm)
    errs = []
    for k in range(6):
        hh = 1e-2 / 2 ** k
        Jh, _ = _J(s, M + hh * dm, eta, src, q, rec, d)
        errs.append(abs(Jh - J0 - hh * gd))
    ratios = [errs[i] / errs[i + 1] for i in range(5)]
    assert all(3.6 < x < 4.4 for x in ratios), ratios


# --------------------------------------------------------------------------
# Interpolation identities (Sec. 5.2)
# --------------------------------------------------------------------------

def test_interp_on_grid_identity_and_partition_of_unity():
    s = oracle.Setup((11, 9, 7), (10.0, 12.5, 5.0), 4, 3, 1.0, 1)
    pts = grid_coords((11, 9, 7), (10.0, 12.5, 5.0))
    idx, w = oracle.interp(s, pts)
    assert np.allclose(w.sum(1), 1.0, rtol=0, atol=1e-15)
    n = s.comp_shape
    flat = []
    for x, y, z in pts:
        i, j, k = int(round(x / 10.0)), int(round(y / 12.5)), int(round(z / 5.0))
        flat.append(((i + 3) * n[1] + j + 3) * n[2] + k + 3)
    flat = np.array(flat)
    on = np.take_along_axis(idx, np.argmax(w, 1)[:, None], 1)[:, 0]
    assert np.array_equal(on, flat)
    assert np.allclose(w.max(1), 1.0, rtol=0, atol=1e-15)


def test_interp_reproduces_linear_fields():
    s = oracle.Setup((13, 17), (10.0, 7.0), 4, 4, 1.0, 1)
    rng = np.random.default_rng(2)
    top = np.array([120.0, 112.0])
    pts = rng.uniform(0, 1, (50, 2)) * top
    pts[0] = top  # last grid line in both axes
    pts[1] = [0.0, 0.0]
    idx, w = oracle.interp(s, pts)
    n = s.comp_shape
    ii, kk = np.meshgrid(np.arange(n[0]), np.arange(n[1]), indexing="ij")
    field = 3.0 + 0.5 * (ii - 4) * 10.0 - 0.25 * (kk - 4) * 7.0   # linear in metres
    vals = (w * field.ravel()[idx]).sum(1)
    exp = 3.0 + 0.5 * pts[:, 0] - 0.25 * pts[:, 1]
    assert np.allclose(vals, exp, rtol=0, atol=1e-12)


def test_interp_last_line_tie_break_and_domain():
    s = oracle.Setup((5, 5), 10.0, 2, 2, 1.0, 1)
    idx, w = oracle.interp(s, [[40.0, 40.0]])
    n = s.comp_shape
    # cell (3,3) in physical indices (= N-2), weight 1 on the far corner (+1,+1)
    assert idx[0, 3] == (3 + 1 + 2) * n[1] + (3 + 1 + 2) and w[0, 3] == 1.0
    for bad in ([-1e-9, 10.0], [10.0, 40.0000001]):
        with pytest.raises(oracle.OracleError):
            oracle.interp(s, [bad])


# --------------------------------------------------------------------------
# Energy identity and the absorbing layer
# --------------------------------------------------------------------------

def _energy(hist, M, h, p, dt):
    """E^{n+1/2} = 1/2 sum m ((u^{n+1}-u^n)/dt)^2 - 1/2 <u^{n+1}, L u^n>."""
    E = []
    for n in range(hist.shape[0] - 1):
        du = (hist[n + 1] - hist[n]) / dt
        E.append(0.5 * np.sum(M * du * du)
                 - 0.5 * np.sum(hist[n + 1] * np_laplacian(hist[n], (h,) * M.ndim, p)))
    return np.array(E)


@pytest.mark.parametrize("p", [4, 8])
def test_energy_conserved_without_damping_and_decays_with_it(p):
    n, h = 40, 10.0
    v = _two_layer((n, n))
    dt = 0.9 * oracle.dt_max(2, h, p, v.max())
    nt = 260
    q = np.zeros((nt, 1))
    q[:40, 0] = W.ricker(40.0, dt, 40)
    src = [[195.0, 140.0]]
    # no layer: energy is constant once the source has stopped
    s = oracle.Setup((n, n), h, p, 0, dt, nt)
    M = 1 / v ** 2
    _, hist = oracle.forward(s, M, np.zeros_like(M), src, q, src, history=True)
    E = _energy(hist, M, h, p, dt)[45:]
    assert np.ptp(E) <= 1e-10 * E.max()
    # with the absorbing layer: energy never increases after the source stops
    s2 = oracle.Setup((n, n), h, p, 10, dt, nt)
    M2 = oracle.extend_model(s2, M)
    eta = oracle.damping(s2, v.max())
    assert eta.min() == 0.0 and eta.max() > 0.0
    _, hist2 = oracle.forward(s2, M2, eta, src, q, src, history=True)
    E2 = _energy(hist2, M2, h, p, dt)[45:]
    assert np.all(np.diff(E2) <= 1e-12 * E2.max())
    assert E2[-1] < 0.2 * E2[0]


def test_damping_profile_shape():
    s = oracle.Setup((20, 16), (10.0, 5.0), 4, 8, 1.0, 1)
    eta = oracle.damping(s, 2.0)
    emax = [3 * math.log(1000) / (2 * 8 * h * 2.0) for h in (10.0, 5.0)]
    assert np.all(eta[8:28, 8:24] == 0.0)
    assert eta[0, 12] == pytest.approx(emax[0])           # d = nbl along x only
    assert eta[12, 0] == pytest.approx(emax[1])
    assert eta[0, 0] == pytest.approx(emax[0] + emax[1])
    assert eta[4, 12] == pytest.approx(emax[0] * 0.25)    # d = nbl/2: quadratic


def test_layer_reflection_below_one_percent():
    """Constant model: traces with the 40-point layer vs the same receivers in a
    domain large enough that nothing returns within the window."""
    h, p, v, f = 10.0, 8, 1.5, 10.0
    dt = W.choose_dt(oracle.dt_max(2, h, p, v))
    nt = int(900.0 / dt)
    q = W.ricker(f, dt, nt)[:, None]
    small = (61, 61)
    s = oracle.Setup(small, h, p, 40, dt, nt)
    M = oracle.extend_model(s, np.full(small, 1 / v ** 2))
    tr = oracle.forward(s, M, oracle.damping(s, v), [[300.0, 300.0]], q, [[300.0, 100.0]])
    big = (181, 181)   # same point 600 m further from every edge
    sb = oracle.Setup(big, h, p, 0, dt, nt)
    trb = oracle.forward(sb, np.full(big, 1 / v ** 2), np.zeros(big), [[900.0, 900.0]], q,
                         [[900.0, 700.0]])
    late = slice(int(420.0 / dt), nt)    # after the direct wavelet has passed
    assert np.abs(tr[late, 0] - trb[late, 0]).max() < 0.01 * np.abs(trb[:, 0]).max()


# --------------------------------------------------------------------------
# 2D diffusion worked example (Sec. 4, Listing 5)
# --------------------------------------------------------------------------

def test_diffusion_matches_generated_code_constants():
    g = _golden("paper_diffusion_generated.json")
    dx = dy = g["spacing"]
    alpha = 1.0
    dt = dx * dx * dy * dy / (2 * alpha * (dx * dx + dy * dy))      # Eq. 2
    u0 = np.random.default_rng(4).standard_normal((40, 30))
    u1 = oracle.diffusion(u0, dx, dy, alpha, dt, 1)
    w, wc = g["neighbour_weight"], g["centre_weight"]
    ref = u0.copy()
    ref[1:-1, 1:-1] = (w * (u0[2:, 1:-1] + u0[:-2, 1:-1] + u0[1:-1, 2:] + u0[1:-1, :-2])
                       + wc * u0[1:-1, 1:-1])
    assert np.allclose(u1, ref, rtol=0, atol=1e-12)
    assert g["interior_first"] == 1 and g["interior_last"] == g["nx"] - 2


# ---------------------------------------------------------------- model extension
# The paper gives only "40 points of damping layer" (Sec. 5.4); the reading is
# that the model is extended into the layer by repeating its edge values, and
# the gradient with respect to the physical model is the adjoint (transpose)
# of that extension.  The index maps below are spelled out by hand for
# nbl = 2: computational index i takes physical index clamp(i - 2), so a
# physical axis of 3 points becomes [0,0,0,1,2,2,2] and one of 4 points
# [0,0,0,1,2,3,3,3].  A clamp shifted by one changes these lists.
_MAP3 = [0, 0, 0, 1, 2, 2, 2]
_MAP4 = [0, 0, 0, 1, 2, 3, 3, 3]


def test_extend_model_2d_spelled_out():
    m = np.arange(1.0, 13.0).reshape(3, 4) ** 1.5   # non-constant, all values distinct
    s = oracle.Setup((3, 4), 10.0, 4, 2, 1.0, 2)
    M = oracle.extend_model(s, m)
    assert M.shape == (7, 8)
    for i in range(7):
        for k in range(8):
            assert M[i, k] == m[_MAP3[i], _MAP4[k]], (i, k)


def test_extend_model_3d_spelled_out():
    rng = np.random.default_rng(12)
    m = rng.uniform(0.1, 0.5, (3, 3, 4))
    s = oracle.Setup((3, 3, 4), 10.0, 4, 2, 1.0, 2)
    M = oracle.extend_model(s, m)
    assert M.shape == (7, 7, 8)
    for i in range(7):
        for j in range(7):
            for k in range(8):
                assert M[i, j, k] == m[_MAP3[i], _MAP3[j], _MAP4[k]], (i, j, k)


def test_fold_model_counts_repetitions():
    # folding a field of ones counts how many computational points repeat
    # each physical point: (nbl + 1) at an edge, 1 inside, per axis
    s = oracle.Setup((3, 4), 10.0, 4, 2, 1.0, 2)
    f = oracle.fold_model(s, np.ones((7, 8)))
    cx = [3, 1, 3]
    cz = [3, 1, 1, 3]
    assert np.array_equal(f, np.outer(cx, cz).astype(float))
    s3 = oracle.Setup((3, 3, 4), 10.0, 4, 2, 1.0, 2)
    f3 = oracle.fold_model(s3, np.ones((7, 7, 8)))
    assert np.array_equal(f3, np.einsum("i,j,k->ijk", cx, cx, cz).astype(float))


@pytest.mark.parametrize("shape,nbl", [((3, 4), 2), ((3, 3, 4), 2), ((5, 2, 6), 3), ((7, 9), 0)])
def test_fold_is_adjoint_of_extension(shape, nbl):
    rng = np.random.default_rng(len(shape) * 10 + nbl)
    s = oracle.Setup(shape, 10.0, 4, nbl, 1.0, 2)
    m = rng.standard_normal(shape)
    g = rng.standard_normal(s.comp_shape)
    a = float(np.sum(oracle.extend_model(s, m) * g))
    b = float(np.sum(m * oracle.fold_model(s, g)))
    assert abs(a - b) <= 1e-13 * max(abs(a), 1.0)
