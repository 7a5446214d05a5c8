"""Seeded synthetic inputs for the acoustic workloads.

This module makes inputs only: velocity models, source wavelets, source and
receiver coordinates and shot lists.  It holds none of the method's arithmetic
(no stencil weights, no stability limit, no damping, no interpolation), so the
CUDA library and the FP64 oracle can both be fed from it without sharing any
part of the computation.  Random numbers come from numpy's PCG64.

The paper uses no public dataset (arXiv 1609.03361, Sec. 5.4 models a
201x201x70 grid with a 10 Hz Ricker source); every workload here is synthetic.
Units: metres, milliseconds, km/s (= m/ms); squared slowness m = 1/v**2.
Axis order is (x, y, z) in 3D and (x, z) in 2D, z being depth and the
contiguous axis of every field.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "ricker", "choose_dt", "two_layer_model", "anomaly", "Workload",
    "config_2d_small", "config_3d", "batched_shots", "fwi_shots",
]


def ricker(f_hz: float, dt_ms: float, nt: int, t0_ms: float | None = None) -> np.ndarray:
    """Ricker wavelet sampled at t = n*dt (n = 0..nt-1), peak frequency f_hz,
    delay t0 = 1/f unless given, unit amplitude, float64."""
    f = f_hz * 1e-3  # cycles per ms
    t0 = 1.0 / f if t0_ms is None else t0_ms
    t = np.arange(nt, dtype=np.float64) * dt_ms - t0
    a = (math.pi * f * t) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


def choose_dt(dt_max: float, fraction: float = 0.9) -> float:
    """fraction * dt_max rounded down to 4 significant digits."""
    x = fraction * dt_max
    e = math.floor(math.log10(x)) - 3
    return math.floor(x / 10.0 ** e) * 10.0 ** e


def _smooth_noise(shape, sigma_cells: float, seed: int) -> np.ndarray:
    from scipy.ndimage import gaussian_filter
    g = np.random.Generator(np.random.PCG64(seed)).standard_normal(shape)
    g = gaussian_filter(g, sigma_cells, mode="nearest")
    return g / np.max(np.abs(g))


def two_layer_model(shape, v_top=1.5, v_bottom=2.5, perturb=0.05, sigma_cells=4.0,
                    seed=0) -> np.ndarray:
    """Velocity (km/s, float64, physical shape): v_top above half depth, v_bottom
    below, times (1 + perturb*g) with g a seeded N(0,1) field smoothed by a
    Gaussian of sigma_cells and normalised to max|g| = 1."""
    shape = tuple(int(s) for s in shape)
    nz = shape[-1]
    v = np.full(shape, v_top, dtype=np.float64)
    v[..., nz // 2:] = v_bottom
    if perturb:
        v *= 1.0 + perturb * _smooth_noise(shape, sigma_cells, seed)
    return v


def anomaly(v: np.ndarray, amplitude=0.05, sigma_cells=10.0) -> np.ndarray:
    """v times (1 + amplitude * Gaussian bump of sigma_cells at the grid centre)."""
    grids = np.meshgrid(*[np.arange(n, dtype=np.float64) - (n - 1) / 2.0 for n in v.shape],
                        indexing="ij")
    r2 = sum(g * g for g in grids)
    return v * (1.0 + amplitude * np.exp(-0.5 * r2 / sigma_cells ** 2))


@dataclass
class Workload:
    """One shot: physical grid, model, wavelet parameters and point sets."""
    name: str
    shape: tuple
    spacing: float
    space_order: int
    nbl: int
    nt: int
    f_hz: float
    velocity: np.ndarray               # physical shape, km/s
    src: np.ndarray                    # [nsrc][ndim] metres
    rec: np.ndarray                    # [nrec][ndim] metres
    dt: float | None = None            # ms; filled by the caller from the stability limit
    extra: dict = field(default_factory=dict)

    @property
    def ndim(self):
        return len(self.shape)

    @property
    def vmax(self):
        return float(self.velocity.max())

    @property
    def m(self):
        return 1.0 / self.velocity ** 2

    @property
    def comp_shape(self):
        return tuple(n + 2 * self.nbl for n in self.shape)

    def wavelet(self):
        assert self.dt is not None, "dt not chosen"
        return ricker(self.f_hz, self.dt, self.nt)


def config_2d_small(n=101, h=10.0, space_order=4, nt=500, nbl=40) -> Workload:
    """2D, n x n physical points at h, constant 1.5 km/s, 10 Hz Ricker at the
    centre, a line of receivers every h at 20 m depth (all on grid nodes)."""
    v = np.full((n, n), 1.5)
    L = (n - 1) * h
    src = np.array([[L / 2.0, L / 2.0]])
    xs = np.arange(n, dtype=np.float64) * h
    rec = np.stack([xs, np.full(n, 20.0)], axis=1)
    return Workload("2d-%d-so%d" % (n, space_order), (n, n), h, space_order, nbl, nt, 10.0,
                    v, src, rec)


def config_3d(n=256, h=12.5, space_order=8, nt=1000, nbl=40, f_hz=15.0, nrec_side=128,
              seed=0, velocity=None) -> Workload:
    """3D n^3 at h: two-layer 1.5/2.5 km/s model with a smoothed +-5% seeded
    perturbation; one off-grid source at the centre + (0.3h, 0.7h), 40 m deep;
    nrec_side^2 receivers spanning [0, (n-1)h]^2 at 20 m depth (off-grid)."""
    shape = (n, n, n)
    v = two_layer_model(shape, seed=seed) if velocity is None else velocity
    L = (n - 1) * h
    src = np.array([[L / 2.0 + 0.3 * h, L / 2.0 + 0.7 * h, 40.0]])
    g = np.linspace(0.0, L, nrec_side)
    gx, gy = np.meshgrid(g, g, indexing="ij")
    rec = np.stack([gx.ravel(), gy.ravel(), np.full(gx.size, 20.0)], axis=1)
    return Workload("3d-%d-so%d" % (n, space_order), shape, h, space_order, nbl, nt, f_hz,
                    v, src, rec)


def batched_shots(nshots=64, lo=96, hi=192, h=12.5, space_order=8, nt=800, nbl=40,
                  f_hz=15.0, nrec_side=64, seed=1) -> list:
    """Shots on cubes whose side is drawn uniformly from the integers [lo, hi]
    (seed), each with the two-layer recipe (seed 100+s), a source at the
    aperture centre 40 m deep and nrec_side^2 receivers at 20 m."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sides = rng.integers(lo, hi + 1, size=nshots)
    shots = []
    for s, n in enumerate(sides):
        n = int(n)
        shape = (n, n, n)
        v = two_layer_model(shape, seed=100 + s)
        L = (n - 1) * h
        src = np.array([[L / 2.0, L / 2.0, 40.0]])
        g = np.linspace(0.0, L, nrec_side)
        gx, gy = np.meshgrid(g, g, indexing="ij")
        rec = np.stack([gx.ravel(), gy.ravel(), np.full(gx.size, 20.0)], axis=1)
        shots.append(Workload("shot%d-%d" % (s, n), shape, h, space_order, nbl, nt, f_hz,
                              v, src, rec))
    return shots


def fwi_shots(n=256, h=12.5, space_order=8, nt=2000, nbl=40, f_hz=15.0, nshots=16,
              nrec_side=128, seed=0):
    """FWI survey: the config_3d model and receivers, sources on a sqrt(nshots)
    square grid over the surface at 40 m depth.  Returns (shots on the smooth
    model, velocity of the true model with a +5% Gaussian anomaly)."""
    base = config_3d(n, h, space_order, nt, nbl, f_hz, nrec_side, seed)
    k = int(round(math.sqrt(nshots)))
    L = (n - 1) * h
    pos = (np.arange(k) + 0.5) * L / k
    shots = []
    for i in range(k):
        for j in range(k):
            w = Workload("fwi%d" % (i * k + j), base.shape, h, space_order, nbl, nt, f_hz,
                         base.velocity, np.array([[pos[i], pos[j], 40.0]]), base.rec)
            shots.append(w)
    return shots, anomaly(base.velocity)


def diffusion_field(nx=1000, ny=1000, seed=0, noise=0.01):
    """Initial field of the 2D diffusion example (Sec. 4): 1 on a centred square
    of a quarter of each side, 0 elsewhere, plus seeded uniform noise of the
    given amplitude (so that no symmetry hides an index error)."""
    rng = np.random.default_rng(seed)
    u = noise * (2.0 * rng.random((nx, ny)) - 1.0)
    u[3 * nx // 8: 5 * nx // 8, 3 * ny // 8: 5 * ny // 8] += 1.0
    return u


def diffusion_dt(dx, dy, alpha=1.0):
    """Largest stable forward-Euler step of Sec. 4, Eq. 2."""
    return dx * dx * dy * dy / (2.0 * alpha * (dx * dx + dy * dy))
