"""Seeded test problems run through both the CUDA library and the FP64 oracle.

Only inputs are shared (the same float32 model, wavelets and coordinates);
each side computes everything else itself.
"""
from __future__ import annotations

import numpy as np

import oracle
from paper_1609_03361_gb300 import workloads as W


class Problem:
    def __init__(self, shape, h, p, nbl, nt, nsrc=1, nrec=6, seed=0, f_hz=25.0, vfac=0.9,
                 ongrid=False):
        self.shape = tuple(shape)
        self.ndim = len(shape)
        self.h = h
        self.p = p
        self.nbl = nbl
        self.nt = nt
        rng = np.random.default_rng(seed)
        self.v = W.two_layer_model(self.shape, seed=seed) if min(shape) > 4 else \
            np.full(self.shape, 1.5)
        self.vmax = float(self.v.max())
        dtm = oracle.dt_max(self.ndim, h, p, self.vmax)
        self.dt = W.choose_dt(dtm, vfac)
        self.m32 = (1.0 / self.v ** 2).astype(np.float32)
        top = np.array([(n - 1) * h for n in self.shape])
        if ongrid:
            idx = rng.integers(0, np.array(self.shape), size=(nsrc + nrec, self.ndim))
            pts = idx * h
        else:
            pts = rng.uniform(0.0, 1.0, (nsrc + nrec, self.ndim)) * top
        self.src = pts[:nsrc].astype(np.float64)
        self.rec = pts[nsrc:].astype(np.float64)
        q = np.stack([W.ricker(f_hz * (1 + 0.1 * i), self.dt, nt) for i in range(nsrc)], axis=1) \
            if nsrc else np.zeros((nt, 0))
        self.q32 = q.astype(np.float32)
        self.setup = oracle.Setup(self.shape, h, p, nbl, self.dt, nt)

    # ---- oracle side
    def oracle_model(self, m32=None):
        m = self.m32 if m32 is None else m32
        return oracle.extend_model(self.setup, m.astype(np.float64))

    def oracle_eta(self):
        return oracle.damping(self.setup, self.vmax)

    def oracle_forward(self, m32=None, final=False):
        return oracle.forward(self.setup, self.oracle_model(m32), self.oracle_eta(), self.src,
                              self.q32.astype(np.float64), self.rec, final=final)

    def oracle_adjoint(self, d):
        return oracle.adjoint(self.setup, self.oracle_model(), self.oracle_eta(), self.rec,
                              np.asarray(d, np.float64), self.src)

    def oracle_gradient(self, resid):
        return oracle.gradient(self.setup, self.oracle_model(), self.oracle_eta(), self.src,
                               self.q32.astype(np.float64), self.rec,
                               np.asarray(resid, np.float64))

    # ---- CUDA side
    def solver(self, fw, device=0, mtype="f32", tiling=None):
        s = fw.Solver(self.shape, self.h, self.p, self.nbl, self.dt, self.nt, self.vmax, device)
        if tiling is not None:
            s.set_tiling(*tiling)
        s.set_model(self.m32, "physical", mtype)
        s.set_sources(self.src)
        s.set_receivers(self.rec)
        return s


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def assert_close(got, want, tol=1e-4, what=""):
    """Parity of an FP32 result with the FP64 oracle: relative L2 error and the
    largest point-wise error relative to the largest reference value, both
    within tol (a local fault in one tile would hide in the norm alone)."""
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    scale = np.abs(want).max()
    assert scale > 0, f"{what}: the reference is zero"
    r = rel_l2(got, want)
    e = float(np.abs(got - want).max() / scale)
    assert r < tol and e <= tol, f"{what}: rel L2 {r:.3e}, max point-wise {e:.3e} (tol {tol:.0e})"
