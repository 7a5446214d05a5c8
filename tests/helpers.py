"""Test-side helpers written independently of both the oracle and the CUDA path.

- ``fornberg_weights``: Fornberg's recursive algorithm (B. Fornberg, "Generation
  of finite difference formulas on arbitrarily spaced grids", Math. Comp. 51,
  1988) in exact rational arithmetic, used to pin the oracle's closed-form
  stencil weights.
- ``np_laplacian``: a numpy zero-halo Laplacian used only for invariants
  (discrete energy) of fields the oracle produced.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np


def fornberg_weights(deriv: int, nodes, x0=0):
    """Weights w_i with sum_i w_i f(nodes[i]) ~ f^(deriv)(x0), exact Fractions."""
    nodes = [Fraction(x) for x in nodes]
    x0 = Fraction(x0)
    N = len(nodes)
    d = [[[Fraction(0)] * N for _ in range(N)] for _ in range(deriv + 1)]
    d[0][0][0] = Fraction(1)
    c1 = Fraction(1)
    for n in range(1, N):
        c2 = Fraction(1)
        for v in range(n):
            c3 = nodes[n] - nodes[v]
            c2 *= c3
            for k in range(min(n, deriv) + 1):
                lower = d[k - 1][n - 1][v] if k else Fraction(0)
                d[k][n][v] = ((nodes[n] - x0) * d[k][n - 1][v] - k * lower) / c3
        for k in range(min(n, deriv) + 1):
            lower = d[k - 1][n - 1][n - 1] if k else Fraction(0)
            d[k][n][n] = c1 / c2 * (k * lower - (nodes[n - 1] - x0) * d[k][n - 1][n - 1])
        c1 = c2
    return d[deriv][N - 1]


def central_second_derivative(p: int):
    """[c_0, c_1, ..., c_r] for the 2r+1 point central 2nd derivative (exact)."""
    r = p // 2
    nodes = [0]
    for j in range(1, r + 1):
        nodes += [j, -j]
    w = fornberg_weights(2, nodes)
    c = [w[0]]
    for j in range(1, r + 1):
        a, b = w[2 * j - 1], w[2 * j]
        assert a == b, "central weights must be symmetric"
        c.append(a)
    return c


def np_laplacian(u, spacing, p):
    """Zero-halo order-p Laplacian of a 2D/3D numpy field (weights from Fornberg)."""
    c = [float(x) for x in central_second_derivative(p)]
    r = p // 2
    out = np.zeros_like(u)
    for a in range(u.ndim):
        h2 = spacing[a] ** 2
        pad = [(0, 0)] * u.ndim
        pad[a] = (r, r)
        up = np.pad(u, pad)
        n = u.shape[a]
        acc = c[0] * u
        for k in range(1, r + 1):
            sl_p = [slice(None)] * u.ndim
            sl_m = [slice(None)] * u.ndim
            sl_p[a] = slice(r + k, r + k + n)
            sl_m[a] = slice(r - k, r - k + n)
            acc = acc + c[k] * (up[tuple(sl_p)] + up[tuple(sl_m)])
        out += acc / h2
    return out


def grid_coords(shape, spacing):
    """Coordinates [npts][ndim] of every node of a physical grid (row-major)."""
    axes = [np.arange(n, dtype=np.float64) * h for n, h in zip(shape, spacing)]
    mesh = np.meshgrid(*axes, indexing="ij")
    return np.stack([g.ravel() for g in mesh], axis=1)


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
