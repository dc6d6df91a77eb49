"""Initial decomposition of a wave given on the grid (FP64).

Test infrastructure only (see the package docstring).

Eq. 2.6 and 2.8 (Sec. 2.1, Step 1 of Algorithms 1-3): the amplitude of the
packet at (q, p) is A(0, q, p) = 2^{d/2} u0hat(q, p) with

    u0hat(q, p) = int u0(y) exp(-i p.(y - q)/eps - |y - q|^2/(2 eps)) dy,

i.e. the L2 product of u0 with the conjugate of the packet G(y; q, p).  For a
wave known on the uniform grid x_m = lo + m h the integral is the rectangle
rule on the grid (exact to rounding for integrands that vanish at the ends),
restricted to the same box window |y_l - q_l| <= R sqrt(eps) as the
reconstruction (fga.window_bounds).  Packets are treated one by one, in index
order.
"""

from __future__ import annotations

import math

import numpy as np

from . import fga


def decompose(u, grid: dict, q, p, eps: float, R: float = 8.0) -> np.ndarray:
    """A(0, q_j, p_j) for every packet j; returns a (2, M) real array (re, im).

    u: complex array of shape n[0..d-1] (the wave on the grid); q, p: (d, M).
    """
    d = int(grid["d"])
    q = np.asarray(q, dtype=np.float64).reshape(d, -1)
    p = np.asarray(p, dtype=np.float64).reshape(d, -1)
    M = q.shape[1]
    u = np.asarray(u, dtype=np.complex128)
    axes = [fga.grid_axis(grid, l) for l in range(d)]
    h = [(float(grid["hi"][l]) - float(grid["lo"][l])) / int(grid["n"][l]) for l in range(d)]
    weight = 2.0 ** (d / 2.0) * math.prod(h)
    bounds = [fga.window_bounds(q[l], grid, l, eps, R) for l in range(d)]
    out = np.zeros((2, M))
    for j in range(M):
        if any(bounds[l][0][j] > bounds[l][1][j] for l in range(d)):
            continue
        sl = tuple(slice(bounds[l][0][j], bounds[l][1][j] + 1) for l in range(d))
        xs = np.meshgrid(*[axes[l][sl[l]] for l in range(d)], indexing="ij", sparse=True)
        phase = 0.0
        g2 = 0.0
        for l in range(d):
            dx = xs[l] - q[l, j]
            phase = phase + p[l, j] * dx
            g2 = g2 + dx * dx
        theta = -phase / eps
        kernel = np.exp(-g2 / (2.0 * eps)) * (np.cos(theta) + 1j * np.sin(theta))
        a = weight * np.sum(u[sl] * kernel)
        out[0, j], out[1, j] = a.real, a.imag
    return out
