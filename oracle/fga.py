"""Frozen Gaussian packets and the windowed direct reconstruction (FP64).

Test infrastructure only (see the package docstring).

Notation (Sec. 2.1): a packet j carries a centre Q_j in R^d, a momentum P_j,
an action S_j and a complex amplitude A_j.  On the uniform grid
x_m = lo + m*h (h = (hi-lo)/n per dimension) the reconstruction is eq. 2.10:

    u(x) = (dq dp)^d / (2 pi eps)^{3d/2} * sum_j A_j exp(i/eps (S_j + P_j.(x-Q_j))
                                                       - |x-Q_j|^2 / (2 eps)).

Readings of the paper used here:
* Prefactor: eq. 2.9 / 2.10, i.e. (dq dp)^d / (2 pi eps)^{3d/2} with
  A(0) = 2^{d/2} u0hat (eq. 2.6).  The extra 2^{d/2} in eq. 2.1 would count that
  factor twice; Proposition 1 (tested) fixes the normalisation.
* (x - Q)^2 in eq. 2.10 is read as |x - Q|^2.
* The sum is truncated to a box window per dimension, |x_l - Q_l| <= R sqrt(eps),
  decided in FP64 as m_lo = ceil(((Q - R sqrt(eps)) - lo) / h),
  m_hi = floor(((Q + R sqrt(eps)) - lo) / h), clipped to [0, n).  The paper does
  not state a window; R = 8 for FP64 results and R = 6 for FP32 results.
  ``brute=True`` drops the window.
* Free space: grid points outside [lo, hi) do not exist; nothing wraps.
"""

from __future__ import annotations

import math

import numpy as np


def prefactor(d: int, eps: float, dq: float, dp: float) -> float:
    """(dq dp)^d / (2 pi eps)^{3d/2} of eq. 2.10."""
    return (dq * dp) ** d / (2.0 * math.pi * eps) ** (1.5 * d)


def grid_axis(grid: dict, l: int) -> np.ndarray:
    """x_m = lo + m*h for dimension l."""
    n = int(grid["n"][l])
    lo, hi = float(grid["lo"][l]), float(grid["hi"][l])
    h = (hi - lo) / n
    return lo + np.arange(n) * h


def gaussian_packet(x, Q, P, eps: float):
    """G(x; Q, P, eps) of eq. 2.16 at points x of shape (d, N)."""
    x = np.asarray(x, dtype=np.float64)
    Q = np.asarray(Q, dtype=np.float64).reshape(-1, 1)
    P = np.asarray(P, dtype=np.float64).reshape(-1, 1)
    dx = x - Q
    return np.exp(1j / eps * np.sum(P * dx, axis=0) - np.sum(dx * dx, axis=0) / (2.0 * eps))


def inner_product(Qbar, Pbar, Qtil, Ptil, eps: float):
    """<g, h> = int g h^dagger dx for g = G(.; Qbar, Pbar), h = G(.; Qtil, Ptil).

    Closed form of eq. 2.15.  Arrays broadcast; the last axis is the dimension.
    """
    Qbar, Pbar = np.asarray(Qbar, float), np.asarray(Pbar, float)
    Qtil, Ptil = np.asarray(Qtil, float), np.asarray(Ptil, float)
    d = Qbar.shape[-1]
    dQ = Qtil - Qbar
    dP = Ptil - Pbar
    expo = (-np.sum(dQ * dQ, axis=-1) / (4 * eps) - np.sum(dP * dP, axis=-1) / (4 * eps)
            + 1j / (2 * eps) * np.sum(dQ * (Ptil + Pbar), axis=-1))
    return (math.pi * eps) ** (d / 2.0) * np.exp(expo)


def window_bounds(Q, grid: dict, l: int, eps: float, R: float):
    """Inclusive window [m_lo, m_hi] of each centre Q (1-D array) in dimension l.

    Empty windows have m_lo > m_hi.
    """
    n = int(grid["n"][l])
    lo, hi = float(grid["lo"][l]), float(grid["hi"][l])
    h = (hi - lo) / n
    rs = R * math.sqrt(eps)
    Q = np.asarray(Q, dtype=np.float64)
    m_lo = np.ceil(((Q - rs) - lo) / h)
    m_hi = np.floor(((Q + rs) - lo) / h)
    m_lo = np.clip(m_lo, 0, n).astype(np.int64)
    m_hi = np.clip(m_hi, -1, n - 1).astype(np.int64)
    return m_lo, m_hi


def _terms(A, S, Q, P, xs, eps):
    """A_j exp(i/eps (S + P.(x-Q)) - |x-Q|^2/(2 eps)) for one packet on a point set.

    xs: list of d arrays broadcastable against each other (points).
    """
    phase = S
    g2 = 0.0
    for l, xl in enumerate(xs):
        dx = xl - Q[l]
        phase = phase + P[l] * dx
        g2 = g2 + dx * dx
    theta = phase / eps
    return A * np.exp(-g2 / (2.0 * eps)) * (np.cos(theta) + 1j * np.sin(theta))


def direct_sum(packets: dict, grid: dict, eps: float, dq: float, dp: float, R: float = 8.0,
               points=None, brute: bool = False):
    """Windowed direct sum of eq. 2.10 in FP64.

    packets: dict with q (d,M), p (d,M), s (M,), a (2,M).
    points: None for the full grid (returns an array of shape n[0..d-1]); or an
    integer array (d, K) of grid multi-indices (returns K values).
    Packets are summed in index order.
    """
    d = int(grid["d"])
    q, p, s = packets["q"], packets["p"], packets["s"]
    A = packets["a"][0] + 1j * packets["a"][1]
    M = s.shape[0]
    pref = prefactor(d, eps, dq, dp)
    axes = [grid_axis(grid, l) for l in range(d)]
    shape = tuple(int(n) for n in grid["n"][:d])
    bounds = [window_bounds(q[l], grid, l, eps, R) for l in range(d)]

    if points is None:
        u = np.zeros(shape, dtype=np.complex128)
        for j in range(M):
            if brute:
                sl = tuple(slice(0, shape[l]) for l in range(d))
            else:
                if any(bounds[l][0][j] > bounds[l][1][j] for l in range(d)):
                    continue
                sl = tuple(slice(bounds[l][0][j], bounds[l][1][j] + 1) for l in range(d))
            xs = np.meshgrid(*[axes[l][sl[l]] for l in range(d)], indexing="ij", sparse=True)
            u[sl] += _terms(A[j], s[j], q[:, j], p[:, j], xs, eps)
        return pref * u

    pts = np.asarray(points, dtype=np.int64).reshape(d, -1)
    K = pts.shape[1]
    out = np.zeros(K, dtype=np.complex128)
    # candidate search along dimension 0: m_lo and m_hi are non-decreasing in Q_0
    order = np.argsort(q[0], kind="stable")
    lo0 = bounds[0][0][order]
    hi0 = bounds[0][1][order]
    for i in range(K):
        idx = pts[:, i]
        if brute:
            sel = np.arange(M)
        else:
            first = np.searchsorted(hi0, idx[0], side="left")   # m_hi >= i0
            last = np.searchsorted(lo0, idx[0], side="right")   # m_lo <= i0
            cand = np.sort(order[first:last])
            ok = np.ones(cand.shape, dtype=bool)
            for l in range(d):
                ok &= (bounds[l][0][cand] <= idx[l]) & (idx[l] <= bounds[l][1][cand])
            sel = cand[ok]
        xs = [np.full(sel.shape, axes[l][idx[l]]) for l in range(d)]
        phase = s[sel].copy()
        g2 = np.zeros(sel.shape)
        for l in range(d):
            dx = xs[l] - q[l, sel]
            phase = phase + p[l, sel] * dx
            g2 = g2 + dx * dx
        theta = phase / eps
        terms = A[sel] * np.exp(-g2 / (2.0 * eps)) * (np.cos(theta) + 1j * np.sin(theta))
        out[i] = np.sum(terms)
    return pref * out


def direct_sum_tensor(axes, amps, actions, sel, grid: dict, eps: float, dq: float, dp: float, points,
                      R: float = 8.0, phase: complex = 1.0):
    """Eq. 2.10 at grid multi-indices ``points`` (d, K) for packets that form a
    selection of a tensor product of per-dimension lists.

    Packet j has the row-major multi-index (i_0, ..., i_{d-1}) = sel[j] and sits
    at Q_l = axes[l][0][i_l], P_l = axes[l][1][i_l] in dimension l, with
    amplitude phase * prod_l amps[l][i_l] and action sum_l actions[l][i_l].
    Its term A exp(i(S + P.(x - Q))/eps - |x - Q|^2/(2 eps)), box window
    included, is then a product over dimensions of
        f_l(i_l, x_l) = amps[l][i_l] exp(i (actions[l][i_l] + P_l (x_l - Q_l))/eps
                        - (x_l - Q_l)^2 / (2 eps)) [x_l in the window of Q_l],
    so u = pref phase sum over the selected multi-indices of the product of the
    d factors: a masked contraction over the list entries whose windows hold
    the point (the first dimension contracted once per distinct first index of
    the points).  Same sum as ``direct_sum`` on the expanded packets, in
    another order.
    """
    d = int(grid["d"])
    L = [int(np.asarray(q).size) for q, _ in axes]
    mask = np.zeros(int(np.prod(L)), dtype=np.float64)
    mask[np.asarray(sel, dtype=np.int64)] = 1.0
    mask = mask.reshape(L[0], -1)
    pref = prefactor(d, eps, dq, dp)
    xs = [grid_axis(grid, l) for l in range(d)]
    bounds = [window_bounds(axes[l][0], grid, l, eps, R) for l in range(d)]

    def factor(l, m):
        lo, hi = bounds[l]
        inwin = np.nonzero((lo <= m) & (m <= hi))[0]
        q = np.asarray(axes[l][0])[inwin]
        p = np.asarray(axes[l][1])[inwin]
        dx = xs[l][m] - q
        theta = (np.asarray(actions[l])[inwin] + p * dx) / eps
        f = np.asarray(amps[l])[inwin] * np.exp(-dx * dx / (2.0 * eps)) * (np.cos(theta) + 1j * np.sin(theta))
        return inwin, f

    pts = np.asarray(points, dtype=np.int64).reshape(d, -1)
    out = np.zeros(pts.shape[1], dtype=np.complex128)
    for m0 in np.unique(pts[0]):
        i0, f0 = factor(0, m0)
        # T[i_1, ..., i_{d-1}] = sum over i_0 of f_0(i_0) mask[i_0, ...]
        T = (f0.real @ mask[i0] + 1j * (f0.imag @ mask[i0])).reshape(L[1:]) if i0.size else None
        for k in np.nonzero(pts[0] == m0)[0]:
            if T is None:
                continue
            val = T
            for l in range(1, d):
                il, fl = factor(l, pts[l, k])
                val = np.tensordot(fl, val[il], axes=(0, 0)) if il.size else 0.0
            out[k] = val
    return pref * phase * out
