"""Frozen Gaussian grid-point correction, Algorithm 2 Steps 3-4 (FP64).

Test infrastructure only (see the package docstring).

For each packet j the LSA coefficients c_j^(k) onto the neighbours
N(Q_j, P_j; k) (Def. 1, eq. 2.18) come from ``lsa.coefficients``.  Eq. 2.25
aggregates them onto phase-space grid nodes,

    W(q, p) = sum over (j, k) with N(Q_j,P_j;k) = (q, p) of A_j exp(i S_j/eps) c_j^(k),

(the paper calls this array A~(q, p); here it is W, since A~ also names the
Gram matrix of eq. 3.9), and eq. 2.24 sums the on-grid packets,

    u(x) = (dq dp)^d / (2 pi eps)^{3d/2} sum_{(q,p)} W(q, p) G(x; q, p),

which is eq. 2.10 applied to packets sitting on the nodes with S = 0 and
amplitude W; the same box window as the direct sum is used.
"""

from __future__ import annotations

import numpy as np

from . import fga, lsa


def aggregate(packets: dict, eps: float, dq: float, dp: float, strat: lsa.Strategy):
    """Eq. 2.25.  Returns integer node indices (d,K) for q (a) and p (b), and W (K,).

    Node (a, b) sits at (a dq, b dp).  Contributions are summed in the order
    (packet, neighbour).  Nodes are returned sorted lexicographically.
    """
    q = packets["q"]
    d, M = q.shape
    a0, b0, c = lsa.coefficients(packets, dq, dp, strat)
    A = packets["a"][0] + 1j * packets["a"][1]
    weight0 = A * np.exp(1j * packets["s"] / eps)            # A_j e^{i S_j / eps}
    n1 = strat.n1
    n = n1 ** d
    combos = np.array(np.unravel_index(np.arange(n), (n1,) * d))  # (d, n)
    # coefficient of neighbour (k_1..k_d): product over dimensions (tensor set)
    coef = np.ones((M, n), dtype=np.complex128)
    for l in range(d):
        coef = coef * c[l][:, combos[l]]
    contrib = weight0[:, None] * coef                          # (M, n)
    node_a = np.stack([a0[l][:, None] + strat.shifts[combos[l], 0].astype(np.int64)[None, :]
                       for l in range(d)])                     # (d, M, n)
    node_b = np.stack([b0[l][:, None] + strat.shifts[combos[l], 1].astype(np.int64)[None, :]
                       for l in range(d)])
    keys = np.concatenate([node_a.reshape(d, -1), node_b.reshape(d, -1)], axis=0)  # (2d, M*n)
    if keys.shape[1] == 0:
        return np.zeros((d, 0), np.int64), np.zeros((d, 0), np.int64), np.zeros(0, np.complex128)
    uniq, inv = np.unique(keys, axis=1, return_inverse=True)
    W = np.zeros(uniq.shape[1], dtype=np.complex128)
    np.add.at(W, inv.reshape(-1), contrib.reshape(-1))
    return uniq[:d], uniq[d:], W


def on_grid_packets(node_a, node_b, W, dq: float, dp: float) -> dict:
    """The aggregated nodes as a packet set (Q = a dq, P = b dp, S = 0, A = W)."""
    return {"q": node_a.astype(np.float64) * dq, "p": node_b.astype(np.float64) * dp,
            "s": np.zeros(W.shape[0]), "a": np.stack([W.real, W.imag])}


def reconstruct(packets: dict, grid: dict, eps: float, dq: float, dp: float,
                strat: lsa.Strategy, R: float = 8.0, points=None):
    """u_fggc on the grid (or at grid multi-indices ``points``), eq. 2.24-2.25."""
    node_a, node_b, W = aggregate(packets, eps, dq, dp, strat)
    cells = on_grid_packets(node_a, node_b, W, dq, dp)
    return fga.direct_sum(cells, grid, eps, dq, dp, R=R, points=points)


def multistep(u0, grid: dict, mesh: dict, flow: dict, eps: float, dq: float, dp: float,
              strat: lsa.Strategy, steps: int, R: float = 8.0):
    """Algorithm 3 (multi-step FGGC) with a fixed phase-space mesh.

    mesh: packets at the mesh positions (q, p) onto which every step decomposes
    the current wave (Step 1, eq. 2.8); flow: the same packets propagated over
    one step T_evo from unit amplitude (Step 2, the map learned once: Q, P, S
    and the amplitude factor, since eq. 2.6 is linear in A).  Each step
    decomposes u, multiplies the amplitudes by the factors and reconstructs by
    FGGC (Step 3); returns u after `steps` steps.
    """
    from . import decompose as dec
    factor = flow["a"][0] + 1j * flow["a"][1]
    u = np.asarray(u0, dtype=np.complex128)
    for _ in range(steps):
        a0 = dec.decompose(u, grid, mesh["q"], mesh["p"], eps, R=R)
        a = (a0[0] + 1j * a0[1]) * factor
        packets = {"q": flow["q"], "p": flow["p"], "s": flow["s"], "a": np.stack([a.real, a.imag])}
        u = reconstruct(packets, grid, eps, dq, dp, strat, R=R)
    return u
