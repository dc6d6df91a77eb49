"""Inputs of the multi-step examples of Sec. 4.4 (Examples 4 and 5).

Example 4: d = 1, eps = 2^-12 on [-2, 2), T = 0.8; Example 5: d = 2,
eps = 2^-6 on [-2, 2)^2, T = 1.6.  Both start from
u0 = (64/pi)^{d/4} exp(-32 |x|^2 + i (x_1 + ... + x_d) / eps), with the grid
step dx = eps, the mesh steps dq = sqrt(eps)/2, dp = pi sqrt(eps)/8, RK4 with
dt = 1e-4 and the Q2P2 neighbours.  V2 = |x|^2/2 (both examples) and, for
Example 4, V1 = 1 - cos(pi x).  (Example 5's V1 = 1 - exp(|x|^2) is not a
separable potential of the library.)  The T_evo x T_multi splits of Tables
17-22 are (8000 or 16000 steps) / T_multi for T_multi = 1, 2, 4, 8, 16, 32.

The fixed phase-space mesh of Algorithm 3 is, per dimension, the rectangle of
nodes (a dq, b dp) that holds every node where the wave's decomposition
exceeds 1e-9 of its largest value at any restart time (found once from the
closed-form harmonic solution; listed below), plus two nodes of margin.  A
dimension's list is ordered a-major (sorted by q); the d-dimensional mesh is
the tensor product of d such lists.
"""

from __future__ import annotations

import math

import numpy as np

EXAMPLES = {
    4: dict(d=1, eps=2.0 ** -12, T=0.8, dt=1e-4, q=(-0.8046875, 1.28125), p=(0.1169, 1.2889),
            potentials={"V1": dict(kind="cossum", c0=1.0, amp=-1.0, k=math.pi),
                        "V2": dict(kind="harmonic", omega=1.0)}),
    5: dict(d=2, eps=2.0 ** -6, T=1.6, dt=1e-4, q=(-1.125, 2.125), p=(-1.1655, 2.1234),
            potentials={"V2": dict(kind="harmonic", omega=1.0)}),
}
SPLITS = (1, 2, 4, 8, 16, 32)
BETA = 32.0  # u0 = n0 exp(-BETA |x|^2 + i p0.x / eps), p0 = (1, ..., 1)


def example_grid(ex: int) -> dict:
    e = EXAMPLES[ex]
    n = int(round(4.0 / e["eps"]))
    return dict(d=e["d"], n=[n] * e["d"], lo=[-2.0] * e["d"], hi=[2.0] * e["d"])


def example_axes_x(ex: int):
    g = example_grid(ex)
    return [g["lo"][l] + np.arange(g["n"][l]) * (g["hi"][l] - g["lo"][l]) / g["n"][l] for l in range(g["d"])]


def example_n0(ex: int) -> float:
    return (64.0 / math.pi) ** (EXAMPLES[ex]["d"] / 4.0)


def example_u0(ex: int) -> np.ndarray:
    e = EXAMPLES[ex]
    out = np.array(example_n0(ex), dtype=np.complex128)
    for x in example_axes_x(ex):
        f = np.exp(-BETA * x * x + 1j * x / e["eps"])
        out = np.multiply.outer(out, f) if out.ndim else out * f
    return out


def example_axis(ex: int):
    """(q, p) of one dimension's mesh list, a-major."""
    e = EXAMPLES[ex]
    dq = math.sqrt(e["eps"]) / 2
    dp = math.pi * math.sqrt(e["eps"]) / 8
    a = np.arange(math.floor(e["q"][0] / dq) - 2, math.ceil(e["q"][1] / dq) + 3)
    b = np.arange(math.floor(e["p"][0] / dp) - 2, math.ceil(e["p"][1] / dp) + 3)
    q = np.repeat(a * dq, b.size)
    p = np.tile(b * dp, a.size)
    return np.ascontiguousarray(q), np.ascontiguousarray(p)
