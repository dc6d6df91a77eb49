"""The fixed mesh of the multi-step examples (workloads/examples.py) holds the
wave: at every restart time of the T_multi = 32 split, the decomposition of the
exact harmonic solution (eq. 2.8, oracle) outside the mesh's rectangle stays
below 1e-9 of its largest value.  Checked on a band of nodes just outside the
rectangle in each direction of phase space (Example 4, one dimension)."""

import math

import numpy as np

from oracle import decompose, exact
from workloads.examples import BETA, EXAMPLES, example_axes_x, example_axis, example_grid


def test_example4_mesh_holds_the_wave():
    ex = 4
    e = EXAMPLES[ex]
    eps = e["eps"]
    grid = example_grid(ex)
    x = example_axes_x(ex)[0]
    q, p = example_axis(ex)
    dq, dp = math.sqrt(eps) / 2, math.pi * math.sqrt(eps) / 8
    qs = np.unique(q)
    ps = np.unique(p)
    # the ring of nodes just outside the rectangle, three deep
    ring_q, ring_p = [], []
    for a in range(1, 4):
        for qq in (qs[0] - a * dq, qs[-1] + a * dq):
            for pp in np.concatenate([ps[::6], [ps[-1]]]):
                ring_q.append(qq)
                ring_p.append(pp)
        for pp in (ps[0] - a * dp, ps[-1] + a * dp):
            for qq in np.concatenate([qs[::6], [qs[-1]]]):
                ring_q.append(qq)
                ring_p.append(pp)
    ring = (np.array(ring_q)[None, :], np.array(ring_p)[None, :])
    for k in range(0, 33, 4):
        t = e["T"] * k / 32
        u = exact.harmonic_gaussian_1d(x, t, eps, BETA, 0.0, 1.0)
        out = decompose.decompose(u, grid, ring[0], ring[1], eps, R=8)
        # the largest amplitude: at the classical centre (q, p) of time t
        qc, pc = math.sin(t), math.cos(t)
        qn = np.round(qc / dq) * dq + dq * np.arange(-3, 4)
        pn = np.round(pc / dp) * dp + dp * np.arange(-3, 4)
        QN, PN = np.meshgrid(qn, pn, indexing="ij")
        core = decompose.decompose(u, grid, QN.reshape(1, -1), PN.reshape(1, -1), eps, R=8)
        amax = np.max(np.hypot(core[0], core[1]))
        assert np.max(np.hypot(out[0], out[1])) <= 1e-9 * amax, t


def test_example_inputs_follow_sec_4_4():
    from workloads.examples import EXAMPLES, SPLITS, example_u0
    e4, e5 = EXAMPLES[4], EXAMPLES[5]
    assert (e4["d"], e4["eps"], e4["T"]) == (1, 2.0 ** -12, 0.8)
    assert (e5["d"], e5["eps"], e5["T"]) == (2, 2.0 ** -6, 1.6)
    # 8000 and 16000 RK4 steps of 1e-4, split as in Tables 17-22
    assert round(e4["T"] / e4["dt"]) == 8000 and round(e5["T"] / e5["dt"]) == 16000
    assert SPLITS == (1, 2, 4, 8, 16, 32)
    for ex in (4, 5):
        e = EXAMPLES[ex]
        g = example_grid(ex)
        h = [(g["hi"][l] - g["lo"][l]) / g["n"][l] for l in range(g["d"])]
        assert all(abs(hl - e["eps"]) <= 1e-15 for hl in h)  # dx = eps on [-2, 2)
        u0 = example_u0(ex)
        # (64/pi)^{d/4} exp(-32|x|^2): unit L2 norm
        assert abs(math.sqrt(float(np.prod(h)) * np.sum(np.abs(u0) ** 2)) - 1) <= 1e-12
