"""GPU parity of the binned FGGC scatter (d = 2, 3, FP32) against the FP64
oracle's FGGC (Algorithm 2; eq. 2.24-2.25).

The library bins packets by the anchor cell (a0, b0) of their outer
dimensions and, for cells holding at least 32 packets, accumulates their
contributions to each row of the node array in a private plane before adding
it to the node array; cells with fewer packets take the per-packet kernel.
These packet sets put chosen numbers of packets into chosen outer cells, with
random inner positions, so that every path runs: small cells (per-packet),
cells of one and of several 256-packet items, inner spreads that fit one plane
and ones that need several windows of it, and a momentum spread wider than a
plane (per-contribution reductions inside the binned kernel).  The oracle
evaluates at sampled grid points (1e-5, relative L2).
"""

import math

import numpy as np
import pytest

from oracle import fggc, lsa
from workloads import mesh_for

from . import _gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def clustered(seed, d, eps, cells, sizes, inner_q, inner_p):
    """sizes[i] packets whose outer (dimensions 0..d-2) Q and P lie in the
    anchor cell cells[i] = [(a, b) per outer dimension]; inner Q, P uniform."""
    mesh = mesh_for(d, eps)
    rng = np.random.default_rng(seed)
    qs, ps = [], []
    for cell, n in zip(cells, sizes):
        q = np.empty((d, n))
        p = np.empty((d, n))
        for l, (a, b) in enumerate(cell):
            q[l] = (a + rng.uniform(0.02, 0.98, n)) * mesh.dq
            p[l] = (b + rng.uniform(0.02, 0.98, n)) * mesh.dp
        q[d - 1] = rng.uniform(*inner_q, n)
        p[d - 1] = rng.uniform(*inner_p, n)
        qs.append(q)
        ps.append(p)
    q = np.concatenate(qs, axis=1)
    p = np.concatenate(ps, axis=1)
    m = q.shape[1]
    perm = rng.permutation(m)  # cells interleaved in packet order
    a = rng.standard_normal((2, m)) / math.sqrt(2)
    return {"q": np.ascontiguousarray(q[:, perm]), "p": np.ascontiguousarray(p[:, perm]),
            "s": rng.uniform(-3, 3, m), "a": np.ascontiguousarray(a)}, mesh


def _check(pk, mesh, grid, eps, npts=600, seed=0):
    rng = np.random.default_rng(seed)
    pts = np.stack([rng.integers(0, grid["n"][l], npts) for l in range(grid["d"])])
    ref = fggc.reconstruct(pk, grid, eps, mesh.dq, mesh.dp, lsa.Strategy(nq=4, np_=2), R=6, points=pts)
    got = _gpu.reconstruct("fggc", pk, grid, eps, _gpu.options("fp32"))
    err = _gpu.rel_l2(got[tuple(pts)], ref)
    print("binned FGGC d=%d, %d packets: rel L2 %.3e" % (grid["d"], pk["s"].size, err))
    assert err <= 1e-5
    return got


def _grid(ns, lo=-math.pi, hi=math.pi):
    return dict(d=len(ns), n=list(ns), lo=[lo] * len(ns), hi=[hi] * len(ns))


@pytest.mark.parametrize("inner_q,inner_p", [((-1.5, 1.5), (-1.0, 1.0)), ((-2.5, 2.5), (-3.0, 3.0))])
def test_binned_2d(inner_q, inner_p):
    # cells of 40 (one item), 300 and 700 (several items), 10 and 3 (per-packet);
    # the second spread needs several plane windows
    eps = 1 / 64
    cells = [[(3, 5)], [(-4, 10)], [(0, 0)], [(7, -2)], [(-1, 1)]]
    pk, mesh = clustered(11, 2, eps, cells, [40, 300, 700, 10, 3], inner_q, inner_p)
    _check(pk, mesh, _grid((96, 80)), eps)


@pytest.mark.parametrize("inner_q,inner_p", [((-0.8, 0.8), (-0.5, 0.5)), ((-2.0, 2.0), (-2.0, 2.0))])
def test_binned_3d(inner_q, inner_p):
    eps = 1 / 64
    cells = [[(2, 3), (-1, 4)], [(0, 0), (0, 0)], [(-5, 2), (6, -3)], [(1, 1), (1, 2)]]
    pk, mesh = clustered(12, 3, eps, cells, [64, 300, 600, 20], inner_q, inner_p)
    _check(pk, mesh, _grid((40, 36, 44)), eps, npts=500)


def test_binned_wide_momentum_takes_reductions_per_contribution():
    # an inner momentum spread of more than 4096 p-nodes: the binned kernel
    # cannot hold a line of its plane and adds each contribution itself
    eps = 1 / 1024
    cells = [[(2, 3)], [(-6, 40)]]
    pk, mesh = clustered(13, 2, eps, cells, [100, 280], (-1.0, 1.0), (-30.0, 30.0))
    _check(pk, mesh, _grid((300, 2048)), eps)


def test_binned_matches_per_packet_scatter_on_workload_like_cells():
    # packets of a separable flow share outer cells by the hundred (as in the
    # 2-D and 3-D workloads); the binned result equals the direct sum's within
    # the least-squares error, and two calls agree to rounding
    eps = 1 / 256
    rng = np.random.default_rng(5)
    mesh = mesh_for(2, eps)
    q1 = (np.arange(-8, 8) + 0.37) * mesh.dq
    p1 = (np.arange(-8, 8) + 0.61) * mesh.dp
    Q0, P0 = np.meshgrid(q1, p1, indexing="ij")
    inner_q = rng.uniform(-0.6, 0.6, 64)
    inner_p = rng.uniform(-0.5, 0.5, 64)
    q = np.stack([np.repeat(Q0.ravel(), 64), np.tile(inner_q, Q0.size)])
    p = np.stack([np.repeat(P0.ravel(), 64), np.tile(inner_p, P0.size)])
    m = q.shape[1]
    pk = {"q": q, "p": p, "s": rng.uniform(-1, 1, m), "a": rng.standard_normal((2, m))}
    grid = _grid((256, 256), lo=-1.5, hi=1.5)
    got = _check(pk, mesh, grid, eps, npts=800, seed=3)
    again = _gpu.reconstruct("fggc", pk, grid, eps, _gpu.options("fp32"))
    direct = _gpu.reconstruct("direct", pk, grid, eps, _gpu.options("fp32"))
    assert _gpu.rel_l2(again, got) <= 1e-6
    assert _gpu.rel_l2(got, direct) <= 1e-5
