"""GPU parity of the binned FGGC scatter (3-D, FP32) against the FP64
oracle's FGGC (Algorithm 2; eq. 2.24-2.25).

In 3-D the library bins packets by the anchor cell (a0, b0) of their outer
dimensions; for cells holding at least 8 packets a CTA lists which of the
packets' inner neighbours land on each cell of the inner plane and sums every
row of a cell in registers before adding it to the node array; cells with
fewer packets take the per-packet kernel (as every 1-D and 2-D problem does).
These packet sets put chosen numbers of packets into chosen outer cells, with
random inner positions, so that every path runs: small cells (per-packet),
cells of one and of several 256-packet items, inner spreads that fit one
window of target cells and ones that need several, and a momentum spread
wider than a window (per-contribution reductions inside the binned kernel).
The same clustered sets in 2-D check the per-packet kernel on them.  The
oracle evaluates at sampled grid points (1e-5, relative L2).
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
def test_clustered_2d(inner_q, inner_p):
    # the same cell sizes in 2-D, where the per-packet kernel runs
    eps = 1 / 64
    cells = [[(3, 5)], [(-4, 10)], [(0, 0)], [(7, -2)], [(-1, 1)]]
    pk, mesh = clustered(11, 2, eps, cells, [40, 300, 700, 10, 3], inner_q, inner_p)
    _check(pk, mesh, _grid((96, 80)), eps)


@pytest.mark.parametrize("inner_q,inner_p", [((-0.8, 0.8), (-0.5, 0.5)), ((-2.0, 2.0), (-2.0, 2.0))])
def test_binned_3d(inner_q, inner_p):
    # cells of 64 (one item), 300 and 600 (several items), 20 and 9 (small
    # items) and 5 (per-packet); the second spread needs several windows of
    # target cells
    eps = 1 / 64
    cells = [[(2, 3), (-1, 4)], [(0, 0), (0, 0)], [(-5, 2), (6, -3)], [(1, 1), (1, 2)], [(3, -2), (-2, 0)],
             [(-3, -1), (2, 2)]]
    pk, mesh = clustered(12, 3, eps, cells, [64, 300, 600, 20, 9, 5], inner_q, inner_p)
    _check(pk, mesh, _grid((40, 36, 44)), eps, npts=500)


def test_binned_wide_momentum_takes_reductions_per_contribution():
    # an inner momentum spread of more than 2048 p-nodes: the binned kernel
    # cannot hold one line of its target window and adds each contribution itself
    eps = 1 / 1024
    cells = [[(2, 3), (0, 1)], [(-6, 40), (3, -2)]]
    pk, mesh = clustered(13, 3, eps, cells, [100, 280], (-0.5, 0.5), (-15.0, 15.0))
    _check(pk, mesh, _grid((48, 40, 1024)), eps, npts=400)


def test_binned_matches_direct_sum_on_workload_like_cells():
    # packets of a separable flow share outer cells by the dozen (as in the
    # 3-D workload): a tensor product of outer cells with the same inner
    # packets; the binned result equals the oracle's FGGC and the direct sum's
    # within the least-squares error, and two calls agree to rounding
    eps = 1 / 256
    rng = np.random.default_rng(5)
    mesh = mesh_for(3, eps)
    qa = (np.arange(-1, 1) + 0.37) * mesh.dq
    pa = (np.arange(-2, 2) + 0.61) * mesh.dp
    Q0, P0, Q1, P1 = (x.ravel() for x in np.meshgrid(qa, pa, qa, pa, indexing="ij"))
    n_in = 48
    inner_q = rng.uniform(-0.4, 0.4, n_in)
    inner_p = rng.uniform(-0.3, 0.3, n_in)
    q = np.stack([np.repeat(Q0, n_in), np.repeat(Q1, n_in), np.tile(inner_q, Q0.size)])
    p = np.stack([np.repeat(P0, n_in), np.repeat(P1, n_in), np.tile(inner_p, Q0.size)])
    m = q.shape[1]
    pk = {"q": q, "p": p, "s": rng.uniform(-1, 1, m), "a": rng.standard_normal((2, m))}
    grid = _grid((40, 40, 64), lo=-1.0, hi=1.0)
    got = _check(pk, mesh, grid, eps, npts=500, seed=3)
    again = _gpu.reconstruct("fggc", pk, grid, eps, _gpu.options("fp32"))
    direct = _gpu.reconstruct("direct", pk, grid, eps, _gpu.options("fp32"))
    assert _gpu.rel_l2(again, got) <= 1e-6
    assert _gpu.rel_l2(got, direct) <= 1e-5


def test_rows_left_from_an_earlier_call_are_not_read():
    # The binned path clears only the rows of the node array that its packets
    # reach.  A first call with a wide packet set leaves non-zero rows in the
    # context's memory; a second call with packets in other outer cells must
    # still equal the oracle (unmarked rows are neither scanned nor contracted).
    import paper_2504_21785_gb300 as fgr
    eps = 1 / 64
    grid = _grid((40, 36, 44))
    wide, mesh = clustered(21, 3, eps, [[(c, 2 * c), (-c, c)] for c in range(-6, 7, 2)], [64] * 7,
                           (-2.0, 2.0), (-2.0, 2.0))
    other, _ = clustered(22, 3, eps, [[(1, -3), (2, 5)], [(-3, 0), (0, -2)]], [300, 40], (-1.0, 1.0), (-1.5, 1.5))
    opt = _gpu.options("fp32")
    with fgr.Context(3, grid, eps, opt) as ctx:
        _gpu.reconstruct("fggc", wide, grid, eps, opt, ctx=ctx)
        got = _gpu.reconstruct("fggc", other, grid, eps, opt, ctx=ctx)
    rng = np.random.default_rng(4)
    pts = np.stack([rng.integers(0, n, 500) for n in grid["n"]])
    ref = fggc.reconstruct(other, grid, eps, mesh.dq, mesh.dp, lsa.Strategy(nq=4, np_=2), R=6, points=pts)
    assert _gpu.rel_l2(got[tuple(pts)], ref) <= 1e-5
    alone = _gpu.reconstruct("fggc", other, grid, eps, opt)
    assert _gpu.rel_l2(got, alone) <= 1e-6
