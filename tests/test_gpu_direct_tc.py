"""GPU parity of the tensor-core direct sum (FP32, d = 2 and 3; the default
FP32 path for d >= 2) against the FP64 oracle's windowed direct sum (eq. 2.10), and against
the CUDA-core path (FGR_FLAG_DIRECT_FMA) on the same inputs.

Cases: ragged grids (no extent a multiple of the 128 x 64 or 8 x 16 x 64 super
tile)
with packets whose windows leave the grid and some zero amplitudes; a dense
case whose super tiles hold far more than 1024 records per work item, so that
the tensor-memory accumulator is read back several times per item; an empty
packet set.  Tolerance 1e-5 (relative L2), the FP32 bar."""

import math

import numpy as np
import pytest

from oracle import fga
from workloads import random_packets, mesh_for

from . import _gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fgr():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2504_21785_gb300 as pkg
    pkg.fgr.load()
    return pkg


def _grid(n0, n1):
    return dict(d=2, n=[n0, n1], lo=[-math.pi, -math.pi], hi=[math.pi, math.pi])


def test_tc_ragged_grid_matches_oracle(fgr):
    eps = 1 / 128
    mesh = mesh_for(2, eps)
    grid = _grid(301, 77)
    pk = random_packets(31, 2, 2500, q_range=(-3.8, 3.8), p_range=(-2.5, 2.5), s_range=(-3, 3), mesh=mesh,
                        on_node_fraction=0.1)
    pk["a"][:, ::17] = 0.0  # some zero amplitudes
    ref = fga.direct_sum(pk, grid, eps, mesh.dq, mesh.dp, R=6)
    got = _gpu.reconstruct("direct", pk, grid, eps, _gpu.options("fp32"))
    fma = _gpu.reconstruct("direct", pk, grid, eps, _gpu.options("fp32", flags=fgr.FGR_FLAG_DIRECT_FMA))
    assert got.dtype == np.complex64
    e_tc, e_fma = _gpu.rel_l2(got, ref), _gpu.rel_l2(fma, ref)
    print("ragged: tensor cores %.3e, CUDA cores %.3e" % (e_tc, e_fma))
    assert e_tc <= 1e-5
    assert e_fma <= 1e-5
    # every point off the packets' windows stays exactly zero on both paths
    assert np.all(got[ref == 0] == 0)


def test_tc_dense_items_read_back_several_times(fgr):
    # 60000 packets on a 160 x 96 grid with one work item per SM: every item
    # carries thousands of records, so the accumulator is read back (every
    # 1024 records) several times per item
    eps = 1 / 64
    mesh = mesh_for(2, eps)
    grid = _grid(160, 96)
    pk = random_packets(32, 2, 60000, q_range=(-3.0, 3.0), p_range=(-2.0, 2.0), s_range=(-3, 3), mesh=mesh)
    opt = _gpu.options("fp32")
    with fgr.Context(2, grid, eps, opt) as ctx:
        fgr.fgr_set_tuning(ctx.handle, 1, 16, 0)
        got = _gpu.reconstruct("direct", pk, grid, eps, opt, ctx=ctx)
    fma = _gpu.reconstruct("direct", pk, grid, eps, _gpu.options("fp32", flags=fgr.FGR_FLAG_DIRECT_FMA))
    rng = np.random.default_rng(3)
    pts = np.stack([rng.integers(0, 160, 400), rng.integers(0, 96, 400)])
    ref = fga.direct_sum(pk, grid, eps, mesh.dq, mesh.dp, R=6, points=pts)
    assert _gpu.rel_l2(got[tuple(pts)], ref) <= 1e-5
    assert _gpu.rel_l2(got, fma) <= 1e-5


def test_tc_empty_and_repeated_calls(fgr):
    eps = 1 / 64
    mesh = mesh_for(2, eps)
    grid = _grid(130, 33)
    empty = random_packets(33, 2, 0)
    got = _gpu.reconstruct("direct", empty, grid, eps, _gpu.options("fp32"))
    assert got.shape == (130, 33) and not np.any(got)
    pk = random_packets(34, 2, 700, q_range=(-3, 3), p_range=(-2, 2), mesh=mesh)
    ref = fga.direct_sum(pk, grid, eps, mesh.dq, mesh.dp, R=6)
    opt = _gpu.options("fp32")
    with fgr.Context(2, grid, eps, opt) as ctx:
        a = _gpu.reconstruct("direct", pk, grid, eps, opt, ctx=ctx)
        b = _gpu.reconstruct("direct", pk, grid, eps, opt, ctx=ctx)
    assert _gpu.rel_l2(a, ref) <= 1e-5
    assert _gpu.rel_l2(b, ref) <= 1e-5


def _grid3(n):
    return dict(d=3, n=list(n), lo=[-math.pi] * 3, hi=[math.pi] * 3)


def test_tc_3d_ragged_grid_matches_oracle(fgr):
    # 8 x 16 x 64 super tiles on a grid that none of the extents fills
    eps = 1 / 64
    mesh = mesh_for(3, eps)
    grid = _grid3((37, 29, 70))
    pk = random_packets(35, 3, 600, q_range=(-3.5, 3.5), p_range=(-1.5, 1.5), s_range=(-3, 3), mesh=mesh,
                        on_node_fraction=0.1)
    pk["a"][:, ::13] = 0.0
    ref = fga.direct_sum(pk, grid, eps, mesh.dq, mesh.dp, R=6)
    got = _gpu.reconstruct("direct", pk, grid, eps, _gpu.options("fp32"))
    fma = _gpu.reconstruct("direct", pk, grid, eps, _gpu.options("fp32", flags=fgr.FGR_FLAG_DIRECT_FMA))
    e_tc, e_fma = _gpu.rel_l2(got, ref), _gpu.rel_l2(fma, ref)
    print("3-D ragged: tensor cores %.3e, CUDA cores %.3e" % (e_tc, e_fma))
    assert e_tc <= 1e-5
    assert e_fma <= 1e-5
    assert np.all(got[ref == 0] == 0)


def test_tc_3d_dense_items(fgr):
    # many records per item: several accumulator phases and read-backs per item
    eps = 1 / 64
    mesh = mesh_for(3, eps)
    grid = _grid3((24, 40, 64))
    pk = random_packets(36, 3, 30000, q_range=(-1.5, 1.5), p_range=(-1.0, 1.0), s_range=(-3, 3), mesh=mesh)
    opt = _gpu.options("fp32")
    with fgr.Context(3, grid, eps, opt) as ctx:
        fgr.fgr_set_tuning(ctx.handle, 1, 16, 0)
        got = _gpu.reconstruct("direct", pk, grid, eps, opt, ctx=ctx)
    fma = _gpu.reconstruct("direct", pk, grid, eps, _gpu.options("fp32", flags=fgr.FGR_FLAG_DIRECT_FMA))
    rng = np.random.default_rng(4)
    pts = np.stack([rng.integers(0, n, 300) for n in (24, 40, 64)])
    ref = fga.direct_sum(pk, grid, eps, mesh.dq, mesh.dp, R=6, points=pts)
    assert _gpu.rel_l2(got[tuple(pts)], ref) <= 1e-5
    assert _gpu.rel_l2(got, fma) <= 1e-5
