"""GPU parity of the initial decomposition (fgr_decompose, eq. 2.6 / 2.8) with
the FP64 oracle on the same seeded inputs: FP64 to 1e-12 and FP32 to 1e-5
(relative L2 over the amplitudes), d = 1..3, windows that span several hundred
points and are clipped by the grid edges, packets whose window misses the grid,
host and device buffers, and the 1-D workload's mesh at full size."""

import math

import numpy as np
import pytest

from oracle import decompose, fga
from workloads import config_workload, random_packets, WKB_TANH

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


CASES = {1: (3001, 700, 1 / 256), 2: ((70, 101), 300, 1 / 64), 3: ((20, 17, 23), 60, 1 / 16)}


def _case(d, seed):
    n, m, eps = CASES[d]
    ns = list(n) if isinstance(n, tuple) else [n]
    grid = dict(d=d, n=ns, lo=[-math.pi] * d, hi=[math.pi] * d)
    rng = np.random.default_rng(seed)
    u = rng.standard_normal(ns) + 1j * rng.standard_normal(ns)
    pk = random_packets(seed, d, m, q_range=(-3.6, 3.6), p_range=(-4, 4))
    pk["q"][:, :3] = 20.0   # windows off the grid
    return grid, eps, u, pk


def _run(fgr, grid, eps, u, pk, precision, on_device=True):
    import torch
    d = grid["d"]
    cdt = np.complex128 if precision == "fp64" else np.complex64
    with fgr.Context(d, grid, eps, _gpu.options(precision)) as ctx:
        if on_device:
            arrs = _gpu.to_device(pk)
            ut = torch.tensor(u.astype(cdt), device="cuda")
            fgr.fgr_decompose(ctx.handle, ut, fgr.make_packets(*arrs))
            torch.cuda.synchronize()
            return arrs[3].cpu().numpy(), arrs[2].cpu().numpy()
        host = {k: np.array(pk[k], dtype=np.float64, order="C", copy=True) for k in "qpsa"}
        host["s"][:] = 7.0
        fgr.fgr_decompose(ctx.handle, np.ascontiguousarray(u.astype(cdt)),
                          fgr.make_packets(host["q"], host["p"], host["s"], host["a"]))
        return host["a"], host["s"]


def _rel(got, ref):
    g, r = got[0] + 1j * got[1], ref[0] + 1j * ref[1]
    return float(np.linalg.norm(g - r) / np.linalg.norm(r))


@pytest.mark.parametrize("d", [1, 2, 3])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_decompose_matches_oracle(fgr, d, precision):
    grid, eps, u, pk = _case(d, 40 + d)
    R = 8 if precision == "fp64" else 6
    ref = decompose.decompose(u, grid, pk["q"], pk["p"], eps, R=R)
    a, s = _run(fgr, grid, eps, u, pk, precision)
    assert _rel(a, ref) <= (1e-12 if precision == "fp64" else 1e-5)
    assert np.all(a[:, :3] == 0) and np.all(s == 0)


def test_decompose_host_buffers_equal_device(fgr):
    grid, eps, u, pk = _case(1, 50)
    a_dev, _ = _run(fgr, grid, eps, u, pk, "fp64", on_device=True)
    a_host, s_host = _run(fgr, grid, eps, u, pk, "fp64", on_device=False)
    assert _rel(a_host, a_dev) <= 1e-15 and np.all(s_host == 0)


def test_decompose_workload_mesh_full_size(fgr):
    # the 1-D workload's 262144-packet mesh, u0 of its WKB data on its 32768-point
    # grid (FP32 context); the oracle evaluates a seeded sample of packets
    w = config_workload(2)
    grid, eps, pk = w["grid"], w["eps"], w["packets"]
    x = fga.grid_axis(grid, 0)
    u = WKB_TANH.u0(x[None, :], eps)
    a, _ = _run(fgr, grid, eps, u, pk, "fp32")
    rng = np.random.default_rng(9)
    sel = np.sort(rng.choice(pk["s"].size, 3000, replace=False))
    ref = decompose.decompose(u, grid, pk["q"][:, sel], pk["p"][:, sel], eps, R=6)
    assert _rel(a[:, sel], ref) <= 1e-5


def test_decompose_empty_and_invalid(fgr):
    import torch
    grid = dict(d=1, n=[64], lo=[-1.0], hi=[1.0])
    with fgr.Context(1, grid, 1 / 64, _gpu.options("fp64")) as ctx:
        empty = random_packets(1, 1, 0)
        u = torch.zeros(64, dtype=torch.complex128, device="cuda")
        fgr.fgr_decompose(ctx.handle, u, fgr.make_packets(*_gpu.to_device(empty)))
        bad = random_packets(2, 1, 4)
        bad["q"][0, 1] = np.nan
        with pytest.raises(fgr.FgrError):
            fgr.fgr_decompose(ctx.handle, np.zeros(64, np.complex128),
                              fgr.make_packets(*[np.ascontiguousarray(bad[k]) for k in "qpsa"]))


@pytest.mark.parametrize("d", [2, 3])
def test_decompose_grouped_packets_ragged_tail(fgr, d):
    # enough packets that every warp takes 32 of them (the last group ragged);
    # the oracle evaluates a seeded sample, the first and the last packets
    n = (70, 101) if d == 2 else (20, 17, 23)
    m = 200003
    grid = dict(d=d, n=list(n), lo=[-math.pi] * d, hi=[math.pi] * d)
    eps = 1 / 64
    rng = np.random.default_rng(70 + d)
    u = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    pk = random_packets(80 + d, d, m, q_range=(-3.6, 3.6), p_range=(-4, 4))
    for prec, tol in (("fp32", 1e-5), ("fp64", 1e-12)):
        a, s = _run(fgr, grid, eps, u, pk, prec)
        sel = np.unique(np.concatenate([rng.choice(m, 1500, replace=False), np.arange(40), np.arange(m - 40, m)]))
        ref = decompose.decompose(u, grid, pk["q"][:, sel], pk["p"][:, sel], eps, R=8 if prec == "fp64" else 6)
        assert _rel(a[:, sel], ref) <= tol, prec
        assert np.all(s == 0)


@pytest.mark.parametrize("shape", [(40, 300), (40, 600), (24, 1500), (12, 10, 400)])
def test_decompose_long_last_dimension(fgr, shape):
    # windows of about 70, 140 and 360 points along the last dimension: the
    # FP32 kernel keeps them in 2, 4 or 8 registers per lane, or reads the table
    d = len(shape)
    grid = dict(d=d, n=list(shape), lo=[-math.pi] * d, hi=[math.pi] * d)
    eps = 1 / 64
    rng = np.random.default_rng(sum(shape))
    u = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    pk = random_packets(len(shape) * 7 + shape[-1], d, 300, q_range=(-3.6, 3.6), p_range=(-4, 4))
    ref = decompose.decompose(u, grid, pk["q"], pk["p"], eps, R=6)
    a, _ = _run(fgr, grid, eps, u, pk, "fp32")
    assert _rel(a, ref) <= 1e-5
