"""Batched direct sum (fgr_reconstruct_direct_batch): several requests with
their own grids, eps and packets in one persistent launch.  Each request must
give what a separate fgr_reconstruct_direct gives (same arithmetic; only the
order of the atomic additions differs) and match the FP64 oracle (eq. 2.10) at
the tolerances of the single-request parity tests; the call must also replay
correctly from a captured CUDA graph."""

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


# (d, eps, grid sizes, packet counts): ragged tails, one request with no
# packets and one whose packets all sit outside its grid
REQUESTS = {
    1: (1 / 256, [1000, 4097, 777, 2048, 300, 1500], [900, 2500, 0, 1200, 60, 700]),
    2: (1 / 64, [(70, 101), (64, 64), (33, 40), (96, 50)], [400, 900, 150, 0]),
}


def _make(fgr, d, precision, seed):
    import torch
    eps, sizes, counts = REQUESTS[d]
    mesh = mesh_for(d, eps)
    opt = _gpu.options(precision)
    reqs = []
    for r, (n, m) in enumerate(zip(sizes, counts)):
        ns = list(n) if isinstance(n, tuple) else [n]
        grid = dict(d=d, n=ns, lo=[-math.pi] * d, hi=[math.pi] * d)
        far = r == len(sizes) - 2 and d == 1   # packets far outside [-pi, pi)
        qr = (9.0, 12.0) if far else (-3.2, 3.2)
        pk = random_packets(seed + r, d, m, q_range=qr, p_range=(-3, 3), s_range=(-1, 1), mesh=mesh)
        ctx = fgr.Context(d, grid, eps, opt)
        arrs = _gpu.to_device(pk)
        dtype = torch.complex128 if precision == "fp64" else torch.complex64
        u = torch.full(tuple(ns), 7.0 + 1j, dtype=dtype, device="cuda")   # must be overwritten
        reqs.append(dict(pk=pk, grid=grid, ctx=ctx, arrs=arrs, packets=fgr.make_packets(*arrs), u=u))
    return eps, mesh, reqs


@pytest.mark.parametrize("d", [1, 2])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_matches_single_calls_and_oracle(fgr, d, precision):
    import torch
    eps, mesh, reqs = _make(fgr, d, precision, seed=10 * d)
    try:
        fgr.fgr_reconstruct_direct_batch([r["ctx"] for r in reqs], [r["packets"] for r in reqs],
                                         [r["u"] for r in reqs])
        torch.cuda.synchronize()
        R = 8 if precision == "fp64" else 6
        # FP32: the batch runs the CUDA-core kernel; a single 2-D call runs the
        # tensor-core one (3 x TF32), so the two agree to the FP32 tolerance
        tol_single = 1e-13 if precision == "fp64" else (1e-6 if d == 1 else 1e-5)
        tol_oracle = 1e-12 if precision == "fp64" else 1e-5
        for r in reqs:
            got = r["u"].cpu().numpy()
            single = torch.zeros_like(r["u"])
            fgr.fgr_reconstruct_direct(r["ctx"].handle, r["packets"], single)
            torch.cuda.synchronize()
            single = single.cpu().numpy()
            ref = fga.direct_sum(r["pk"], r["grid"], eps, mesh.dq, mesh.dp, R=R)
            if np.linalg.norm(ref) == 0:
                assert np.all(got == 0) and np.all(single == 0)
                continue
            assert _gpu.rel_l2(got, single) <= tol_single
            assert _gpu.rel_l2(got, ref) <= tol_oracle
    finally:
        for r in reqs:
            r["ctx"].close()


@pytest.mark.parametrize("d", [1, 2])
def test_batch_replays_from_a_cuda_graph(fgr, d):
    # d = 2 runs the balanced batch (items planned on the device)
    import torch
    eps, mesh, reqs = _make(fgr, d, "fp32", seed=40 + d)
    try:
        ctxs = [r["ctx"] for r in reqs]
        pks = [r["packets"] for r in reqs]
        us = [r["u"] for r in reqs]
        fgr.fgr_reconstruct_direct_batch(ctxs, pks, us)
        torch.cuda.synchronize()
        eager = [u.clone() for u in us]
        s = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            for u in us:
                u.fill_(3.0)
            g.capture_begin()
            fgr.fgr_reconstruct_direct_batch(ctxs, pks, us, stream=s)
            g.capture_end()
        torch.cuda.synchronize()
        for it in range(3):
            for u in us:
                u.fill_(-1.0)
            # new packet values in the same buffers: the replay must see them
            scale = 1.0 + it
            for r in reqs:
                r["arrs"][3].copy_(torch.tensor(r["pk"]["a"] * scale, dtype=torch.float64, device="cuda"))
            g.replay()
            torch.cuda.synchronize()
            for u, e in zip(us, eager):
                assert _gpu.rel_l2(u.cpu().numpy(), scale * e.cpu().numpy()) <= 1e-6
    finally:
        for r in reqs:
            r["ctx"].close()


def test_batch_rejects_mixed_or_invalid_requests(fgr):
    import torch
    grid1 = dict(d=1, n=[256], lo=[-math.pi], hi=[math.pi])
    grid2 = dict(d=2, n=[16, 16], lo=[-math.pi] * 2, hi=[math.pi] * 2)
    pk = random_packets(1, 1, 50, q_range=(-2, 2), p_range=(-2, 2))
    arrs = _gpu.to_device(pk)
    packets = fgr.make_packets(*arrs)
    with fgr.Context(1, grid1, 1 / 64, _gpu.options("fp64")) as a, \
            fgr.Context(1, grid1, 1 / 64, _gpu.options("fp32")) as b, \
            fgr.Context(2, grid2, 1 / 64, _gpu.options("fp64")) as c:
        u = torch.zeros(256, dtype=torch.complex128, device="cuda")
        u2 = torch.zeros(256, dtype=torch.complex128, device="cuda")
        with pytest.raises(fgr.FgrError, match="request 1"):
            fgr.fgr_reconstruct_direct_batch([a, b], [packets, packets], [u, u2])
        with pytest.raises(fgr.FgrError, match="request 1"):
            fgr.fgr_reconstruct_direct_batch([a, c], [packets, packets], [u, u2])
        with pytest.raises(fgr.FgrError, match="not device memory"):
            fgr.fgr_reconstruct_direct_batch([a], [packets], [np.zeros(256, np.complex128)])
        with pytest.raises(fgr.FgrError):
            fgr.fgr_reconstruct_direct_batch([a] * 65, [packets] * 65, [u] * 65)
