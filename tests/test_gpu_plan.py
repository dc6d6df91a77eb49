"""FGGC plans: a planned reconstruction equals fgr_reconstruct_fggc (same
arithmetic on a wider node box, so only the order of the atomic additions
differs) and the FP64 oracle; planned calls replay from a captured CUDA graph
with new packet values; packets that leave the planned box raise the overflow
flag; mismatched contexts and host buffers are refused."""

import math

import numpy as np
import pytest

from oracle import fggc, lsa
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


def _grid(d, n):
    ns = list(n) if isinstance(n, tuple) else [n] * d
    return dict(d=d, n=ns, lo=[-math.pi] * d, hi=[math.pi] * d)


CASES = [(1, 2048, 1 / 256, 900, "fp64"), (1, 4096, 1 / 512, 3000, "fp32"), (2, (64, 80), 1 / 64, 500, "fp32")]


@pytest.mark.parametrize("d,n,eps,m,prec", CASES)
def test_planned_equals_unplanned_and_oracle(fgr, d, n, eps, m, prec):
    import torch
    mesh = mesh_for(d, eps)
    pk = random_packets(20 + d, d, m, q_range=(-2.5, 2.5), p_range=(-2, 2), s_range=(-1, 1), mesh=mesh)
    grid = _grid(d, n)
    opt = _gpu.options(prec)
    dtype = torch.complex128 if prec == "fp64" else torch.complex64
    with fgr.Context(d, grid, eps, opt) as ctx:
        packets = fgr.make_packets(*_gpu.to_device(pk))
        ref = torch.zeros(tuple(grid["n"]), dtype=dtype, device="cuda")
        fgr.fgr_reconstruct_fggc(ctx.handle, packets, ref)
        plan = fgr.fgr_fggc_plan_create(ctx.handle, packets, 3)
        try:
            nodes, empty = fgr.fgr_fggc_plan_info(plan)
            assert nodes > 0 and not empty
            got = torch.full_like(ref, 5.0)
            fgr.fgr_reconstruct_fggc_planned(ctx.handle, plan, packets, got)
            torch.cuda.synchronize()
            assert not fgr.fgr_fggc_plan_overflow(plan)
        finally:
            fgr.fgr_fggc_plan_destroy(plan)
    g, r = got.cpu().numpy(), ref.cpu().numpy()
    assert _gpu.rel_l2(g, r) <= (1e-13 if prec == "fp64" else 1e-6)
    R = 8 if prec == "fp64" else 6
    oracle = fggc.reconstruct(pk, grid, eps, mesh.dq, mesh.dp, lsa.Strategy(nq=4, np_=2), R=R)
    tol = 4 * np.finfo(float).eps / math.sqrt(lsa.Strategy(nq=4, np_=2).pinv.singular_values[-1]) \
        if prec == "fp64" else 1e-5
    assert _gpu.rel_l2(g, oracle) <= max(tol, 1e-12)


def test_planned_calls_replay_from_a_cuda_graph(fgr):
    import torch
    eps = 1 / 512
    mesh = mesh_for(1, eps)
    reqs = []
    for r, (n, m) in enumerate(((2048, 1500), (4096, 3000), (1024, 700), (8192, 5000))):
        pk = random_packets(60 + r, 1, m, q_range=(-2.5, 2.5), p_range=(-2, 2), s_range=(-1, 1), mesh=mesh)
        ctx = fgr.Context(1, _grid(1, n), eps, _gpu.options("fp32"))
        arrs = _gpu.to_device(pk)
        packets = fgr.make_packets(*arrs)
        plan = fgr.fgr_fggc_plan_create(ctx.handle, packets, 2)
        u = torch.zeros(n, dtype=torch.complex64, device="cuda")
        reqs.append(dict(pk=pk, ctx=ctx, arrs=arrs, packets=packets, plan=plan, u=u))
    try:
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            for r in reqs:   # warm-up outside the capture
                fgr.fgr_reconstruct_fggc_planned(r["ctx"].handle, r["plan"], r["packets"], r["u"], s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            g.capture_begin()
            for r in reqs:
                fgr.fgr_reconstruct_fggc_planned(r["ctx"].handle, r["plan"], r["packets"], r["u"], s)
            g.capture_end()
        torch.cuda.synchronize()
        for it in range(3):
            scale = 0.5 + it
            for r in reqs:
                r["arrs"][3].copy_(torch.tensor(r["pk"]["a"] * scale, dtype=torch.float64, device="cuda"))
                r["u"].fill_(-3.0)
            g.replay()
            torch.cuda.synchronize()
            for r in reqs:
                ref = torch.zeros_like(r["u"])
                fgr.fgr_reconstruct_fggc(r["ctx"].handle, r["packets"], ref)
                torch.cuda.synchronize()
                assert _gpu.rel_l2(r["u"].cpu().numpy(), ref.cpu().numpy()) <= 1e-6
    finally:
        for r in reqs:
            fgr.fgr_fggc_plan_destroy(r["plan"])
            r["ctx"].close()


def test_packets_leaving_the_box_raise_the_overflow_flag(fgr):
    import torch
    eps = 1 / 256
    mesh = mesh_for(1, eps)
    pk = random_packets(70, 1, 800, q_range=(-1, 1), p_range=(-1, 1), mesh=mesh)
    with fgr.Context(1, _grid(1, 2048), eps, _gpu.options("fp32")) as ctx:
        arrs = _gpu.to_device(pk)
        packets = fgr.make_packets(*arrs)
        plan = fgr.fgr_fggc_plan_create(ctx.handle, packets, 2)
        try:
            u = torch.zeros(2048, dtype=torch.complex64, device="cuda")
            # one node step in P stays inside the margin of 2 nodes
            arrs[1].add_(mesh.dp)
            fgr.fgr_reconstruct_fggc_planned(ctx.handle, plan, packets, u)
            assert not fgr.fgr_fggc_plan_overflow(plan)
            # ten node steps do not
            arrs[1].add_(9 * mesh.dp)
            fgr.fgr_reconstruct_fggc_planned(ctx.handle, plan, packets, u)
            assert fgr.fgr_fggc_plan_overflow(plan)
        finally:
            fgr.fgr_fggc_plan_destroy(plan)


def test_plan_argument_checks(fgr):
    import torch
    pk = random_packets(71, 1, 100, q_range=(-1, 1), p_range=(-1, 1))
    with fgr.Context(1, _grid(1, 512), 1 / 64, _gpu.options("fp32")) as a, \
            fgr.Context(1, _grid(1, 1024), 1 / 64, _gpu.options("fp32")) as b:
        packets = fgr.make_packets(*_gpu.to_device(pk))
        with pytest.raises(fgr.FgrError):
            fgr.fgr_fggc_plan_create(a.handle, packets, -1)
        plan = fgr.fgr_fggc_plan_create(a.handle, packets, 1)
        try:
            u = torch.zeros(1024, dtype=torch.complex64, device="cuda")
            with pytest.raises(fgr.FgrError, match="another"):
                fgr.fgr_reconstruct_fggc_planned(b.handle, plan, packets, u)
            with pytest.raises(fgr.FgrError, match="device memory"):
                fgr.fgr_reconstruct_fggc_planned(a.handle, plan, packets, np.zeros(512, np.complex64))
            host = fgr.make_packets(*[np.ascontiguousarray(pk[k]) for k in "qpsa"])
            with pytest.raises(fgr.FgrError, match="device memory"):
                fgr.fgr_reconstruct_fggc_planned(a.handle, plan, host, u[:512])
        finally:
            fgr.fgr_fggc_plan_destroy(plan)
