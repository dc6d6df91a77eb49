"""fgr_reconstruct_fggc_batch: many planned FGGC reconstructions, one launch
per stage for the requests of each dimension.  Each request's output equals
its own planned call (same arithmetic; only the order of the atomic
additions differs) and the FP64 oracle's FGGC (Algorithm 2); a batch of
mixed dimensions, more than one launch's worth of requests, empty requests
and packets that leave their planned box are covered; the batch replays
from a captured CUDA graph with new packet values; bad arguments are refused."""

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
    ns = list(n) if isinstance(n, (tuple, list)) else [n] * d
    return dict(d=d, n=ns, lo=[-math.pi] * d, hi=[math.pi] * d)


def _requests(fgr, prec, count, seed):
    import torch
    rng = np.random.default_rng(seed)
    reqs = []
    for r in range(count):
        d = [1, 1, 2, 1, 3, 2][r % 6]
        eps = float(2.0 ** -rng.uniform(6, 9)) if d < 3 else 1 / 64
        mesh = mesh_for(d, eps)
        m = int(rng.integers(200, 3000)) if d == 1 else (int(rng.integers(100, 600)) if d == 2 else 150)
        n = int(2 ** rng.integers(9, 12)) if d == 1 else ((48, 56) if d == 2 else (20, 24, 28))
        lim = (2.2, 2.0) if d < 3 else (0.3, 0.3)   # 3-D: a compact node box
        pk = random_packets(300 + r, d, m, q_range=(-lim[0], lim[0]), p_range=(-lim[1], lim[1]), s_range=(-1, 1),
                            mesh=mesh)
        grid = _grid(d, n)
        ctx = fgr.Context(d, grid, eps, _gpu.options(prec))
        arrs = _gpu.to_device(pk)
        packets = fgr.make_packets(*arrs)
        plan = fgr.fgr_fggc_plan_create(ctx.handle, packets, 2)
        dt = torch.complex128 if prec == "fp64" else torch.complex64
        u = torch.full(tuple(grid["n"]), 7.0, dtype=dt, device="cuda")
        reqs.append(dict(pk=pk, grid=grid, eps=eps, mesh=mesh, ctx=ctx, arrs=arrs, packets=packets, plan=plan, u=u))
    return reqs


def _close(fgr, reqs):
    for r in reqs:
        fgr.fgr_fggc_plan_destroy(r["plan"])
        r["ctx"].close()


def _batch(fgr, reqs, stream=None):
    fgr.fgr_reconstruct_fggc_batch([r["ctx"] for r in reqs], [r["plan"] for r in reqs],
                                   [r["packets"] for r in reqs], [r["u"] for r in reqs], stream)


@pytest.mark.parametrize("prec,count", [("fp32", 40), ("fp64", 12)])
def test_batch_equals_planned_calls_and_oracle(fgr, prec, count):
    import torch
    reqs = _requests(fgr, prec, count, seed=1 if prec == "fp32" else 2)
    try:
        _batch(fgr, reqs)
        torch.cuda.synchronize()
        tol_self = 1e-13 if prec == "fp64" else 1e-6
        strat = lsa.Strategy(nq=4, np_=2)
        floor = 4 * np.finfo(float).eps / math.sqrt(strat.pinv.singular_values[-1])
        for i, r in enumerate(reqs):
            got = r["u"].cpu().numpy()
            ref = torch.zeros_like(r["u"])
            fgr.fgr_reconstruct_fggc_planned(r["ctx"].handle, r["plan"], r["packets"], ref)
            torch.cuda.synchronize()
            assert not fgr.fgr_fggc_plan_overflow(r["plan"])
            assert _gpu.rel_l2(got, ref.cpu().numpy()) <= tol_self, i
            if i % 4 == 0:  # the oracle on a share of the requests
                R = 8 if prec == "fp64" else 6
                o = fggc.reconstruct(r["pk"], r["grid"], r["eps"], r["mesh"].dq, r["mesh"].dp, strat, R=R)
                assert _gpu.rel_l2(got, o) <= (max(floor, 1e-12) if prec == "fp64" else 1e-5), i
    finally:
        _close(fgr, reqs)


def test_batch_replays_from_a_cuda_graph_and_flags_overflow(fgr):
    import torch
    reqs = _requests(fgr, "fp32", 10, seed=3)
    try:
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            _batch(fgr, reqs, s)   # warm-up outside the capture
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            g.capture_begin()
            _batch(fgr, reqs, s)
            g.capture_end()
        torch.cuda.synchronize()
        for it in range(2):
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
        # request 0's packets leave its box: only its flag is raised
        reqs[0]["arrs"][1].add_(12 * reqs[0]["mesh"].dp)
        g.replay()
        torch.cuda.synchronize()
        assert fgr.fgr_fggc_plan_overflow(reqs[0]["plan"])
        assert not any(fgr.fgr_fggc_plan_overflow(r["plan"]) for r in reqs[1:])
    finally:
        _close(fgr, reqs)


def test_batch_of_an_empty_request_and_argument_checks(fgr):
    import torch
    reqs = _requests(fgr, "fp32", 3, seed=4)
    try:
        # a request whose packets are far from its grid: its output is zero
        eps = 1 / 256
        pk = random_packets(99, 1, 50, q_range=(40, 41), p_range=(-1, 1), mesh=mesh_for(1, eps))
        ctx = fgr.Context(1, _grid(1, 1024), eps, _gpu.options("fp32"))
        arrs = _gpu.to_device(pk)
        packets = fgr.make_packets(*arrs)
        plan = fgr.fgr_fggc_plan_create(ctx.handle, packets, 2)
        u = torch.full((1024,), 5.0, dtype=torch.complex64, device="cuda")
        reqs.append(dict(pk=pk, ctx=ctx, arrs=arrs, packets=packets, plan=plan, u=u))
        _batch(fgr, reqs)
        torch.cuda.synchronize()
        assert float(torch.abs(u).max()) == 0.0
        # another precision in the same batch is refused, naming the request
        other = fgr.Context(1, _grid(1, 1024), eps, _gpu.options("fp64"))
        try:
            with pytest.raises(fgr.FgrError) as e:
                fgr.fgr_reconstruct_fggc_batch([reqs[0]["ctx"], other], [reqs[0]["plan"], plan],
                                               [reqs[0]["packets"], packets], [reqs[0]["u"], u])
            assert e.value.status == fgr.fgr.FGR_E_INVALID and "request 1" in str(e.value)
        finally:
            other.close()
        with pytest.raises(fgr.FgrError):   # a plan of another context
            fgr.fgr_reconstruct_fggc_batch([reqs[1]["ctx"]], [plan], [reqs[1]["packets"]], [reqs[1]["u"]])
    finally:
        _close(fgr, reqs)
