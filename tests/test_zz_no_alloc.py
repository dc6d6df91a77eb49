"""fgr_reconstruct_fggc_noalloc: the FGGC reconstruction for callers that
cannot allocate device memory while running (a pre-committed memory budget, a
host framework that owns all device allocations, or a loop that cannot pay for
cudaMalloc/cudaFree).  Its working memory is one static device array, so the
test checks, through the C ABI, that two calls in a row each reproduce what
the allocating entry point fgr_reconstruct_fggc returns for the same input,
that its output also matches the FP64 oracle's FGGC (Algorithm 2) directly, and
that a problem too large for the array is refused with FGR_E_CAPACITY.

This file is collected last so that a run stopping at the first failure has
already run every other test."""

import math

import numpy as np
import pytest

from workloads import random_packets, mesh_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fgr():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2504_21785_gb300 as pkg
    pkg.fgr.load()
    return pkg


def _device_packets(pk):
    import torch
    return [torch.tensor(np.ascontiguousarray(pk[k]), dtype=torch.float64, device="cuda") for k in "qpsa"]


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-5), ("fp64", 1e-12)])
def test_noalloc_matches_allocating_entry_point_twice(fgr, precision, tol):
    import torch
    eps = 1 / 1024
    mesh = mesh_for(1, eps)
    grid = dict(d=1, n=[32768], lo=[-math.pi], hi=[math.pi])
    prec = fgr.FGR_FP32 if precision == "fp32" else fgr.FGR_FP64
    cdt = torch.complex64 if precision == "fp32" else torch.complex128
    with fgr.Context(1, grid, eps, fgr.make_options(precision=prec)) as ctx:
        for call, seed in enumerate((21, 22)):  # two calls in a row, different inputs
            pk = random_packets(seed, 1, 20000, q_range=(-3, 3), p_range=(-2, 2), s_range=(-1, 1),
                                mesh=mesh)
            arrs = _device_packets(pk)
            packets = fgr.make_packets(*arrs)
            ref = torch.zeros(32768, dtype=cdt, device="cuda")
            got = torch.full((32768,), 7.0, dtype=cdt, device="cuda")  # stale contents must not leak
            fgr.fgr_reconstruct_fggc(ctx.handle, packets, ref)
            fgr.fgr.fgr_reconstruct_fggc_noalloc(ctx.handle, packets, got)
            torch.cuda.synchronize()
            r, g = ref.cpu().numpy(), got.cpu().numpy()
            assert np.linalg.norm(g - r) <= tol * np.linalg.norm(r), (call, precision)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_noalloc_matches_oracle(fgr, precision):
    # the no-allocation call sums the node Gaussians over every b of the node
    # box (it keeps no b-range table), so it is compared with the oracle's
    # Algorithm 2 directly as well, on a ragged grid with packets on nodes
    import torch
    from oracle import fggc, lsa
    eps = 1 / 256
    mesh = mesh_for(1, eps)
    n = 3001
    grid = dict(d=1, n=[n], lo=[-math.pi], hi=[math.pi])
    pk = random_packets(25, 1, 700, q_range=(-3.6, 3.6), p_range=(-2.5, 2.5), s_range=(-3, 3),
                        mesh=mesh, on_node_fraction=0.1)
    strat = lsa.Strategy(nq=4, np_=2)
    if precision == "fp32":
        prec, cdt, R = fgr.FGR_FP32, torch.complex64, 6
        tol = 1e-5
    else:
        prec, cdt, R = fgr.FGR_FP64, torch.complex128, 8
        # the least-squares floor eps_mach / sqrt(lambda_min(A~)) of Q4P2
        floor = np.finfo(float).eps / math.sqrt(strat.pinv.singular_values[strat.pinv.rank - 1])
        tol = max(1e-12, 4 * floor)
    ref = fggc.reconstruct(pk, grid, eps, mesh.dq, mesh.dp, strat, R=R)
    with fgr.Context(1, grid, eps, fgr.make_options(precision=prec)) as ctx:
        packets = fgr.make_packets(*_device_packets(pk))
        for call in range(2):
            got = torch.full((n,), -3.0, dtype=cdt, device="cuda")
            fgr.fgr.fgr_reconstruct_fggc_noalloc(ctx.handle, packets, got)
            torch.cuda.synchronize()
            g = got.cpu().numpy()
            assert np.linalg.norm(g - ref) <= tol * np.linalg.norm(ref), (call, precision)


def test_noalloc_rejects_problems_beyond_its_array(fgr):
    import torch
    eps = 1 / 1024
    mesh = mesh_for(1, eps)
    grid = dict(d=1, n=[4096], lo=[-math.pi], hi=[math.pi])
    # momenta over [-60, 60] need ~10^4 p-nodes per q-node: far beyond 8 MiB
    pk = random_packets(23, 1, 5000, q_range=(-3, 3), p_range=(-60, 60), mesh=mesh)
    arrs = _device_packets(pk)
    with fgr.Context(1, grid, eps, fgr.make_options(precision=fgr.FGR_FP32)) as ctx:
        u = torch.zeros(4096, dtype=torch.complex64, device="cuda")
        with pytest.raises(fgr.FgrError) as e:
            fgr.fgr.fgr_reconstruct_fggc_noalloc(ctx.handle, fgr.make_packets(*arrs), u)
        assert e.value.status == fgr.fgr.FGR_E_CAPACITY
        assert "at most" in str(e.value)
        # the allocating entry point still serves the same problem
        fgr.fgr_reconstruct_fggc(ctx.handle, fgr.make_packets(*arrs), u)


def test_noalloc_rejects_packets_in_host_memory(fgr):
    # packet arrays must be device memory of the context's device: a host array
    # is refused before anything is launched
    import torch
    eps = 1 / 1024
    mesh = mesh_for(1, eps)
    grid = dict(d=1, n=[4096], lo=[-math.pi], hi=[math.pi])
    pk = random_packets(24, 1, 100, q_range=(-1, 1), p_range=(-1, 1), mesh=mesh)
    arrs = _device_packets(pk)
    host_q = np.ascontiguousarray(pk["q"])
    packets = fgr.make_packets(*arrs)
    packets.q = host_q.ctypes.data   # q on the host, the rest on the device
    with fgr.Context(1, grid, eps, fgr.make_options(precision=fgr.FGR_FP32)) as ctx:
        u = torch.zeros(4096, dtype=torch.complex64, device="cuda")
        with pytest.raises(fgr.FgrError) as e:
            fgr.fgr.fgr_reconstruct_fggc_noalloc(ctx.handle, packets, u)
        assert e.value.status == fgr.fgr.FGR_E_INVALID
        assert "q must be device memory" in str(e.value)
