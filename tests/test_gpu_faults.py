"""Failure handling without faulting the GPU: an allocation failure injected on
the host (FGR_INJECT_ALLOC_FAILURE=n fails the n-th scratch allocation of the
process) must come back as FGR_E_NOMEM with a message, leave the context
usable, and fail only its own request in the server."""

import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(code: str, fail_at: int) -> str:
    env = dict(os.environ, FGR_INJECT_ALLOC_FAILURE=str(fail_at), PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", textwrap.dedent(code)], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    return r.stdout


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_injected_allocation_failure_is_reported_and_recoverable():
    out = _run("""
        import math, numpy as np, torch
        import paper_2504_21785_gb300 as fgr
        from workloads import random_packets
        pk = random_packets(1, 1, 500, q_range=(-2, 2), p_range=(-2, 2))
        arrs = [torch.tensor(np.ascontiguousarray(pk[k]), dtype=torch.float64, device="cuda") for k in "qpsa"]
        grid = dict(d=1, n=[2048], lo=[-math.pi], hi=[math.pi])
        ctx = fgr.Context(1, grid, 1/256, fgr.make_options(precision=fgr.FGR_FP32))
        u = torch.zeros(2048, dtype=torch.complex64, device="cuda")
        try:
            fgr.fgr_reconstruct_direct(ctx.handle, fgr.make_packets(*arrs), u)
            print("NO-ERROR")
        except fgr.FgrError as e:
            print("STATUS", e.status, "injected" in str(e))
        fgr.fgr_reconstruct_direct(ctx.handle, fgr.make_packets(*arrs), u)   # recovers
        v = torch.zeros_like(u)
        fgr.fgr_reconstruct_direct(ctx.handle, fgr.make_packets(*arrs), v)
        torch.cuda.synchronize()
        print("AGREE", bool(torch.allclose(u, v, rtol=1e-5, atol=1e-6)))
    """, fail_at=2)
    assert "STATUS 2 True" in out
    assert "AGREE True" in out


def test_injected_failure_fails_only_its_request_in_the_server():
    out = _run("""
        import math, numpy as np, torch
        import paper_2504_21785_gb300 as fgr
        from workloads import random_packets
        pk = random_packets(2, 1, 800, q_range=(-2, 2), p_range=(-2, 2))
        srv = fgr.fgr_server_create(1 << 30, 1)
        sid = fgr.fgr_register_packets(srv, 1, fgr.make_packets(*[np.ascontiguousarray(pk[k]) for k in "qpsa"]))
        grid = dict(d=1, n=[1024], lo=[-math.pi], hi=[math.pi])
        opt = fgr.make_options(precision=fgr.FGR_FP32)
        outs = [torch.zeros(1024, dtype=torch.complex64, device="cuda") for _ in range(3)]
        st = []
        for u in outs:   # one slot: requests run one after the other
            t = fgr.fgr_submit(srv, fgr.make_request(0, grid, 1/256, opt, sid, u))
            st.append(fgr.fgr_poll(srv, t, -1).status)
        fgr.fgr_server_destroy(srv)
        print("STATUSES", st)
    """, fail_at=6)
    # each direct reconstruction takes four scratch buffers: the sixth is the
    # second request's second buffer
    assert "STATUSES [0, 2, 0]" in out
