"""Examples 4 and 5 of Sec. 4.4 end to end on the GPU with V2 = |x|^2/2,
against the closed-form harmonic solution (oracle/exact.py): the L2 error of
single-step FGA (decompose, propagate over T, direct sum) and of multi-step
FGGC (Algorithm 3, Q2P2) for the T_evo x T_multi splits of Tables 18 and 20.
The paper measures these errors against a time-splitting spectral solution.
For this potential FGA itself is exact up to the mesh and the window (error
below 1e-9 here), so the printed FGA error of Example 4 (3.151e-5, Table 18)
is read as the error of that reference; combined in quadrature with it, the
single-step error here must reproduce the printed 3.376e-5 to 10 %, and every
split must stay below 1.2 x its printed value.  In Example 5 (eps = 2^-6) the
reference error is small (printed FGA error 6.6e-6) and the multi-step errors
must reproduce Table 20 to 25 % (T_multi = 8, 16, 32; the shorter splits take
minutes of RK4 on 17M packets and are timed by the bench study instead).
FP64 contexts (R = 8)."""

import math

import pytest

from oracle import exact
from workloads.examples import (BETA, EXAMPLES, example_axes_x, example_axis, example_grid, example_n0,
                                example_u0)

from . import _gpu

pytestmark = pytest.mark.gpu

TABLE18 = {"FGA": 3.151e-5, 1: 3.376e-5, 2: 6.003e-5, 4: 1.147e-4, 8: 1.582e-4, 16: 1.755e-4, 32: 2.509e-4}
TABLE20 = {"FGA": 6.640e-6, 1: 7.793e-5, 2: 1.947e-5, 4: 6.855e-5, 8: 8.337e-5, 16: 1.936e-4, 32: 3.130e-4}


@pytest.fixture(scope="module")
def fgr():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2504_21785_gb300 as pkg
    pkg.fgr.load()
    return pkg


def _exact(ex):
    e = EXAMPLES[ex]
    d = e["d"]
    return exact.harmonic_gaussian(example_axes_x(ex), e["T"], e["eps"], BETA, [0.0] * d, [1.0] * d,
                                   example_n0(ex))


def _h(ex):
    g = example_grid(ex)
    return [(g["hi"][l] - g["lo"][l]) / g["n"][l] for l in range(g["d"])]


def _mesh_packets(torch, ex):
    """The tensor-product mesh expanded into packets on the device (row-major)."""
    d = EXAMPLES[ex]["d"]
    q, p = example_axis(ex)
    aq, ap = torch.tensor(q, device="cuda"), torch.tensor(p, device="cuda")
    L = q.size
    idx = torch.arange(L ** d, device="cuda")
    cols = []
    for l in range(d):
        cols.append((idx // (L ** (d - 1 - l))) % L)
    Q = torch.stack([aq[c] for c in cols]).contiguous()
    P = torch.stack([ap[c] for c in cols]).contiguous()
    return Q, P, (aq, ap)


def _flow(fgr, torch, ctx, Q, P, pot, t, dt):
    m = Q.shape[1]
    fs = torch.zeros(m, dtype=torch.float64, device="cuda")
    fa = torch.zeros((2, m), dtype=torch.float64, device="cuda")
    fa[0] = 1.0
    pk = fgr.make_packets(Q.clone(), P.clone(), fs, fa)
    fgr.fgr_propagate(ctx.handle, pk, fgr.make_potential(**pot), t, dt)
    return pk


def _run(fgr, ex, splits, with_fga):
    import torch
    e = EXAMPLES[ex]
    d, eps = e["d"], e["eps"]
    grid = example_grid(ex)
    u0 = torch.tensor(example_u0(ex), device="cuda")
    ref = _exact(ex)
    pot = e["potentials"]["V2"]
    Q, P, (aq, ap) = _mesh_packets(torch, ex)
    errs = {}
    with fgr.Context(d, grid, eps, _gpu.options("fp64", nq=2, np_=2)) as ctx:
        if with_fga:
            m = Q.shape[1]
            s = torch.zeros(m, dtype=torch.float64, device="cuda")
            a = torch.zeros((2, m), dtype=torch.float64, device="cuda")
            pk = fgr.make_packets(Q.clone(), P.clone(), s, a)
            fgr.fgr_decompose(ctx.handle, u0, pk)
            fgr.fgr_propagate(ctx.handle, pk, fgr.make_potential(**pot), e["T"], e["dt"])
            u = torch.zeros_like(u0)
            fgr.fgr_reconstruct_direct(ctx.handle, pk, u)
            torch.cuda.synchronize()
            errs["FGA"] = exact.l2_error(u.cpu().numpy(), ref, _h(ex))
        axes = fgr.make_axes([(aq, ap)] * d)
        for M in splits:
            flow = _flow(fgr, torch, ctx, Q, P, pot, e["T"] / M, e["dt"])
            u = torch.zeros_like(u0)
            fgr.fgr_fggc_multistep_tensor(ctx.handle, axes, None, flow, u0, u, M)
            torch.cuda.synchronize()
            errs[M] = exact.l2_error(u.cpu().numpy(), ref, _h(ex))
            del flow
    return errs


def _report(name, errs, table):
    print("\n%s: %s" % (name, "  ".join("%s %.3e (paper %.3e)" % (k, v, table[k]) for k, v in errs.items())))


def test_example4_v2_errors_against_the_exact_solution(fgr):
    errs = _run(fgr, 4, (1, 2, 4, 8, 16, 32), with_fga=True)
    _report("Example 4, V2", errs, TABLE18)
    assert errs["FGA"] <= 1e-9
    assert abs(math.hypot(errs[1], TABLE18["FGA"]) / TABLE18[1] - 1) <= 0.10
    for k in (1, 2, 4, 8, 16, 32):
        assert errs[k] <= 1.2 * TABLE18[k], (k, errs[k])


def test_example5_v2_errors_against_the_exact_solution(fgr):
    errs = _run(fgr, 5, (8, 16, 32), with_fga=False)
    _report("Example 5, V2", errs, TABLE20)
    for k, v in errs.items():
        assert abs(v / TABLE20[k] - 1) <= 0.25, (k, v)
