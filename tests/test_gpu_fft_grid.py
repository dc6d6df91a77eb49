"""GPU parity of the DFT grid stage (FGR_FLAG_FFT_GRID): FGGC on meshes
commensurate with the grid (h dp / eps = 2 pi / N), where the sum over the
p-nodes of each q-node is an inverse DFT (Sec. 2.3 after eq. 2.25; Remark 3).
Checked on the meshes of Examples 4 and 5 of Sec. 4.4 (h = eps, so
N = 16 / sqrt(eps): 1024 and 128) against the FP64 oracle's FGGC (eq. 2.24
evaluated node by node) and against the library's direct grid stage.

Tolerances: FP64 at the least-squares conditioning floor (as for the direct
grid stage: max(1e-12, 4 eps_mach / sqrt(lambda_min))), FP32 1e-5 against the
oracle; the two GPU routes agree to 1e-12 (FP64) and 1e-6 (FP32)."""

import math

import numpy as np
import pytest

import paper_2504_21785_gb300 as fgr
from oracle import fggc, lsa
from workloads import random_packets, mesh_for
from workloads.examples import EXAMPLES, example_grid

from . import _gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fgr.fgr.load()


def _fp64_tol(nq, np_):
    strat = lsa.Strategy(nq=nq, np_=np_)
    floor = np.finfo(float).eps / math.sqrt(strat.pinv.singular_values[strat.pinv.rank - 1])
    return max(1e-12, 4 * floor)


def _packets(ex, m, seed):
    e = EXAMPLES[ex]
    mesh = mesh_for(e["d"], e["eps"])
    pk = random_packets(seed, e["d"], m, q_range=(e["q"][0] + 0.1, e["q"][1] - 0.1),
                        p_range=(e["p"][0] + 0.1, e["p"][1] - 0.1), s_range=(-2, 2), mesh=mesh,
                        on_node_fraction=0.05)
    return pk, mesh, e["eps"], example_grid(ex)


def _opts(precision, nq, np_, fft):
    return _gpu.options(precision, nq=nq, np_=np_) if not fft else _fft_options(precision, nq, np_)


def _fft_options(precision, nq, np_):
    o = _gpu.options(precision, nq=nq, np_=np_)
    o.flags = fgr.FGR_FLAG_FFT_GRID
    return o


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("nq,np_", [(2, 2), (4, 2)])
def test_example4_mesh_matches_oracle(precision, nq, np_):
    pk, mesh, eps, grid = _packets(4, 3000, seed=41)
    R = 8 if precision == "fp64" else 6
    ref = fggc.reconstruct(pk, grid, eps, mesh.dq, mesh.dp, lsa.Strategy(nq=nq, np_=np_), R=R)
    got = _gpu.reconstruct("fggc", pk, grid, eps, _fft_options(precision, nq, np_))
    k5 = _gpu.reconstruct("fggc", pk, grid, eps, _gpu.options(precision, nq=nq, np_=np_))
    err, diff = _gpu.rel_l2(got, ref), _gpu.rel_l2(got, k5)
    print("DFT grid stage, Example 4 mesh, %s Q%dP%d: vs oracle %.3e, vs direct stage %.3e"
          % (precision, nq, np_, err, diff))
    assert err <= (_fp64_tol(nq, np_) if precision == "fp64" else 1e-5)
    assert diff <= (1e-12 if precision == "fp64" else 1e-6)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_example5_mesh_matches_oracle(precision):
    pk, mesh, eps, grid = _packets(5, 1500, seed=42)
    R = 8 if precision == "fp64" else 6
    rng = np.random.default_rng(7)
    pts = np.stack([rng.integers(0, grid["n"][l], 700) for l in range(2)])
    ref = fggc.reconstruct(pk, grid, eps, mesh.dq, mesh.dp, lsa.Strategy(nq=2, np_=2), R=R, points=pts)
    got = _gpu.reconstruct("fggc", pk, grid, eps, _fft_options(precision, 2, 2))
    k5 = _gpu.reconstruct("fggc", pk, grid, eps, _gpu.options(precision, nq=2, np_=2))
    err, diff = _gpu.rel_l2(got[tuple(pts)], ref), _gpu.rel_l2(got, k5)
    print("DFT grid stage, Example 5 mesh, %s: vs oracle %.3e, vs direct stage %.3e" % (precision, err, diff))
    assert err <= (_fp64_tol(2, 2) if precision == "fp64" else 1e-5)
    assert diff <= (1e-12 if precision == "fp64" else 1e-6)


def test_wide_momentum_range_folds_modulo_n():
    # p-ranges longer than N p-nodes fold onto the same DFT bins (the kernel is
    # N-periodic in b): Example 5's N = 128, momenta over [-8, 8] span ~330 nodes
    e = EXAMPLES[5]
    mesh = mesh_for(2, e["eps"])
    pk = random_packets(43, 2, 800, q_range=(-1.0, 1.0), p_range=(-8, 8), s_range=(-1, 1), mesh=mesh)
    grid = example_grid(5)
    rng = np.random.default_rng(8)
    pts = np.stack([rng.integers(0, grid["n"][l], 500) for l in range(2)])
    ref = fggc.reconstruct(pk, grid, e["eps"], mesh.dq, mesh.dp, lsa.Strategy(nq=4, np_=2), R=8, points=pts)
    got = _gpu.reconstruct("fggc", pk, grid, e["eps"], _fft_options("fp64", 4, 2))
    assert _gpu.rel_l2(got[tuple(pts)], ref) <= _fp64_tol(4, 2)


def test_incommensurate_grid_is_rejected_and_snap_makes_it_commensurate():
    eps = 2.0 ** -12
    grid = dict(d=1, n=[1000], lo=[-2.0], hi=[2.0])   # h dp / eps = 2 pi / 62.6
    with pytest.raises(fgr.FgrError) as e:
        fgr.Context(1, grid, eps, _fft_options("fp64", 4, 2))
    assert e.value.status == fgr.fgr.FGR_E_INVALID
    o = _fft_options("fp64", 4, 2)
    o.flags = fgr.FGR_FLAG_FFT_GRID | fgr.FGR_FLAG_SNAP_CP
    with fgr.Context(1, grid, eps, o) as ctx:
        info = fgr.fgr_get_info(ctx.handle)
        h = 4.0 / 1000
        n = 2 * math.pi * eps / (h * info.dp)
        assert abs(n - 64) <= 1e-9 * 64                       # snapped to N = 64
        cp = info.dp / math.sqrt(eps)
        assert abs(cp - math.pi / 8) / (math.pi / 8) < 0.03   # a 2 % change of cp
        # the snapped mesh through both grid stages
        mesh = mesh_for(1, eps, cp=cp)
        pk = random_packets(44, 1, 2000, q_range=(-1.5, 1.5), p_range=(-1, 1), mesh=mesh)
        got = _gpu.reconstruct("fggc", pk, grid, eps, o, ctx=ctx)
    plain = _gpu.options("fp64", nq=4, np_=2, cp=cp)
    k5 = _gpu.reconstruct("fggc", pk, grid, eps, plain)
    ref = fggc.reconstruct(pk, grid, eps, mesh.dq, mesh.dp, lsa.Strategy(nq=4, np_=2, cp=cp), R=8)
    assert _gpu.rel_l2(got, k5) <= 1e-12
    assert _gpu.rel_l2(got, ref) <= _fp64_tol(4, 2)


def test_fft_grid_stage_through_a_plan():
    torch = pytest.importorskip("torch")
    pk, mesh, eps, grid = _packets(4, 2000, seed=45)
    o = _fft_options("fp32", 4, 2)
    arrs = _gpu.to_device(pk)
    packets = fgr.make_packets(*arrs)
    with fgr.Context(1, grid, eps, o) as ctx:
        plan = fgr.fgr_fggc_plan_create(ctx.handle, packets, 2)
        try:
            u = torch.zeros(grid["n"][0], dtype=torch.complex64, device="cuda")
            fgr.fgr_reconstruct_fggc_planned(ctx.handle, plan, packets, u)
            torch.cuda.synchronize()
            assert not fgr.fgr_fggc_plan_overflow(plan)
        finally:
            fgr.fgr_fggc_plan_destroy(plan)
    k5 = _gpu.reconstruct("fggc", pk, grid, eps, _gpu.options("fp32"))
    assert _gpu.rel_l2(u.cpu().numpy(), k5) <= 1e-6
