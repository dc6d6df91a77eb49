"""Multi-step FGGC on the GPU (fgr_fggc_multistep, Algorithm 3 with a fixed mesh
and the flow learned once) against the oracle's multi-step FGGC on the same
inputs: the harmonic oscillator (V = x^2/2) over quarter-period steps, whose
full period the oracle reproduces in closed form (-u0).  Tolerances: FP64 steps
x the FGGC parity tolerance (the least-squares floor eps_mach / sqrt(lambda_min)
per reconstruction), FP32 1e-5."""

import math

import numpy as np
import pytest

from oracle import fga, fggc, lsa, trajectories as tr
from workloads import mesh_for

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


EPS = 1 / 64
POT = {"kind": "harmonic", "omega": 1.0}


def _setup():
    mesh = mesh_for(1, EPS)
    qs = np.arange(-40, 40) * mesh.dq
    ps = np.arange(-80, 80) * mesh.dp
    Q, P = np.meshgrid(qs, ps, indexing="ij")
    M = Q.size
    grid_mesh = {"q": Q.reshape(1, -1), "p": P.reshape(1, -1), "s": np.zeros(M),
                 "a": np.stack([np.ones(M), np.zeros(M)])}
    flow = tr.propagate(grid_mesh, POT, math.pi / 2, 1e-3)
    grid = dict(d=1, n=[512], lo=[-4.0], hi=[4.0])
    x = fga.grid_axis(grid, 0)
    u0 = np.exp(-(x - 0.5) ** 2 / (2 * 0.15)) * np.exp(1j * 0.7 * x / EPS)
    return mesh, grid_mesh, flow, grid, x, u0


def _gpu_multistep(fgr, grid, mesh_pk, flow, u0, steps, precision, on_device=True):
    import torch
    cdt = np.complex128 if precision == "fp64" else np.complex64
    with fgr.Context(1, grid, EPS, _gpu.options(precision)) as ctx:
        if on_device:
            m_arrs, f_arrs = _gpu.to_device(mesh_pk), _gpu.to_device(flow)
            uin = torch.tensor(u0.astype(cdt), device="cuda")
            out = torch.zeros_like(uin)
            fgr.fgr_fggc_multistep(ctx.handle, fgr.make_packets(*m_arrs), fgr.make_packets(*f_arrs), uin, out,
                                   steps)
            torch.cuda.synchronize()
            return out.cpu().numpy()
        hm = [np.ascontiguousarray(mesh_pk[k], dtype=np.float64) for k in "qpsa"]
        hf = [np.ascontiguousarray(flow[k], dtype=np.float64) for k in "qpsa"]
        out = np.zeros(u0.shape, dtype=cdt)
        fgr.fgr_fggc_multistep(ctx.handle, fgr.make_packets(*hm), fgr.make_packets(*hf),
                               np.ascontiguousarray(u0.astype(cdt)), out, steps)
        return out


def _fp64_tol(steps):
    strat = lsa.Strategy(nq=4, np_=2)
    floor = np.finfo(float).eps / math.sqrt(strat.pinv.singular_values[strat.pinv.rank - 1])
    return steps * max(1e-12, 4 * floor)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_multistep_matches_oracle(fgr, precision):
    mesh, grid_mesh, flow, grid, x, u0 = _setup()
    R = 8 if precision == "fp64" else 6
    ref = fggc.multistep(u0, grid, grid_mesh, flow, EPS, mesh.dq, mesh.dp, lsa.Strategy(nq=4, np_=2), 2, R=R)
    got = _gpu_multistep(fgr, grid, grid_mesh, flow, u0, 2, precision)
    tol = _fp64_tol(2) if precision == "fp64" else 1e-5
    assert _gpu.rel_l2(got, ref) <= tol


def test_multistep_full_period_with_the_gpu_flow(fgr):
    # the learned flow itself from fgr_propagate (unit amplitudes); four
    # quarter periods return -u0 (closed form of the harmonic oscillator)
    mesh, grid_mesh, flow, grid, x, u0 = _setup()
    gflow = _gpu.propagate(grid_mesh, 1, POT, math.pi / 2, 1e-3)
    got = _gpu_multistep(fgr, grid, grid_mesh, gflow, u0, 4, "fp32")
    assert _gpu.rel_l2(got, -u0) <= 1e-5


def test_multistep_host_buffers_zero_steps_and_checks(fgr):
    mesh, grid_mesh, flow, grid, x, u0 = _setup()
    a = _gpu_multistep(fgr, grid, grid_mesh, flow, u0, 1, "fp64", on_device=True)
    b = _gpu_multistep(fgr, grid, grid_mesh, flow, u0, 1, "fp64", on_device=False)
    assert _gpu.rel_l2(b, a) <= 1e-13
    z = _gpu_multistep(fgr, grid, grid_mesh, flow, u0, 0, "fp64")
    assert np.array_equal(z, u0)
    short = {k: np.ascontiguousarray(v[..., :10]) for k, v in flow.items() if k in "qpsa"}
    with pytest.raises(fgr.FgrError, match="same"):
        _gpu_multistep(fgr, grid, grid_mesh, short, u0, 1, "fp64")
