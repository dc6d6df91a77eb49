"""GPU parity of the tensor-product decomposition (fgr_decompose_tensor, eq. 2.8
factorised over dimensions) and of multi-step FGGC over a tensor mesh
(fgr_fggc_multistep_tensor, Algorithm 3) with the FP64 oracle, which sums
every packet of the expanded mesh one by one: FP64 to 1e-12, FP32 to 1e-5
(relative L2 over the amplitudes).  Cases: d = 1..3, whole products and
selections (host and device), unsorted axes, windows clipped by or off the
grid, the 2-D workload mesh at full size on a sample, and invalid selections."""

import math

import numpy as np
import pytest

from oracle import decompose, fggc, lsa, trajectories as tr
from workloads import config_workload, workload_axes, WKB_TANH

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


SHAPES = {1: (3001,), 2: (70, 101), 3: (20, 17, 23)}


def _axes(d, seed, lens, sort=True):
    rng = np.random.default_rng(seed)
    axes = []
    for l in range(d):
        q = rng.uniform(-3.6, 3.6, lens[l])
        q[0] = 20.0  # one entry whose window misses the grid
        p = rng.uniform(-4, 4, lens[l])
        if sort:
            o = np.argsort(q, kind="stable")
            q, p = q[o], p[o]
        axes.append((np.ascontiguousarray(q), np.ascontiguousarray(p)))
    return axes


def _expand(axes, sel):
    d = len(axes)
    idx = np.unravel_index(sel, tuple(ax[0].size for ax in axes))
    q = np.stack([axes[l][0][idx[l]] for l in range(d)])
    p = np.stack([axes[l][1][idx[l]] for l in range(d)])
    return q, p


def _run(fgr, grid, eps, u, axes, sel, m, precision, device=True):
    import torch
    d = grid["d"]
    cdt = np.complex128 if precision == "fp64" else np.complex64
    with fgr.Context(d, grid, eps, _gpu.options(precision)) as ctx:
        if device:
            ax = fgr.make_axes([(torch.tensor(q, device="cuda"), torch.tensor(p, device="cuda")) for q, p in axes])
            ut = torch.tensor(u.astype(cdt), device="cuda")
            st = None if sel is None else torch.tensor(sel, device="cuda")
            out = torch.zeros((2, m), dtype=torch.float64, device="cuda")
            fgr.fgr_decompose_tensor(ctx.handle, ax, ut, m, st, out)
            torch.cuda.synchronize()
            return out.cpu().numpy()
        ax = fgr.make_axes(axes)
        out = np.zeros((2, m))
        fgr.fgr_decompose_tensor(ctx.handle, ax, np.ascontiguousarray(u.astype(cdt)), m,
                                 None if sel is None else np.ascontiguousarray(sel), out)
        return out


def _rel(got, ref):
    g, r = got[0] + 1j * got[1], ref[0] + 1j * ref[1]
    return float(np.linalg.norm(g - r) / np.linalg.norm(r))


LENS = {1: (700,), 2: (40, 50), 3: (9, 8, 10)}
EPS = {1: 1 / 256, 2: 1 / 64, 3: 1 / 16}


@pytest.mark.parametrize("d", [1, 2, 3])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_tensor_decompose_matches_oracle(fgr, d, precision):
    n = SHAPES[d]
    grid = dict(d=d, n=list(n), lo=[-math.pi] * d, hi=[math.pi] * d)
    rng = np.random.default_rng(d)
    u = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    axes = _axes(d, 10 + d, LENS[d])
    total = int(np.prod(LENS[d]))
    sel = np.arange(total)
    q, p = _expand(axes, sel)
    R = 8 if precision == "fp64" else 6
    ref = decompose.decompose(u, grid, q, p, EPS[d], R=R)
    got = _run(fgr, grid, EPS[d], u, axes, None, total, precision)
    assert _rel(got, ref) <= (1e-12 if precision == "fp64" else 1e-5)
    off = np.any(q == 20.0, axis=0)  # windows off the grid
    assert off.any() and np.all(got[:, off] == 0)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_tensor_decompose_selection_host_device_unsorted(fgr, d):
    n = SHAPES[d]
    grid = dict(d=d, n=list(n), lo=[-math.pi] * d, hi=[math.pi] * d)
    rng = np.random.default_rng(20 + d)
    u = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    axes = _axes(d, 30 + d, LENS[d], sort=False)
    total = int(np.prod(LENS[d]))
    sel = rng.choice(total, 517, replace=True).astype(np.int64)  # repeats allowed
    q, p = _expand(axes, sel)
    ref = decompose.decompose(u, grid, q, p, EPS[d], R=6)
    dev = _run(fgr, grid, EPS[d], u, axes, sel, sel.size, "fp32", device=True)
    host = _run(fgr, grid, EPS[d], u, axes, sel, sel.size, "fp32", device=False)
    assert _rel(dev, ref) <= 1e-5
    assert _rel(host, dev) <= 1e-6


def test_tensor_decompose_equals_per_packet_kernel(fgr):
    import torch
    d, n = 2, SHAPES[2]
    grid = dict(d=d, n=list(n), lo=[-math.pi] * d, hi=[math.pi] * d)
    rng = np.random.default_rng(5)
    u = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    axes = _axes(d, 6, LENS[2])
    total = int(np.prod(LENS[2]))
    t = _run(fgr, grid, EPS[2], u, axes, None, total, "fp64")
    q, p = _expand(axes, np.arange(total))
    with fgr.Context(d, grid, EPS[2], _gpu.options("fp64")) as ctx:
        arrs = [torch.tensor(x, device="cuda") for x in (q, p, np.zeros(total), np.zeros((2, total)))]
        fgr.fgr_decompose(ctx.handle, torch.tensor(u, device="cuda"), fgr.make_packets(*arrs))
        torch.cuda.synchronize()
        per = arrs[3].cpu().numpy()
    assert _rel(t, per) <= 1e-13


def test_tensor_decompose_workload_mesh_full_size(fgr):
    # the 2-D workload's 64^2 x 32^2 = 4.2M-packet mesh on its 1024^2 grid,
    # u0 of its WKB data; the oracle sums a seeded sample of packets
    import torch
    w = config_workload(3)
    grid, eps = w["grid"], w["eps"]
    axes, sel = workload_axes(w)
    ax0 = np.linspace(-math.pi, math.pi, grid["n"][0], endpoint=False)
    X = np.stack(np.meshgrid(ax0, ax0, indexing="ij"))
    u = WKB_TANH.u0(X, eps)
    m = sel.size
    got = _run(fgr, grid, eps, u, axes, sel, m, "fp32")
    rng = np.random.default_rng(11)
    pick = np.sort(rng.choice(m, 1500, replace=False))
    pk = w["packets"]
    ref = decompose.decompose(u, grid, pk["q"][:, pick], pk["p"][:, pick], eps, R=6)
    assert _rel(got[:, pick], ref) <= 1e-5
    del torch


def test_tensor_decompose_invalid(fgr):
    import torch
    grid = dict(d=2, n=[16, 16], lo=[-1.0, -1.0], hi=[1.0, 1.0])
    axes = _axes(2, 1, (4, 5))
    u = np.zeros((16, 16), np.complex128)
    with fgr.Context(2, grid, 1 / 64, _gpu.options("fp64")) as ctx:
        ax = fgr.make_axes(axes)
        with pytest.raises(fgr.FgrError):  # m != product without sel
            fgr.fgr_decompose_tensor(ctx.handle, ax, u, 19, None, np.zeros((2, 19)))
        with pytest.raises(fgr.FgrError, match="outside"):  # host sel out of range
            fgr.fgr_decompose_tensor(ctx.handle, ax, u, 2, np.array([0, 20], np.int64), np.zeros((2, 2)))
        bad = torch.tensor([3, -1, 7], dtype=torch.int64, device="cuda")
        with pytest.raises(fgr.FgrError, match="outside"):  # device sel out of range
            fgr.fgr_decompose_tensor(ctx.handle, ax, u, 3, bad, np.zeros((2, 3)))
        # the context stays usable
        out = np.zeros((2, 20))
        fgr.fgr_decompose_tensor(ctx.handle, ax, u, 20, None, out)
        assert np.all(out == 0)


def test_multistep_tensor_matches_oracle(fgr):
    # 2-D harmonic oscillator, mesh = tensor product of two 1-D meshes, one
    # quarter-period step, flow from the oracle's RK4 of the expanded mesh
    import torch
    from workloads import mesh_for
    eps = 1 / 16
    mesh = mesh_for(2, eps)
    ax = []
    for l in range(2):
        qs = np.arange(-5, 5) * mesh.dq
        ps = np.arange(-10, 10) * mesh.dp
        Q, P = np.meshgrid(qs, ps, indexing="ij")
        ax.append((np.ascontiguousarray(Q.reshape(-1)), np.ascontiguousarray(P.reshape(-1))))
    total = ax[0][0].size * ax[1][0].size
    q, p = _expand(ax, np.arange(total))
    grid_mesh = {"q": q, "p": p, "s": np.zeros(total), "a": np.stack([np.ones(total), np.zeros(total)])}
    flow = tr.propagate(grid_mesh, {"kind": "harmonic", "omega": 1.0}, math.pi / 2, 1e-3)
    grid = dict(d=2, n=[48, 40], lo=[-3.0, -3.0], hi=[3.0, 3.0])
    x0 = np.linspace(-3, 3, 48, endpoint=False)
    x1 = np.linspace(-3, 3, 40, endpoint=False)
    X0, X1 = np.meshgrid(x0, x1, indexing="ij")
    u0 = np.exp(-((X0 - 0.4) ** 2 + (X1 + 0.3) ** 2) / (2 * 0.2)) * np.exp(1j * (0.5 * X0 - 0.8 * X1) / eps)
    ref = fggc.multistep(u0, grid, grid_mesh, flow, eps, mesh.dq, mesh.dp, lsa.Strategy(nq=4, np_=2), 1, R=6)
    with fgr.Context(2, grid, eps, _gpu.options("fp32")) as ctx:
        axd = fgr.make_axes([(torch.tensor(a, device="cuda"), torch.tensor(b, device="cuda")) for a, b in ax])
        fl = [torch.tensor(np.ascontiguousarray(flow[k]), device="cuda") for k in "qpsa"]
        uin = torch.tensor(u0.astype(np.complex64), device="cuda")
        out = torch.zeros_like(uin)
        fgr.fgr_fggc_multistep_tensor(ctx.handle, axd, None, fgr.make_packets(*fl), uin, out, 1)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
    assert _gpu.rel_l2(got, ref) <= 1e-5


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_multistep_tensor_with_selection_matches_oracle(fgr, precision):
    # 2-D harmonic oscillator on a selected subset of a tensor mesh (host and
    # device selections), two quarter-period steps, flow from the oracle's RK4
    import torch
    from workloads import mesh_for
    eps = 1 / 16
    mesh = mesh_for(2, eps)
    ax = []
    for l in range(2):
        qs = np.arange(-5, 5) * mesh.dq
        ps = np.arange(-9, 9) * mesh.dp
        Q, P = np.meshgrid(qs, ps, indexing="ij")
        ax.append((np.ascontiguousarray(Q.reshape(-1)), np.ascontiguousarray(P.reshape(-1))))
    total = ax[0][0].size * ax[1][0].size
    rng = np.random.default_rng(12)
    sel = np.sort(rng.choice(total, total * 3 // 4, replace=False)).astype(np.int64)
    q, p = _expand(ax, sel)
    m = sel.size
    sub = {"q": q, "p": p, "s": np.zeros(m), "a": np.stack([np.ones(m), np.zeros(m)])}
    flow = tr.propagate(sub, {"kind": "harmonic", "omega": 1.0}, math.pi / 2, 1e-3)
    grid = dict(d=2, n=[40, 36], lo=[-3.0, -3.0], hi=[3.0, 3.0])
    x0 = np.linspace(-3, 3, 40, endpoint=False)
    x1 = np.linspace(-3, 3, 36, endpoint=False)
    X0, X1 = np.meshgrid(x0, x1, indexing="ij")
    u0 = np.exp(-((X0 - 0.3) ** 2 + (X1 + 0.2) ** 2) / (2 * 0.2)) * np.exp(1j * (0.4 * X0 - 0.6 * X1) / eps)
    R = 8 if precision == "fp64" else 6
    ref = fggc.multistep(u0, grid, sub, flow, eps, mesh.dq, mesh.dp, lsa.Strategy(nq=4, np_=2), 2, R=R)
    cdt = np.complex128 if precision == "fp64" else np.complex64
    tol = 2 * max(1e-12, 4 * np.finfo(float).eps / math.sqrt(
        lsa.Strategy(nq=4, np_=2).pinv.singular_values[lsa.Strategy(nq=4, np_=2).pinv.rank - 1])) \
        if precision == "fp64" else 1e-5
    with fgr.Context(2, grid, eps, _gpu.options(precision)) as ctx:
        fl = [torch.tensor(np.ascontiguousarray(flow[k]), device="cuda") for k in "qpsa"]
        for on_device in (True, False):
            if on_device:
                axd = fgr.make_axes([(torch.tensor(a, device="cuda"), torch.tensor(b, device="cuda")) for a, b in ax])
                s_arg = torch.tensor(sel, device="cuda")
            else:
                axd = fgr.make_axes(ax)
                s_arg = sel
            uin = torch.tensor(u0.astype(cdt), device="cuda")
            out = torch.zeros_like(uin)
            fgr.fgr_fggc_multistep_tensor(ctx.handle, axd, s_arg, fgr.make_packets(*fl), uin, out, 2)
            torch.cuda.synchronize()
            assert _gpu.rel_l2(out.cpu().numpy(), ref) <= tol, on_device
