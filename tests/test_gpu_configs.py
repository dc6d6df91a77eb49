"""The 2-D and 3-D workloads at their full sizes, in the launch configuration
the benchmark uses (device-resident packets, FP32, complex64 output).

Oracle inputs come from the oracle or from closed forms pinned against it:
* 2-D (V = 2 + cos x1 + cos x2, separable): the flow of each packet is the
  product of 1-D flows (tests/test_oracle_trajectories.py pins this), so the
  oracle integrates the 2 x 2048 distinct (q, p) pairs and assembles the
  4194304 packets from them.
* 3-D (V = |x|^2/2): the harmonic closed form of eq. 2.3-2.7 (pinned in
  tests/test_oracle_trajectories.py).
The oracle evaluates the direct sum at sampled grid points (3-D: 1024 points
in 4 x 4 boxes on tile edges, faces, corners and random places, each box over
the packets whose windows reach it); FGGC is compared with the GPU direct sum
on the full grid, with the oracle's direct sum at the points and with the
oracle's FGGC of a packet subset.
"""

import math

import numpy as np
import pytest

from oracle import fga, fggc, lsa, trajectories as tr
from workloads import config_workload

from . import _gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _separable_2d_flow(w):
    """Oracle propagation of the 2-D workload through its 1-D factors."""
    pk = w["packets"]
    nq, np_ = w["nq"], w["np_"]
    M = pk["s"].size
    j = np.arange(M)
    b2 = j % np_
    b1 = (j // np_) % np_
    a2 = (j // (np_ * np_)) % nq
    a1 = j // (np_ * np_ * nq)
    out = {"q": np.empty_like(pk["q"]), "p": np.empty_like(pk["p"]), "s": np.zeros(M)}
    fac = np.ones(M, dtype=complex)
    pot1 = {"kind": "cossum", "c0": 1.0, "amp": 1.0, "k": 1.0}
    for l, (aa, bb) in enumerate(((a1, b1), (a2, b2))):
        pair = aa * np_ + bb
        uniq, first = np.unique(pair, return_index=True)
        one = {"q": pk["q"][l:l + 1, first].copy(), "p": pk["p"][l:l + 1, first].copy(),
               "s": np.zeros(uniq.size), "a": np.stack([np.ones(uniq.size), np.zeros(uniq.size)])}
        f = tr.propagate(one, pot1, w["t"], w["dt"])
        pos = np.searchsorted(uniq, pair)
        out["q"][l] = f["q"][0, pos]
        out["p"][l] = f["p"][0, pos]
        out["s"] += f["s"][pos]
        fac *= (f["a"][0] + 1j * f["a"][1])[pos]
    A = (pk["a"][0] + 1j * pk["a"][1]) * fac
    out["a"] = np.stack([A.real, A.imag])
    return out


def _harmonic_flow(pk, t):
    q, p = pk["q"], pk["p"]
    c, s = math.cos(t), math.sin(t)
    S = np.sum((p ** 2 - q ** 2) * math.sin(2 * t) / 4 - q * p * s * s, axis=0)
    A = (pk["a"][0] + 1j * pk["a"][1]) * np.exp(-0.5j * q.shape[0] * t)
    return {"q": q * c + p * s, "p": -q * s + p * c, "s": S, "a": np.stack([A.real, A.imag])}


def _sample_points(grid, k, seed):
    rng = np.random.default_rng(seed)
    return np.stack([rng.integers(0, grid["n"][l], k) for l in range(grid["d"])])


def _check_propagation(w, ref, idx):
    got = _gpu.propagate(w["packets"], w["d"], w["potential"], w["t"], w["dt"])
    for k in ("q", "p"):
        assert np.max(np.abs(got[k][:, idx] - ref[k][:, idx])) <= 1e-12 * max(1.0, np.max(np.abs(ref[k])))
    assert np.max(np.abs(got["s"][idx] - ref["s"][idx])) <= 1e-12 * max(1.0, np.max(np.abs(ref["s"])))
    A = got["a"][0, idx] + 1j * got["a"][1, idx]
    Ar = ref["a"][0, idx] + 1j * ref["a"][1, idx]
    nz = np.abs(Ar) > 1e-250
    assert np.max(np.abs(A[nz] - Ar[nz]) / np.abs(Ar[nz])) <= 1e-11


def _check_reconstruction(w, prop, n_points, subset):
    grid, eps, mesh = w["grid"], w["eps"], w["mesh"]
    got_d = _gpu.reconstruct("direct", prop, grid, eps, _gpu.options("fp32"))
    got_f = _gpu.reconstruct("fggc", prop, grid, eps, _gpu.options("fp32"))
    pts = _sample_points(grid, n_points, 0)
    ref_d = fga.direct_sum(prop, grid, eps, mesh.dq, mesh.dp, R=6, points=pts)
    assert _gpu.rel_l2(got_d[tuple(pts)], ref_d) <= 1e-5
    # FGGC against the direct sum it replaces, on the full grid
    assert _gpu.rel_l2(got_f, got_d) <= 1e-5
    # FGGC against the oracle's FGGC on a packet subset
    rng = np.random.default_rng(1)
    sel = np.sort(rng.choice(prop["s"].size, size=subset, replace=False))
    sub = {k: np.ascontiguousarray(v[..., sel]) for k, v in prop.items() if k in "qpsa"}
    ref_f = fggc.reconstruct(sub, grid, eps, mesh.dq, mesh.dp, lsa.Strategy(nq=4, np_=2), R=6, points=pts)
    got_fs = _gpu.reconstruct("fggc", sub, grid, eps, _gpu.options("fp32"))
    assert _gpu.rel_l2(got_fs[tuple(pts)], ref_f) <= 1e-5


def test_config3_full_size():
    w = config_workload(3)
    prop = _separable_2d_flow(w)
    rng = np.random.default_rng(2)
    _check_propagation(w, prop, rng.choice(prop["s"].size, size=20000, replace=False))
    _check_reconstruction(w, prop, n_points=256, subset=20000)


def _boxes_3d(n, seed):
    """64 boxes of 4 x 4 points (fixed i0; i1, i2 consecutive) = 1024 points:
    the edges of the direct sum's 8 x 8 x 16 tiles and of the grid passes'
    32- and 128-point tiles where the wave lives (indices 88..208 of 256), the
    grid's first and last points, and random places in the wave."""
    rng = np.random.default_rng(seed)
    edges = [88, 95, 96, 111, 112, 127, 128, 143, 144, 159, 160, 175, 176, 191, 192, 207]
    out = []
    for k in range(64):
        if k < 44:
            i0 = edges[k % len(edges)]
            s1 = edges[(3 * k + 1) % len(edges)] - 2
            s2 = edges[(5 * k + 2) % len(edges)] - 2
        elif k < 48:  # faces and corners of the grid
            i0, s1, s2 = [(0, 0, 0), (n - 1, n - 4, n - 4), (128, 0, n - 4), (n - 1, 126, 126)][k - 44]
        else:
            i0, s1, s2 = (int(x) for x in rng.integers(90, 200, 3))
        out.append((i0, s1, s2))
    return out


def _box_points(box):
    i0, s1, s2 = box
    a, b = np.meshgrid(np.arange(s1, s1 + 4), np.arange(s2, s2 + 4), indexing="ij")
    return np.stack([np.full(16, i0), a.ravel(), b.ravel()])


def _windows(pk, grid, eps, R):
    """Per dimension the window bounds of every packet (fga.window_bounds)."""
    return [tuple(x.astype(np.int32) for x in fga.window_bounds(pk["q"][l], grid, l, eps, R))
            for l in range(grid["d"])]


def _box_subset(pk, win, box):
    """The packets (or on-grid cells) whose windows reach the box: the
    oracle's sum at the box's points over them equals its sum over all
    packets (the others contribute exact zeros)."""
    i0, s1, s2 = box
    keep = np.ones(pk["s"].size, dtype=bool)
    for (m_lo, m_hi), (lo_i, hi_i) in zip(win, ((i0, i0), (s1, s1 + 3), (s2, s2 + 3))):
        keep &= (m_lo <= hi_i) & (m_hi >= lo_i)
    return {k: np.ascontiguousarray(pk[k][..., keep]) for k in ("q", "p", "s", "a")}


def test_config4_full_size():
    w = config_workload(4)
    prop = _harmonic_flow(w["packets"], w["t"])
    rng = np.random.default_rng(3)
    _check_propagation(w, prop, rng.choice(prop["s"].size, size=20000, replace=False))
    grid, eps, mesh = w["grid"], w["eps"], w["mesh"]
    got_d = _gpu.reconstruct("direct", prop, grid, eps, _gpu.options("fp32"))
    got_f = _gpu.reconstruct("fggc", prop, grid, eps, _gpu.options("fp32"))
    # FGGC against the direct sum it replaces, on the full grid
    assert _gpu.rel_l2(got_f, got_d) <= 1e-5
    boxes = _boxes_3d(grid["n"][0], 4)
    pts = np.concatenate([_box_points(b) for b in boxes], axis=1)
    # the oracle's direct sum at 1024 points (tile edges, faces, corners, random)
    # the packets are the kept part of a tensor product of per-dimension (q, p)
    # lists and the harmonic flow acts on each dimension alone, so the oracle's
    # direct sum is evaluated in its factorised form (fga.direct_sum_tensor)
    from workloads import workload_axes
    from workloads.wkb import _FAMILIES, _amplitude_table_1d
    axes0, sel = workload_axes(w)
    t = w["t"]
    ct, st = math.cos(t), math.sin(t)
    axes, amps, acts = [], [], []
    for l, (q, p) in enumerate(axes0):
        _, _, al = _amplitude_table_1d(_FAMILIES[w["family"]], l, mesh, w["nq"], w["np_"])
        axes.append((q * ct + p * st, -q * st + p * ct))
        acts.append((p ** 2 - q ** 2) * math.sin(2 * t) / 4 - q * p * st * st)
        amps.append(al.ravel())
    ref_d = fga.direct_sum_tensor(axes, amps, acts, sel, grid, eps, mesh.dq, mesh.dp, pts, R=6,
                                  phase=np.exp(-0.5j * 3 * t))
    assert _gpu.rel_l2(got_d[tuple(pts)], ref_d) <= 1e-5
    assert _gpu.rel_l2(got_f[tuple(pts)], ref_d) <= 1e-5
    # the oracle's FGGC (Algorithm 2) of a 4000-packet subset at the same points
    sel = np.sort(rng.choice(prop["s"].size, size=4000, replace=False))
    sub = {k: np.ascontiguousarray(v[..., sel]) for k, v in prop.items() if k in "qpsa"}
    na, nb, W = fggc.aggregate(sub, eps, mesh.dq, mesh.dp, lsa.Strategy(nq=4, np_=2))
    cells = fggc.on_grid_packets(na, nb, W, mesh.dq, mesh.dp)
    cwin = _windows(cells, grid, eps, 6)
    ref_f = np.concatenate([fga.direct_sum(_box_subset(cells, cwin, b), grid, eps, mesh.dq, mesh.dp, R=6,
                                           points=_box_points(b)) for b in boxes])
    got_fs = _gpu.reconstruct("fggc", sub, grid, eps, _gpu.options("fp32"))
    assert _gpu.rel_l2(got_fs[tuple(pts)], ref_f) <= 1e-5
