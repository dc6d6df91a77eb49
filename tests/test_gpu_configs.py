"""The 2-D and 3-D workloads at their full sizes, in the launch configuration
the benchmark uses (device-resident packets, FP32, complex64 output).

Oracle inputs come from the oracle or from closed forms pinned against it:
* 2-D (V = 2 + cos x1 + cos x2, separable): the flow of each packet is the
  product of 1-D flows (tests/test_oracle_trajectories.py pins this), so the
  oracle integrates the 2 x 2048 distinct (q, p) pairs and assembles the
  4194304 packets from them.
* 3-D (V = |x|^2/2): the harmonic closed form of eq. 2.3-2.7 (pinned in
  tests/test_oracle_trajectories.py).
The oracle evaluates the direct sum at sampled grid points; FGGC is compared
with the GPU direct sum on the full grid and with the oracle's FGGC on a
packet subset.
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


def test_config4_full_size():
    w = config_workload(4)
    prop = _harmonic_flow(w["packets"], w["t"])
    rng = np.random.default_rng(3)
    _check_propagation(w, prop, rng.choice(prop["s"].size, size=20000, replace=False))
    _check_reconstruction(w, prop, n_points=48, subset=4000)
