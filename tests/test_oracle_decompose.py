"""Pins of the oracle's initial decomposition (eq. 2.6 / 2.8) on the grid.

* A Gaussian packet as the wave: its decomposition is 2^{d/2} times the closed
  form of eq. 2.15 (itself pinned against quadrature in test_oracle_fga.py).
* Proposition 1: decomposing u0 on the phase-space mesh and summing the
  packets back (eq. 2.10 at t = 0) returns u0.
* The decomposition agrees with the cut-off FFT of the input generator
  (Remark 1), an independent evaluation of the same integral.
* Packets whose window misses the grid get zero amplitude.
"""

import numpy as np

from oracle import decompose, fga
from workloads import WKB_TANH, wkb_packets


def _grid(d, n, lo, hi):
    ns = n if isinstance(n, (list, tuple)) else [n] * d
    return dict(d=d, n=list(ns), lo=[lo] * d, hi=[hi] * d)


def test_gaussian_wave_gives_the_closed_form_1d_2d():
    rng = np.random.default_rng(3)
    for d, n in ((1, 2048), (2, 256)):
        eps = 1 / 64
        grid = _grid(d, n, -3.0, 3.0)   # h = 6/n, at most sigma / 5
        q0, p0 = rng.uniform(-0.5, 0.5, d), rng.uniform(-1, 1, d)
        X = np.meshgrid(*[fga.grid_axis(grid, l) for l in range(d)], indexing="ij")
        u = fga.gaussian_packet(np.stack([x.ravel() for x in X]), q0, p0, eps).reshape(X[0].shape)
        q = q0[:, None] + rng.uniform(-0.3, 0.3, (d, 20))
        p = p0[:, None] + rng.uniform(-0.5, 0.5, (d, 20))
        a = decompose.decompose(u, grid, q, p, eps, R=12.0)
        got = a[0] + 1j * a[1]
        ref = 2 ** (d / 2) * fga.inner_product(q0[None, :], p0[None, :], q.T, p.T, eps)
        assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref)), d


def test_proposition1_round_trip_and_the_generator():
    eps = 1 / 64
    pk = wkb_packets(1, eps, 64, 96, WKB_TANH)
    mesh = pk["mesh"]
    fine = _grid(1, 4096, -4.0, 4.0)   # u0 sampled finely enough for the quadrature
    u0 = WKB_TANH.u0(fga.grid_axis(fine, 0)[None, :], eps)
    a = decompose.decompose(u0, fine, pk["q"], pk["p"], eps, R=10.0)
    # against the cut-off FFT of the generator
    ag, ao = pk["a"][0] + 1j * pk["a"][1], a[0] + 1j * a[1]
    assert np.max(np.abs(ao - ag)) <= 1e-12 * np.max(np.abs(ag))
    # eq. 2.9 / 2.10: the packets sum back to u0
    rec = dict(pk, a=a)
    grid = _grid(1, 256, -1.0, 1.0)
    u = fga.direct_sum(rec, grid, eps, mesh.dq, mesh.dp, R=8)
    ref = WKB_TANH.u0(fga.grid_axis(grid, 0)[None, :], eps)
    assert np.linalg.norm(u - ref) / np.linalg.norm(ref) <= 1e-6


def test_windows_off_the_grid_give_zero():
    grid = _grid(1, 128, -1.0, 1.0)
    u = np.ones(128, dtype=complex)
    a = decompose.decompose(u, grid, np.array([[5.0, -7.0]]), np.array([[0.0, 1.0]]), 1 / 64)
    assert np.all(a == 0)
