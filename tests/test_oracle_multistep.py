"""Pins of the oracle's multi-step FGGC (Algorithm 3 with a fixed mesh and the
learned one-step flow) against the harmonic oscillator, whose Schroedinger
propagator is known in closed form: with V = x^2/2 the wave after half a period
(t = pi) is -i u0(-x) and after a full period (t = 2 pi) it is -u0 (d = 1).
Quarter-period steps exercise the decomposition (eq. 2.8), the learned flow
(eq. 2.3-2.6) and the FGGC reconstruction (eq. 2.24-2.25) in turn."""

import math

import numpy as np

from oracle import fga, fggc, lsa, trajectories as tr
from workloads import mesh_for


def _setup():
    eps = 1 / 64
    mesh = mesh_for(1, eps)
    qs = np.arange(-40, 40) * mesh.dq
    ps = np.arange(-80, 80) * mesh.dp
    Q, P = np.meshgrid(qs, ps, indexing="ij")
    M = Q.size
    grid_mesh = {"q": Q.reshape(1, -1), "p": P.reshape(1, -1), "s": np.zeros(M),
                 "a": np.stack([np.ones(M), np.zeros(M)])}
    flow = tr.propagate(grid_mesh, {"kind": "harmonic", "omega": 1.0}, math.pi / 2, 1e-3)
    grid = dict(d=1, n=[512], lo=[-4.0], hi=[4.0])
    x = fga.grid_axis(grid, 0)

    def u0(xx):
        return np.exp(-(xx - 0.5) ** 2 / (2 * 0.15)) * np.exp(1j * 0.7 * xx / eps)
    return eps, mesh, grid_mesh, flow, grid, x, u0


def test_harmonic_half_and_full_period():
    eps, mesh, grid_mesh, flow, grid, x, u0 = _setup()
    st = lsa.Strategy(nq=4, np_=2)
    half = fggc.multistep(u0(x), grid, grid_mesh, flow, eps, mesh.dq, mesh.dp, st, 2)
    full = fggc.multistep(u0(x), grid, grid_mesh, flow, eps, mesh.dq, mesh.dp, st, 4)
    norm = np.linalg.norm(u0(x))
    assert np.linalg.norm(half - (-1j) * u0(-x)) / norm <= 1e-5
    assert np.linalg.norm(full + u0(x)) / norm <= 1e-5


def test_one_step_is_the_plain_composition():
    from oracle import decompose
    eps, mesh, grid_mesh, flow, grid, x, u0 = _setup()
    st = lsa.Strategy(nq=2, np_=2)
    one = fggc.multistep(u0(x), grid, grid_mesh, flow, eps, mesh.dq, mesh.dp, st, 1)
    a0 = decompose.decompose(u0(x), grid, grid_mesh["q"], grid_mesh["p"], eps)
    moved = tr.propagate(dict(grid_mesh, a=a0), {"kind": "harmonic", "omega": 1.0}, math.pi / 2, 1e-3)
    ref = fggc.reconstruct(moved, grid, eps, mesh.dq, mesh.dp, st)
    assert np.linalg.norm(one - ref) <= 1e-12 * np.linalg.norm(ref)
