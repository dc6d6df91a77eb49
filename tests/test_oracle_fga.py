"""Pins of the oracle's direct sum (eq. 2.10) and of its normalisation
(Proposition 1), plus the input generator it is fed with."""

import math

import numpy as np
import pytest

from oracle import fga
from workloads import WKB_TANH, WKB_LINEAR, random_packets, mesh_for, wkb_packets


def _grid(d, n, lo=-math.pi, hi=math.pi):
    return dict(d=d, n=[n] * d, lo=[lo] * d, hi=[hi] * d)


@pytest.mark.parametrize("d,n,m", [(1, 300, 40), (2, 48, 30)])
def test_window_truncation_within_its_bound(d, n, m):
    # brute force (no window) vs R-window: difference bounded by
    # pref * sum|A| * exp(-R^2/2) (every dropped term has |x-Q| > R sqrt(eps))
    eps = 1 / 64
    mesh = mesh_for(d, eps)
    pk = random_packets(11, d, m, q_range=(-3.5, 3.5), p_range=(-2, 2), mesh=mesh)
    grid = _grid(d, n)
    for R in (3.0, 5.0):
        u_w = fga.direct_sum(pk, grid, eps, mesh.dq, mesh.dp, R=R)
        u_b = fga.direct_sum(pk, grid, eps, mesh.dq, mesh.dp, R=R, brute=True)
        pref = fga.prefactor(d, eps, mesh.dq, mesh.dp)
        bound = pref * np.sum(np.hypot(*pk["a"])) * math.exp(-R * R / 2)
        diff = np.max(np.abs(u_w - u_b))
        assert diff <= bound
        assert diff >= 1e-3 * bound  # the window really truncates something


def test_brute_sum_is_the_definition():
    # eq. 2.10 term by term for a handful of packets at a few points
    eps = 1 / 256
    mesh = mesh_for(1, eps)
    pk = random_packets(12, 1, 5, q_range=(-0.5, 0.5), mesh=mesh)
    grid = _grid(1, 64, -1.0, 1.0)
    u = fga.direct_sum(pk, grid, eps, mesh.dq, mesh.dp, brute=True)
    x = fga.grid_axis(grid, 0)
    pref = (mesh.dq * mesh.dp) / (2 * math.pi * eps) ** 1.5
    for i in (0, 17, 40, 63):
        ref = 0j
        for j in range(5):
            A = pk["a"][0, j] + 1j * pk["a"][1, j]
            ref += A * np.exp(1j / eps * (pk["s"][j] + pk["p"][0, j] * (x[i] - pk["q"][0, j]))
                              - (x[i] - pk["q"][0, j]) ** 2 / (2 * eps))
        assert abs(u[i] - pref * ref) <= 1e-13 * abs(pref) * 5


@pytest.mark.parametrize("d", [1, 2])
def test_sampled_points_equal_full_grid(d):
    eps = 1 / 64
    mesh = mesh_for(d, eps)
    pk = random_packets(13, d, 60, q_range=(-4, 4), mesh=mesh)
    grid = _grid(d, 40 if d == 2 else 257)
    u = fga.direct_sum(pk, grid, eps, mesh.dq, mesh.dp, R=6)
    rng = np.random.default_rng(0)
    pts = np.stack([rng.integers(0, grid["n"][l], 25) for l in range(d)])
    v = fga.direct_sum(pk, grid, eps, mesh.dq, mesh.dp, R=6, points=pts)
    assert np.max(np.abs(v - u[tuple(pts)])) <= 1e-13 * max(1.0, np.max(np.abs(u)))


def test_empty_and_out_of_grid_packets():
    eps = 1 / 64
    mesh = mesh_for(1, eps)
    grid = _grid(1, 128)
    empty = random_packets(14, 1, 0, mesh=mesh)
    assert np.all(fga.direct_sum(empty, grid, eps, mesh.dq, mesh.dp) == 0)
    far = random_packets(15, 1, 10, q_range=(50, 60), mesh=mesh)
    assert np.all(fga.direct_sum(far, grid, eps, mesh.dq, mesh.dp) == 0)


def test_proposition1_reconstructs_initial_data_1d():
    # eq. 2.9 with the discrete sum of eq. 2.10: packets of the initial
    # decomposition (A = 2^{d/2} u0hat) give back u0 on the grid.  A prefactor
    # with the extra 2^{d/2} of eq. 2.1 would be off by 41%.
    eps = 1 / 64
    pk = wkb_packets(1, eps, 64, 96, WKB_TANH)
    mesh = pk["mesh"]
    grid = _grid(1, 256, -1.0, 1.0)
    u = fga.direct_sum(pk, grid, eps, mesh.dq, mesh.dp, R=8)
    u0 = WKB_TANH.u0(fga.grid_axis(grid, 0)[None, :], eps)
    assert np.linalg.norm(u - u0) / np.linalg.norm(u0) <= 3e-4


def test_proposition1_reconstructs_initial_data_2d():
    # same in 2-D (fixes the d in (dq dp)^d / (2 pi eps)^{3d/2}); eps = 1/16 keeps
    # the mesh small: q in [-1,1)^2, p within 6 sqrt(eps) of grad S0 = (1, 1)
    eps = 1 / 16
    pk = wkb_packets(2, eps, 16, 32, WKB_LINEAR)
    mesh = pk["mesh"]
    grid = _grid(2, 32, -0.5, 0.5)
    rng = np.random.default_rng(4)
    pts = rng.integers(4, 28, size=(2, 12))
    u = fga.direct_sum(pk, grid, eps, mesh.dq, mesh.dp, R=8, points=pts)
    x = np.stack([fga.grid_axis(grid, l)[pts[l]] for l in range(2)])
    u0 = WKB_LINEAR.u0(x, eps)
    assert np.max(np.abs(u - u0)) <= 1e-4 * np.max(np.abs(u0))


def test_direct_sum_3d_is_the_definition():
    eps = 1 / 64
    mesh = mesh_for(3, eps)
    pk = random_packets(16, 3, 7, q_range=(-0.3, 0.3), mesh=mesh)
    grid = _grid(3, 12, -0.5, 0.5)
    u = fga.direct_sum(pk, grid, eps, mesh.dq, mesh.dp, R=8)
    ub = fga.direct_sum(pk, grid, eps, mesh.dq, mesh.dp, R=8, brute=True)
    assert np.max(np.abs(u - ub)) <= 1e-13 * np.max(np.abs(ub))
    X = np.stack(np.meshgrid(*[fga.grid_axis(grid, l) for l in range(3)], indexing="ij")).reshape(3, -1)
    ref = np.zeros(X.shape[1], dtype=complex)
    for j in range(7):
        A = pk["a"][0, j] + 1j * pk["a"][1, j]
        ref += A * np.exp(1j * pk["s"][j] / eps) * fga.gaussian_packet(X, pk["q"][:, j], pk["p"][:, j], eps)
    ref *= fga.prefactor(3, eps, mesh.dq, mesh.dp)
    assert np.max(np.abs(ub.reshape(-1) - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_direct_sum_tensor_equals_direct_sum_on_the_expanded_packets():
    # a random selection of a 3-D tensor product of per-dimension lists, with
    # per-dimension amplitudes and actions: the factorised evaluation equals the
    # plain sum over the expanded packets (a transposed operand, a dropped
    # action or a wrong window would not)
    from oracle.fga import direct_sum, direct_sum_tensor
    rng = np.random.default_rng(17)
    d, L, eps = 3, 7, 1 / 64
    axes = [(np.sort(rng.uniform(-0.6, 0.6, L)), rng.uniform(-1, 1, L)) for _ in range(d)]
    amps = [rng.standard_normal(L) + 1j * rng.standard_normal(L) for _ in range(d)]
    acts = [rng.uniform(-0.5, 0.5, L) for _ in range(d)]
    sel = np.sort(rng.choice(L ** d, size=200, replace=False))
    idx = np.stack(np.unravel_index(sel, (L,) * d))
    phase = np.exp(-0.7j)
    A = phase * np.prod([amps[l][idx[l]] for l in range(d)], axis=0)
    pk = {"q": np.stack([axes[l][0][idx[l]] for l in range(d)]), "p": np.stack([axes[l][1][idx[l]] for l in range(d)]),
          "s": np.sum([acts[l][idx[l]] for l in range(d)], axis=0), "a": np.stack([A.real, A.imag])}
    grid = dict(d=3, n=[24, 20, 28], lo=[-1.0] * 3, hi=[1.0] * 3)
    pts = np.stack([rng.integers(0, n, 60) for n in grid["n"]])
    dq, dp = 0.0625, 0.05
    ref = direct_sum(pk, grid, eps, dq, dp, R=6, points=pts)
    got = direct_sum_tensor(axes, amps, acts, sel, grid, eps, dq, dp, pts, R=6, phase=phase)
    assert np.count_nonzero(ref) > 30
    assert np.linalg.norm(got - ref) <= 1e-13 * np.linalg.norm(ref)
