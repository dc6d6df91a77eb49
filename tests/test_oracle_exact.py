"""Pins of the exact harmonic-oscillator Gaussian (oracle/exact.py): it is the
initial datum at t = 0, keeps its norm, returns to -u0 after one period in one
dimension (the Maslov sign of the caustics at t = pi/2 and 3 pi/2), solves the
equation i eps u_t = -eps^2/2 u_xx + x^2/2 u (finite-difference residual), and
its centre moves along the classical flow."""

import math

import numpy as np

from oracle import exact

EPS = 1 / 64
BETA, X0, P0 = 32.0, 0.3, 1.0


def _grid(n=4096, lo=-4.0, hi=4.0):
    h = (hi - lo) / n
    return lo + np.arange(n) * h, h


def _u0(x):
    return np.exp(-BETA * (x - X0) ** 2 + 1j * P0 * (x - X0) / EPS)


def test_initial_datum():
    x, _ = _grid()
    u = exact.harmonic_gaussian_1d(x, 0.0, EPS, BETA, X0, P0)
    assert np.max(np.abs(u - _u0(x))) <= 1e-13


def test_norm_is_conserved():
    x, h = _grid()
    n0 = math.sqrt(h) * np.linalg.norm(_u0(x))
    for t in (0.3, 0.8, 1.6, 2.9, 4.0):
        u = exact.harmonic_gaussian_1d(x, t, EPS, BETA, X0, P0)
        assert abs(math.sqrt(h) * np.linalg.norm(u) / n0 - 1) <= 1e-12


def test_full_period_gives_minus_u0():
    x, _ = _grid()
    u = exact.harmonic_gaussian_1d(x, 2 * math.pi, EPS, BETA, X0, P0)
    assert np.max(np.abs(u + _u0(x))) <= 1e-9
    half = exact.harmonic_gaussian_1d(x, math.pi, EPS, BETA, X0, P0)
    # half a period: -i u0(-x)
    assert np.max(np.abs(half - (-1j) * _u0(-x))) <= 1e-9


def test_solves_the_equation():
    # central differences in t and x on a fine grid; the residual relative to
    # the size of the terms is O(dt^2 + h^2)
    x, h = _grid(8192, -2.0, 2.0)
    t, dt = 0.8, 1e-6
    up = exact.harmonic_gaussian_1d(x, t + dt, EPS, BETA, X0, P0)
    um = exact.harmonic_gaussian_1d(x, t - dt, EPS, BETA, X0, P0)
    u = exact.harmonic_gaussian_1d(x, t, EPS, BETA, X0, P0)
    ut = (up - um) / (2 * dt)
    uxx = (np.roll(u, -1) - 2 * u + np.roll(u, 1)) / h ** 2
    lhs = 1j * EPS * ut
    rhs = -0.5 * EPS ** 2 * uxx + 0.5 * x ** 2 * u
    inner = slice(10, -10)
    scale = np.max(np.abs(0.5 * x[inner] ** 2 * u[inner]))
    assert np.max(np.abs(lhs[inner] - rhs[inner])) <= 1e-4 * scale
    # a sign error in S, alpha or the branch breaks it by O(1)
    bad = exact.harmonic_gaussian_1d(x, t, EPS, BETA, X0, -P0)
    assert np.max(np.abs(bad - u)) > 0.1


def test_centre_follows_the_classical_flow():
    x, h = _grid()
    t = 1.1
    u = exact.harmonic_gaussian_1d(x, t, EPS, BETA, X0, P0)
    w = np.abs(u) ** 2
    mean = np.sum(x * w) / np.sum(w)
    assert abs(mean - (X0 * math.cos(t) + P0 * math.sin(t))) <= 1e-10


def test_tensor_product():
    x, h = _grid(256)
    y, _ = _grid(200, -3.0, 3.0)
    u = exact.harmonic_gaussian([x, y], 0.7, EPS, BETA, [X0, -0.2], [P0, 0.5], 2.0)
    ux = exact.harmonic_gaussian_1d(x, 0.7, EPS, BETA, X0, P0)
    uy = exact.harmonic_gaussian_1d(y, 0.7, EPS, BETA, -0.2, 0.5)
    assert np.max(np.abs(u - 2.0 * np.outer(ux, uy))) <= 1e-14
    assert exact.l2_error(u, u, [h, h]) == 0.0
