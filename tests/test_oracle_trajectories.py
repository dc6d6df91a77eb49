"""Pins of the oracle's RK4 integrator (eq. 2.3-2.7): closed forms for the free
particle and the harmonic oscillator, invariants for the cosine potential."""

import math

import numpy as np
import pytest

from oracle import trajectories as tr
from workloads import random_packets


def _packets(d, m, seed=21):
    return random_packets(seed, d, m, q_range=(-1.5, 1.5), p_range=(-2, 2), s_range=(0, 0))


@pytest.mark.parametrize("d", [1, 2, 3])
def test_free_particle_closed_form(d):
    # V = 0: Q = q + p t, P = p, S = |p|^2 t / 2, Z = (2 - i t) I, A = A0 (1 - i t/2)^{d/2}
    pk = _packets(d, 40)
    t = 0.7
    out = tr.propagate(pk, {"kind": "free"}, t, 1e-3)
    assert np.allclose(out["q"], pk["q"] + pk["p"] * t, rtol=0, atol=1e-13)
    assert np.array_equal(out["p"], pk["p"])
    assert np.allclose(out["s"], 0.5 * np.sum(pk["p"] ** 2, axis=0) * t, rtol=1e-13, atol=1e-14)
    A0 = pk["a"][0] + 1j * pk["a"][1]
    A = out["a"][0] + 1j * out["a"][1]
    ref = A0 * (1 - 0.5j * t) ** (d / 2)
    assert np.max(np.abs(A - ref) / np.abs(ref)) <= 1e-12


@pytest.mark.parametrize("d", [1, 2, 3])
@pytest.mark.parametrize("omega", [1.0, 2.5])
def test_harmonic_closed_form(d, omega):
    # V = w^2|x|^2/2: F = K = cos wt, G = sin(wt)/w, H = -w sin wt, so
    # Z/2 = (cos wt - i (w + 1/w)/2 sin wt) I and A = A0 (Z/2)^{d/2}
    # (= A0 e^{-i d w t/2} for w = 1)
    pk = _packets(d, 30)
    t = 0.5
    out = tr.propagate(pk, {"kind": "harmonic", "omega": omega}, t, 1e-4)
    q, p = pk["q"], pk["p"]
    c, s = math.cos(omega * t), math.sin(omega * t)
    assert np.max(np.abs(out["q"] - (q * c + p / omega * s))) <= 1e-12
    assert np.max(np.abs(out["p"] - (-q * omega * s + p * c))) <= 1e-12
    # S = int |P|^2/2 - w^2|Q|^2/2 dt
    S = np.sum((p ** 2 / omega - omega * q ** 2) * math.sin(2 * omega * t) / 4
               - q * p * s * s, axis=0)
    assert np.max(np.abs(out["s"] - S)) <= 1e-12
    A0 = pk["a"][0] + 1j * pk["a"][1]
    A = out["a"][0] + 1j * out["a"][1]
    z = c - 0.5j * (omega + 1 / omega) * s
    assert np.max(np.abs(A - A0 * z ** (d / 2)) / np.abs(A0)) <= 1e-12
    if omega == 1.0:
        assert np.max(np.abs(A - A0 * np.exp(-0.5j * d * t)) / np.abs(A0)) <= 1e-12


def test_cosine_potential_invariants_and_order():
    # V = 1 - cos x (d = 1): energy conservation, symplectic Jacobian,
    # A^2 / A0^2 = det Z / det Z(0), fourth-order convergence in dt.
    pot = {"kind": "cossum", "c0": 1.0, "amp": -1.0, "k": 1.0}
    pk = _packets(1, 25)
    t = 1.0
    out, jac = tr.propagate(pk, pot, t, 1e-3, with_jacobian=True)
    energy = lambda q, p: 0.5 * p ** 2 + 1.0 - np.cos(q)  # noqa: E731
    assert np.max(np.abs(energy(out["q"][0], out["p"][0]) - energy(pk["q"][0], pk["p"][0]))) <= 1e-12
    F, G, H, K = jac[:, 0, 0, 0], jac[:, 1, 0, 0], jac[:, 2, 0, 0], jac[:, 3, 0, 0]
    assert np.max(np.abs(F * K - G * H - 1.0)) <= 1e-12
    Z = F - 1j * G + 1j * H + K
    A0 = pk["a"][0] + 1j * pk["a"][1]
    A = out["a"][0] + 1j * out["a"][1]
    assert np.max(np.abs(A ** 2 / A0 ** 2 - Z / 2.0)) <= 1e-11
    # order 4: error(dt) / error(dt/2) ~ 16 against a fine reference
    ref = tr.propagate(pk, pot, t, 1e-3 / 8)
    e1 = np.max(np.abs(tr.propagate(pk, pot, t, 0.05)["s"] - ref["s"]))
    e2 = np.max(np.abs(tr.propagate(pk, pot, t, 0.025)["s"] - ref["s"]))
    assert 12 < e1 / e2 < 20


def test_cosine_potential_2d_matches_separable_1d():
    # V = 2 + cos x1 + cos x2 separates: Q, P of each dimension follow the 1-D flow,
    # and A = A0 * prod of the 1-D amplitude factors.
    pot2 = {"kind": "cossum", "c0": 2.0, "amp": 1.0, "k": 1.0}
    pot1 = {"kind": "cossum", "c0": 1.0, "amp": 1.0, "k": 1.0}
    pk = _packets(2, 12)
    out = tr.propagate(pk, pot2, 0.5, 1e-3)
    fac = np.ones(12, dtype=complex)
    for l in range(2):
        one = {"q": pk["q"][l:l + 1], "p": pk["p"][l:l + 1], "s": np.zeros(12),
               "a": np.stack([np.ones(12), np.zeros(12)])}
        o1 = tr.propagate(one, pot1, 0.5, 1e-3)
        assert np.max(np.abs(o1["q"][0] - out["q"][l])) <= 1e-13
        fac *= o1["a"][0] + 1j * o1["a"][1]
    A0 = pk["a"][0] + 1j * pk["a"][1]
    assert np.max(np.abs(out["a"][0] + 1j * out["a"][1] - A0 * fac)) <= 1e-12 * np.max(np.abs(A0))


def test_step_count_rule():
    assert tr.nsteps(0.5, 1e-4) == 5000
    assert tr.nsteps(1.0, 1e-4) == 10000
    assert tr.nsteps(0.3, 0.07) == 5
    assert tr.nsteps(0.0, 0.1) == 0
