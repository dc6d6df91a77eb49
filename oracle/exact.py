"""Exact solution of the semi-classical Schroedinger equation with the
harmonic potential V = |x|^2 / 2 for Gaussian initial data (FP64).

Test infrastructure only (see the package docstring).

Examples 4 and 5 of Sec. 4.4 with the potential V_2 start from
u0 = N0 prod_l exp(-beta (x_l - x0_l)^2 + i p0_l (x_l - x0_l) / eps).  For a
quadratic Hamiltonian a Gaussian stays Gaussian: with the classical flow
q(t) = q0 cos t + p0 sin t, p(t) = p0 cos t - q0 sin t, per dimension

    u_l(x, t) = z(t)^{-1/2} exp((i/eps) [alpha(t)/2 (x - q)^2 + p (x - q) + S(t)]),
    alpha(0) = 2 i beta eps,  z(t) = cos t + alpha(0) sin t,
    alpha(t) = (alpha(0) cos t - sin t) / z(t),
    S(t) = (p0^2 - q0^2) sin(2t) / 4 - q0 p0 sin(t)^2,

which solves the eikonal equation phi_t + phi_x^2 / 2 + x^2 / 2 = 0 exactly
(alpha' = -1 - alpha^2, S' = p^2/2 - q^2/2) and the transport equation
A' = -(alpha/2) A, whose solution is z^{-1/2} on the branch that is 1 at
t = 0 and follows z continuously (z turns about the origin once per period).
The product over dimensions times N0 is the solution.  This is the reference
against which the tests measure the errors of FGA and of multi-step FGGC for
V_2 (the paper measures them against a time-splitting spectral solution,
which for this potential converges to the same function).
"""

from __future__ import annotations

import math

import numpy as np


def _z_inv_sqrt(t: float, b: float) -> complex:
    """z(t)^{-1/2} for z = cos t + i b sin t (b > 0) on the continuous branch."""
    k = round(t / math.pi)  # t - k pi in [-pi/2, pi/2]
    arg = math.atan(b * math.tan(t - k * math.pi)) + k * math.pi
    mod = math.hypot(math.cos(t), b * math.sin(t))
    return mod ** -0.5 * complex(math.cos(-arg / 2), math.sin(-arg / 2))


def harmonic_gaussian_1d(x, t: float, eps: float, beta: float, x0: float, p0: float) -> np.ndarray:
    """u_l(x, t) of one dimension (without N0), unit-mass harmonic potential."""
    x = np.asarray(x, dtype=np.float64)
    c, s = math.cos(t), math.sin(t)
    a0 = 2j * beta * eps
    z = c + a0 * s
    alpha = (a0 * c - s) / z
    q = x0 * c + p0 * s
    p = p0 * c - x0 * s
    S = (p0 * p0 - x0 * x0) * math.sin(2 * t) / 4 - x0 * p0 * s * s
    d = x - q
    phase = alpha / 2 * d * d + p * d + S
    return _z_inv_sqrt(t, 2 * beta * eps) * np.exp(1j * phase / eps)


def harmonic_gaussian(axes, t: float, eps: float, beta: float, x0, p0, n0: float) -> np.ndarray:
    """n0 * prod_l u_l(x_l, t) on the tensor grid of the 1-D point arrays `axes`."""
    d = len(axes)
    out = np.array(n0, dtype=np.complex128)
    for l in range(d):
        f = harmonic_gaussian_1d(axes[l], t, eps, beta, float(x0[l]), float(p0[l]))
        out = np.multiply.outer(out, f) if out.ndim else out * f
    return out


def l2_error(u, v, h) -> float:
    """sqrt(prod h_l * sum |u - v|^2): the L2 error on the grid."""
    return float(math.sqrt(float(np.prod(h)) * float(np.sum(np.abs(np.asarray(u) - np.asarray(v)) ** 2))))
