"""Least-squares approximation (LSA) of a packet by on-grid neighbours (FP64).

Test infrastructure only (see the package docstring).

Sec. 2.2-3.2 of the paper.  All functions here are per dimension unless stated:
with a tensor-product neighbour set the d-dimensional Gram matrix and
right-hand side are Kronecker products of the 1-D ones (the exponent of
eq. 3.22 / 3.23 is a sum over dimensions), so the d-dimensional coefficients
are products of 1-D coefficients.  ``coefficients_alg1`` solves the full
d-dimensional problem without that factorisation, as a cross-check.

Readings of the paper used here:
* Neighbour strategy QmPn (Sec. 3.1): tensor set of m q-shifts and n p-shifts;
  2 shifts = {0, 1}, 4 shifts = {-1, 0, 1, 2} (the nearest integers to a point
  of [0, 1)).  The 1-D neighbour index is k = iq*np + ip.  Figure 3.2 is not
  available; under Def. 1 and eq. 3.22 the values printed in Table 2 belong to
  2 q-shifts x 4 p-shifts and those of Table 3 to 4 q-shifts x 2 p-shifts, so the
  two captions are read as swapped.
* Conjugation: eq. 2.14 defines <g,h> = int g h^dagger, and eq. 2.13 builds the
  normal equations from it, which gives the complex conjugate of the true L2
  normal equations sum_k (int psi_j^* psi_k) c_k = int psi_j^* phi.  The oracle
  solves the true L2 least-squares problem, i.e. the coefficients are the
  complex conjugate of the solution of the system as printed.
* Shift back (eq. 3.13): with that conjugation the true coefficients are
  c_k = conj(c~_k) * exp(-(i/eps)(Q - Q^(k)).int P)
      = conj(c~_k) * exp(-i cq cp (s - dq_k) b0)  per dimension.
* Pseudo-inverse (Remark 2): by the SVD A = U S V^H, singular values below
  rcond * s_max dropped (rcond = 1e-14; the paper gives no cut-off).  It is
  applied in factored form, V (S^+ (U^H f)), which keeps the rounding of the
  per-packet products near the conditioning limit; multiplying by the formed
  matrix A^+ adds rounding of order eps_mach * |A^+| (about 1e-7 of the packet
  norm for Q4P2 at the recommended mesh).
* floor() is the true floor in FP64 on Q/dq and P/dp (one FP64 division each).
"""

from __future__ import annotations

import math

import numpy as np

SHIFTS = {2: (0, 1), 4: (-1, 0, 1, 2)}


def shift_pairs(nq: int, np_: int) -> np.ndarray:
    """1-D neighbour shifts (dq_k, dp_k), k = iq*np + ip, as an (n1, 2) float array."""
    return np.array([(a, b) for a in SHIFTS[nq] for b in SHIFTS[np_]], dtype=np.float64)


def int_frac(x, step: float):
    """floor(x/step) and x/step - floor(x/step) (eq. 3.6-3.7 in units of the step)."""
    r = np.asarray(x, dtype=np.float64) / step
    i = np.floor(r)
    return i.astype(np.int64), r - i


def gram_eps_free(cq: float, cp: float, nq: int, np_: int) -> np.ndarray:
    """A~_jk of eq. 3.22 (paper convention), 1-D, shape (n1, n1)."""
    sh = shift_pairs(nq, np_)
    dqj, dpj = sh[:, 0][:, None], sh[:, 1][:, None]
    dqk, dpk = sh[:, 0][None, :], sh[:, 1][None, :]
    return np.exp(-cq * cq / 4 * (dqj - dqk) ** 2 - cp * cp / 4 * (dpj - dpk) ** 2
                  + 1j * cq * cp / 2 * (dqk - dqj) * (dpj + dpk))


def rhs_eps_free(cq: float, cp: float, nq: int, np_: int, s, t) -> np.ndarray:
    """f~_j of eq. 3.23 (paper convention) for fractional parts s, t; shape (..., n1)."""
    sh = shift_pairs(nq, np_)
    s = np.asarray(s, dtype=np.float64)[..., None]
    t = np.asarray(t, dtype=np.float64)[..., None]
    dq, dp = sh[:, 0], sh[:, 1]
    return np.exp(-cq * cq / 4 * (dq - s) ** 2 - cp * cp / 4 * (dp - t) ** 2
                  + 1j * cq * cp / 2 * (s - dq) * (dp + t))


class PseudoInverse:
    """A^+ by the SVD (Remark 2), kept as its factors."""

    def __init__(self, A: np.ndarray, rcond: float = 1e-14):
        U, S, Vh = np.linalg.svd(A)
        keep = S > rcond * S[0]
        self.U = U[:, keep]
        self.S = S[keep]
        self.V = Vh[keep, :].conj().T
        self.singular_values = S
        self.rank = int(keep.sum())

    def apply(self, f: np.ndarray) -> np.ndarray:
        """A^+ f for f of shape (..., n): V (S^{-1} (U^H f))."""
        y = f @ self.U.conj()          # (U^H f) for each row vector
        return (y / self.S) @ self.V.T  # V (S^-1 y)

    def matrix(self) -> np.ndarray:
        return (self.V / self.S) @ self.U.conj().T


class Strategy:
    """Mesh constants and neighbour strategy, with the precomputed A~^+ (Alg. 2, Step 0)."""

    def __init__(self, cq: float = 0.5, cp: float = math.pi / 8, nq: int = 4, np_: int = 2,
                 rcond: float = 1e-14):
        self.cq, self.cp, self.nq, self.np_ = cq, cp, nq, np_
        self.shifts = shift_pairs(nq, np_)
        self.n1 = self.shifts.shape[0]
        self.gram = gram_eps_free(cq, cp, nq, np_)
        self.pinv = PseudoInverse(self.gram, rcond)


def coefficients_1d(Q, P, dq: float, dp: float, strat: Strategy):
    """Algorithm 2, Step 3, one dimension: anchors and true LSA coefficients.

    Q, P: arrays of shape (M,).  Returns a0 (M,), b0 (M,) int64 and c (M, n1)
    complex with G(x;Q,P) ~= sum_k c_k G(x; (a0+dq_k) dq, (b0+dp_k) dp).
    """
    a0, s = int_frac(Q, dq)
    b0, t = int_frac(P, dp)
    f = rhs_eps_free(strat.cq, strat.cp, strat.nq, strat.np_, s, t)
    c_tilde_paper = strat.pinv.apply(f)                      # c~ = A~^+ f~
    c_tilde = np.conj(c_tilde_paper)                         # true L2 solution
    dqk = strat.shifts[:, 0][None, :]
    shift = np.exp(-1j * strat.cq * strat.cp * (s[:, None] - dqk) * b0[:, None].astype(np.float64))
    return a0, b0, c_tilde * shift


def coefficients(packets: dict, dq: float, dp: float, strat: Strategy):
    """d-dimensional coefficients as per-dimension factors.

    Returns a0 (d,M), b0 (d,M) and c (d,M,n1); the coefficient of the
    neighbour (k_1..k_d) is prod_l c[l, j, k_l].
    """
    d = packets["q"].shape[0]
    out = [coefficients_1d(packets["q"][l], packets["p"][l], dq, dp, strat) for l in range(d)]
    a0 = np.stack([o[0] for o in out])
    b0 = np.stack([o[1] for o in out])
    c = np.stack([o[2] for o in out])
    return a0, b0, c


def coefficients_alg1(Q, P, eps: float, dq: float, dp: float, strat: Strategy, rcond=1e-14):
    """Algorithm 1, Step 3 for one packet in d dimensions, without any shift or
    factorisation: neighbours by Def. 1 (tensor set), Gram and right-hand side
    from the closed-form inner product eq. 2.15 at the actual eps, true L2
    convention, minimum-norm solution by the SVD pseudo-inverse.

    Returns (neighbour centres Qn (n,d), Pn (n,d), coefficients c (n,)),
    neighbours ordered row-major over (k_1..k_d).
    """
    from .fga import inner_product
    Q = np.asarray(Q, float)
    P = np.asarray(P, float)
    d = Q.shape[0]
    intQ = np.floor(Q / dq)
    intP = np.floor(P / dp)
    sh = strat.shifts
    n1 = sh.shape[0]
    combos = np.array(np.unravel_index(np.arange(n1 ** d), (n1,) * d)).T  # (n, d)
    Qn = (intQ[None, :] + sh[combos, 0]) * dq
    Pn = (intP[None, :] + sh[combos, 1]) * dp
    # paper convention <psi_j, psi_k>, <psi_j, phi>; true normal equations use conj
    Gpaper = inner_product(Qn[:, None, :], Pn[:, None, :], Qn[None, :, :], Pn[None, :, :], eps)
    fpaper = inner_product(Qn, Pn, Q[None, :], P[None, :], eps)
    Mtrue = np.conj(Gpaper)
    btrue = np.conj(fpaper)
    c = PseudoInverse(Mtrue, rcond).apply(btrue)
    return Qn, Pn, c


def e_lsa(s, t, strat: Strategy):
    """Relative LSA error E_LSA (eq. 3.4) at fractional position (s, t), 1-D.

    With the eps-free Gram (unit diagonal), E^2 = 1 - f^H A^+ f; evaluated as
    1 - sum_i |u_i^H f|^2 / s_i from the SVD of the Hermitian Gram.
    """
    f = rhs_eps_free(strat.cq, strat.cp, strat.nq, strat.np_, s, t)
    y = f @ strat.pinv.U.conj()
    e2 = 1.0 - np.sum(np.abs(y) ** 2 / strat.pinv.S, axis=-1)
    return np.sqrt(np.maximum(e2, 0.0))


def e_lsa_quadrature(s, t, strat: Strategy, coeff=None, half_width=14.0, npts=6001):
    """E_LSA (eq. 3.4) by trapezoid quadrature in eps-free units (eps = 1).

    With coeff=None the coefficients are the least-squares optimum of the
    sampled problem (numpy lstsq); otherwise the given true coefficients c_k of
    the neighbours (dq_k cq, dp_k cp).  Independent of eq. 3.22 / 3.23.
    """
    cq, cp = strat.cq, strat.cp
    y = np.linspace(-half_width, half_width + 2 * cq, npts)
    w = y[1] - y[0]

    def G(Q, P):
        return np.exp(1j * P * (y - Q) - (y - Q) ** 2 / 2)

    psi = np.stack([G(a * cq, b * cp) for a, b in strat.shifts], 1) * math.sqrt(w)
    phi = G(cq * s, cp * t) * math.sqrt(w)
    if coeff is None:
        coeff, *_ = np.linalg.lstsq(psi, phi, rcond=None)
    r = phi - psi @ coeff
    return float(np.linalg.norm(r) / np.linalg.norm(phi))


def m_lsa(strat: Strategy, n_scan: int = 41, refine: bool = True) -> float:
    """M_LSA of eq. 3.25: sup of E_LSA over the unit cell [0,1]^2 (1-D).

    Grid scan of n_scan^2 points, then a bounded local maximisation from the
    best few scan points.
    """
    g = np.linspace(0.0, 1.0, n_scan)
    S, T = np.meshgrid(g, g, indexing="ij")
    E = e_lsa(S, T, strat)
    best = float(E.max())
    if refine:
        from scipy.optimize import minimize
        flat = np.argsort(E.ravel())[::-1][:6]
        for idx in flat:
            x0 = np.array([S.ravel()[idx], T.ravel()[idx]])
            r = minimize(lambda z: -float(e_lsa(z[0], z[1], strat)), x0,
                         bounds=[(0.0, 1.0), (0.0, 1.0)], method="L-BFGS-B")
            best = max(best, -float(r.fun))
    return best


def e_h1(s, t, strat: Strategy, eps: float, npts: int = 8001) -> float:
    """The H1 error ratio of Remark 5 (eq. 3.add8), 1-D, at (Q, P) = (s dq, t dp):
    ||d/dx (G - sum_k c_k G_k)||_L2 / ||G||_H1 with the LSA coefficients c_k of
    coefficients_1d (the L2 optimum), by trapezoid quadrature of the definition
    at the given eps (||G||_H1^2 = ||G||^2 + ||G'||^2)."""
    sig = math.sqrt(eps)
    dq, dp = strat.cq * sig, strat.cp * sig
    Q, P = s * dq, t * dp
    a0, b0, c = coefficients_1d(np.array([Q]), np.array([P]), dq, dp, strat)
    x = np.linspace(Q - 14 * sig - 2 * dq, Q + 14 * sig + 3 * dq, npts)
    w = x[1] - x[0]

    def G(Qc, Pc):
        return np.exp(1j * Pc * (x - Qc) / eps - (x - Qc) ** 2 / (2 * eps))

    def dG(Qc, Pc):  # d/dx of G(x; Qc, Pc)
        return (1j * Pc - (x - Qc)) / eps * G(Qc, Pc)

    r = dG(Q, P)
    for k, (da, db) in enumerate(strat.shifts):
        r = r - c[0, k] * dG((a0[0] + da) * dq, (b0[0] + db) * dp)
    h1 = math.sqrt(w * (np.sum(np.abs(G(Q, P)) ** 2) + np.sum(np.abs(dG(Q, P)) ** 2)))
    return math.sqrt(w * np.sum(np.abs(r) ** 2)) / h1


def m_lsa_h1(strat: Strategy, eps: float, n_scan: int = 11, refine: bool = True) -> float:
    """sup of e_h1 over the cell (Q, P) in [0, dq] x [0, dp] (eq. 3.add8): grid
    scan, then a bounded local maximisation from the best scan points."""
    g = np.linspace(0.0, 1.0, n_scan)
    vals = np.array([[e_h1(a, b, strat, eps) for b in g] for a in g])
    best = float(vals.max())
    if refine:
        from scipy.optimize import minimize
        for idx in np.argsort(vals.ravel())[::-1][:3]:
            i, j = np.unravel_index(idx, vals.shape)
            r = minimize(lambda z: -e_h1(z[0], z[1], strat, eps), np.array([g[i], g[j]]),
                         bounds=[(0.0, 1.0), (0.0, 1.0)], method="L-BFGS-B")
            best = max(best, -float(r.fun))
    return best
