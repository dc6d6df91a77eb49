"""Pins of the oracle's FGGC (Algorithm 2, eq. 2.23-2.25): on-grid exactness,
aggregation against the unaggregated sum, and the LSA errors of Example 1
(Table 6)."""

import math

import numpy as np
import pytest

from oracle import fga, fggc, lsa, trajectories as tr
from workloads import random_packets, mesh_for, wkb_packets
from workloads.wkb import _Family


def _grid(d, n, lo=-math.pi, hi=math.pi):
    return dict(d=d, n=[n] * d, lo=[lo] * d, hi=[hi] * d)


@pytest.mark.parametrize("d", [1, 2])
def test_fggc_of_on_grid_packets_is_the_direct_sum(d):
    # packets on mesh nodes are their own LSA (c = e_k0): FGGC == direct
    eps = 1 / 64
    mesh = mesh_for(d, eps)
    pk = random_packets(31, d, 50, q_range=(-2, 2), p_range=(-2, 2), mesh=mesh, on_node_fraction=1.0)
    grid = _grid(d, 128 if d == 1 else 40)
    strat = lsa.Strategy(nq=4, np_=2)
    ud = fga.direct_sum(pk, grid, eps, mesh.dq, mesh.dp)
    uf = fggc.reconstruct(pk, grid, eps, mesh.dq, mesh.dp, strat)
    # FP64 floor of the LSA: eps_mach / sqrt(lambda_min(A~)) (about 9e-12 for Q4P2)
    floor = np.finfo(float).eps / math.sqrt(strat.pinv.singular_values[-1])
    assert np.linalg.norm(uf - ud) <= max(1e-12, 2 * floor) * np.linalg.norm(ud)


def test_aggregation_equals_unaggregated_expansion():
    # eq. 2.24-2.25 (grouped by node) == eq. 2.23 (each packet's own expansion)
    eps = 1 / 256
    mesh = mesh_for(1, eps)
    pk = random_packets(32, 1, 30, q_range=(-0.3, 0.3), p_range=(-1, 1), mesh=mesh)
    grid = _grid(1, 200, -1.0, 1.0)
    strat = lsa.Strategy(nq=4, np_=2)
    a0, b0, c = lsa.coefficients(pk, mesh.dq, mesh.dp, strat)
    expanded = {"q": [], "p": [], "a": []}
    A = pk["a"][0] + 1j * pk["a"][1]
    for j in range(30):
        for k in range(strat.n1):
            expanded["q"].append((a0[0, j] + strat.shifts[k, 0]) * mesh.dq)
            expanded["p"].append((b0[0, j] + strat.shifts[k, 1]) * mesh.dp)
            expanded["a"].append(A[j] * np.exp(1j * pk["s"][j] / eps) * c[0, j, k])
    e = {"q": np.array([expanded["q"]]), "p": np.array([expanded["p"]]),
         "s": np.zeros(len(expanded["a"])),
         "a": np.stack([np.real(expanded["a"]), np.imag(expanded["a"])])}
    u1 = fga.direct_sum(e, grid, eps, mesh.dq, mesh.dp)
    u2 = fggc.reconstruct(pk, grid, eps, mesh.dq, mesh.dp, strat)
    assert np.linalg.norm(u1 - u2) <= 1e-13 * np.linalg.norm(u1)
    nodes_a, nodes_b, W = fggc.aggregate(pk, eps, mesh.dq, mesh.dp, strat)
    assert nodes_a.shape[1] < 30 * strat.n1          # shared nodes were merged


def test_fggc_approximates_each_packet_within_m_lsa():
    # one packet: ||u_fggc - u_direct|| / ||u_direct|| <= M_LSA (no cancellation)
    eps = 1 / 1024
    mesh = mesh_for(1, eps)
    for nq, np_ in [(2, 2), (4, 2)]:
        strat = lsa.Strategy(nq=nq, np_=np_)
        bound = lsa.m_lsa(strat, n_scan=21)
        pk = random_packets(33, 1, 1, q_range=(0.1, 0.2), p_range=(0.5, 0.6), mesh=mesh)
        grid = _grid(1, 4096, -0.5, 0.8)
        ud = fga.direct_sum(pk, grid, eps, mesh.dq, mesh.dp)
        uf = fggc.reconstruct(pk, grid, eps, mesh.dq, mesh.dp, strat)
        assert np.linalg.norm(uf - ud) / np.linalg.norm(ud) <= 1.05 * bound


class _Example1(_Family):
    """Example 1: u0 = (64/pi)^{1/4} exp(-32 x^2 + i x / eps)."""

    def sqrt_n0(self, l, y):
        return (64 / math.pi) ** 0.25 * np.exp(-32 * np.asarray(y) ** 2)

    def s0(self, l, y):
        return np.asarray(y, dtype=float).copy()

    def ds0(self, l, y):
        return np.ones_like(np.asarray(y, dtype=float))


def test_example1_lsa_error_table6():
    # Example 1 (V = 1 - cos(pi x), [-2, 2], T = 0.8, dx = eps, RK4 dt = 1e-4) at
    # eps = 2^-6: Table 6 prints the FGGC-vs-FGA error 1.135E-04 for Q2P2 and
    # 9.788E-07 / 9.295E-08 for Q4P2 / Q4P4.  The Q2P2 value is reproduced to 2%;
    # for the ill-conditioned strategies the printed values carry the rounding
    # of the paper's solve and bound the oracle's from above.  (The p-mesh
    # extent is not given: +-10 sqrt(eps) around grad S0.)
    eps = 2.0 ** -6
    sig = math.sqrt(eps)
    nq = int(round(4 / (sig / 2)))
    np_ = 2 * int(math.ceil(10 / (math.pi / 8)))
    pk = wkb_packets(1, eps, nq, np_, _Example1())
    mesh = pk["mesh"]
    grid = dict(d=1, n=[int(round(4 / eps))], lo=[-2.0], hi=[2.0])
    pt = tr.propagate(pk, {"kind": "cossum", "c0": 1.0, "amp": -1.0, "k": math.pi}, 0.8, 1e-4)
    ud = fga.direct_sum(pt, grid, eps, mesh.dq, mesh.dp)
    err = {}
    for name, nqq, npp in [("Q2P2", 2, 2), ("Q4P2", 4, 2), ("Q2P4", 2, 4), ("Q4P4", 4, 4)]:
        uf = fggc.reconstruct(pt, grid, eps, mesh.dq, mesh.dp, lsa.Strategy(nq=nqq, np_=npp))
        err[name] = np.linalg.norm(uf - ud) / np.linalg.norm(ud)
    assert abs(err["Q2P2"] / 1.135e-4 - 1) <= 0.02
    assert err["Q4P2"] <= 9.788e-7 and err["Q2P4"] <= 9.788e-7
    assert err["Q4P4"] <= 9.295e-8
