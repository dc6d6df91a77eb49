"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle on
the same seeded inputs, at sizes the oracle finishes in seconds that still span
several tiles and a ragged tail, plus edge cases.

Tolerances (relative L2 over the output unless stated):
* FP64 direct sum: 1e-12.
* FP64 FGGC: max(1e-12, 4 eps_mach / sqrt(lambda_min(A~))): the least-squares
  solve cannot resolve the packet function better than eps_mach / sqrt(lambda_min)
  (about 9e-12 for Q4P2; 1.3e-14 for Q2P2), whichever implementation runs it.
* FP32 paths (complex64 output, FP32 bulk arithmetic): 1e-5 against the FP64 oracle.
* Trajectories: 1e-12 (relative for Q, P, A; absolute for S ~ O(1)).
"""

import math

import numpy as np
import pytest

from oracle import fga, fggc, lsa, trajectories as tr
from workloads import random_packets, mesh_for

from . import _gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2504_21785_gb300 as pkg
    pkg.fgr.load()


def _grid(d, n, lo=-math.pi, hi=math.pi):
    ns = n if isinstance(n, (list, tuple)) else [n] * d
    return dict(d=d, n=list(ns), lo=[lo] * d, hi=[hi] * d)


def _fp64_fggc_tol(nq, np_):
    strat = lsa.Strategy(nq=nq, np_=np_)
    floor = np.finfo(float).eps / math.sqrt(strat.pinv.singular_values[strat.pinv.rank - 1])
    return max(1e-12, 4 * floor)


POTS = {
    "free": {"kind": "free"},
    "cos": {"kind": "cossum", "c0": 1.0, "amp": -1.0, "k": 1.0},
    "harm": {"kind": "harmonic", "omega": 1.3},
}


# ---------------------------------------------------------------------------
# K1 propagate
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("d", [1, 2, 3])
@pytest.mark.parametrize("pot", sorted(POTS))
def test_propagate_matches_oracle(d, pot):
    # dt = 1e-4 as in the workloads: the library's closed-form amplitude and the
    # oracle's RK4-integrated one agree to O(dt^4)
    pk = random_packets(100 + d, d, 1000, q_range=(-2, 2), p_range=(-2, 2), s_range=(0, 0))
    ref = tr.propagate(pk, POTS[pot], 0.3, 1e-4)
    got = _gpu.propagate(pk, d, POTS[pot], 0.3, 1e-4)
    for k in ("q", "p"):
        assert np.max(np.abs(got[k] - ref[k])) <= 1e-12 * max(1.0, np.max(np.abs(ref[k])))
    assert np.max(np.abs(got["s"] - ref["s"])) <= 1e-12 * max(1.0, np.max(np.abs(ref["s"])))
    A, Ar = got["a"][0] + 1j * got["a"][1], ref["a"][0] + 1j * ref["a"][1]
    assert np.max(np.abs(A - Ar) / np.abs(Ar)) <= 1e-12


def test_propagate_large_steps():
    # dt * |P| up to 0.1 takes the direct sincos branch of the stage trigonometry;
    # Q, P, S are the same RK4 as the oracle's; A (closed form in det Z) differs
    # from an RK4-integrated A by O(dt^4)
    pk = random_packets(31, 1, 300, q_range=(-2, 2), p_range=(-2, 2), s_range=(0, 0))
    ref = tr.propagate(pk, POTS["cos"], 1.0, 0.05)
    got = _gpu.propagate(pk, 1, POTS["cos"], 1.0, 0.05)
    for k in ("q", "p", "s"):
        assert np.max(np.abs(got[k] - ref[k])) <= 1e-12 * max(1.0, np.max(np.abs(ref[k])))
    A, Ar = got["a"][0] + 1j * got["a"][1], ref["a"][0] + 1j * ref["a"][1]
    assert np.max(np.abs(A - Ar) / np.abs(Ar)) <= 1e-5


@pytest.mark.parametrize("dt,p_max", [(4e-3, 6.0), (1e-3, 25.0), (5e-4, 50.0)])
def test_propagate_stage_trigonometry_paths(dt, p_max):
    # the stage trigonometry of the cosine potential depends on k h |P|: short
    # series (|P| small), long series, sincos per stage (|P| large); stage 3
    # is rotated from stage 2 while k h^2 |amp k| / 4 <= 1e-6 (dt = 1e-3 and
    # 5e-4 yes, 4e-3 no) and the next step from stage 4 while k h^2 |amp k|
    # <= 1e-6 (5e-4 yes, 4e-3 no); every path must give the oracle's RK4 for
    # Q, P, S
    pk = random_packets(32, 1, 600, q_range=(-2, 2), p_range=(-p_max, p_max), s_range=(0, 0))
    ref = tr.propagate(pk, POTS["cos"], 0.5, dt)
    got = _gpu.propagate(pk, 1, POTS["cos"], 0.5, dt)
    for k in ("q", "p", "s"):
        assert np.max(np.abs(got[k] - ref[k])) <= 1e-12 * max(1.0, np.max(np.abs(ref[k])))
    A, Ar = got["a"][0] + 1j * got["a"][1], ref["a"][0] + 1j * ref["a"][1]
    assert np.max(np.abs(A - Ar) / np.abs(Ar)) <= 1e-7


def test_propagate_host_buffers_and_empty():
    pk = random_packets(7, 2, 257, s_range=(0, 0))
    ref = tr.propagate(pk, POTS["cos"], 0.2, 1e-4)
    got = _gpu.propagate(pk, 2, POTS["cos"], 0.2, 1e-4, on_device=False)
    assert np.max(np.abs(got["q"] - ref["q"])) <= 1e-12
    empty = random_packets(8, 1, 0)
    out = _gpu.propagate(empty, 1, POTS["cos"], 0.2, 1e-3)
    assert out["q"].shape == (1, 0)


def test_propagate_config1_full():
    from workloads import config_workload
    w = config_workload(1)
    ref = tr.propagate(w["packets"], w["potential"], w["t"], w["dt"])
    got = _gpu.propagate(w["packets"], 1, w["potential"], w["t"], w["dt"])
    A, Ar = got["a"][0] + 1j * got["a"][1], ref["a"][0] + 1j * ref["a"][1]
    nz = np.abs(Ar) > 0
    assert np.max(np.abs(got["q"] - ref["q"])) <= 1e-12 * np.max(np.abs(ref["q"]))
    assert np.max(np.abs(got["s"] - ref["s"])) <= 1e-12 * max(1.0, np.max(np.abs(ref["s"])))
    assert np.max(np.abs(A[nz] - Ar[nz]) / np.abs(Ar[nz])) <= 1e-12


# ---------------------------------------------------------------------------
# K2 direct sum
# ---------------------------------------------------------------------------

CASES = {
    # d, grid points, packets, eps: several tiles and a ragged tail each
    1: (1, 3001, 700, 1 / 256),
    2: (2, (70, 101), 300, 1 / 64),
    3: (3, (20, 17, 23), 60, 1 / 16),
}
# phase-space region of the random packets: a dense node box spans it, so the
# 3-D case stays compact (as the packets of a WKB problem are)
RANGES = {1: ((-3.6, 3.6), (-2.5, 2.5)), 2: ((-3.6, 3.6), (-2.5, 2.5)), 3: ((-1.2, 1.2), (-1.0, 1.0))}


def _case(d, seed=1):
    d, n, m, eps = CASES[d]
    mesh = mesh_for(d, eps)
    pk = random_packets(seed, d, m, q_range=RANGES[d][0], p_range=RANGES[d][1], s_range=(-3, 3),
                        mesh=mesh, on_node_fraction=0.1)
    return pk, _grid(d, n), eps, mesh


@pytest.mark.parametrize("d", [1, 2, 3])
def test_direct_fp64_matches_oracle(d):
    pk, grid, eps, mesh = _case(d)
    ref = fga.direct_sum(pk, grid, eps, mesh.dq, mesh.dp, R=8)
    got = _gpu.reconstruct("direct", pk, grid, eps, _gpu.options("fp64"))
    assert _gpu.rel_l2(got, ref) <= 1e-12


@pytest.mark.parametrize("d", [1, 2, 3])
def test_direct_fp32_matches_oracle(d):
    pk, grid, eps, mesh = _case(d, seed=2)
    ref = fga.direct_sum(pk, grid, eps, mesh.dq, mesh.dp, R=6)
    got = _gpu.reconstruct("direct", pk, grid, eps, _gpu.options("fp32"))
    assert got.dtype == np.complex64
    assert _gpu.rel_l2(got, ref) <= 1e-5


def test_direct_host_buffers_match_device():
    pk, grid, eps, mesh = _case(1, seed=3)
    a = _gpu.reconstruct("direct", pk, grid, eps, _gpu.options("fp64"), on_device=True)
    b = _gpu.reconstruct("direct", pk, grid, eps, _gpu.options("fp64"), on_device=False)
    assert _gpu.rel_l2(a, b) <= 1e-15


def test_direct_wide_window_fp32():
    # eps = 1/1024 on a fine grid: ~2000-point windows (the 1-D workload's shape)
    eps = 1 / 1024
    mesh = mesh_for(1, eps)
    pk = random_packets(5, 1, 400, q_range=(-3, 3), p_range=(-4, 4), s_range=(-1, 1), mesh=mesh)
    grid = _grid(1, 32768)
    rng = np.random.default_rng(0)
    pts = rng.integers(0, 32768, size=(1, 1500))
    ref = fga.direct_sum(pk, grid, eps, mesh.dq, mesh.dp, R=6, points=pts)
    got = _gpu.reconstruct("direct", pk, grid, eps, _gpu.options("fp32"))
    assert _gpu.rel_l2(got[tuple(pts)], ref) <= 1e-5


# ---------------------------------------------------------------------------
# K3-K5 FGGC
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("d", [1, 2, 3])
@pytest.mark.parametrize("nq,np_", [(4, 2), (2, 2)])
def test_fggc_fp64_matches_oracle(d, nq, np_):
    pk, grid, eps, mesh = _case(d, seed=4)
    strat = lsa.Strategy(nq=nq, np_=np_)
    ref = fggc.reconstruct(pk, grid, eps, mesh.dq, mesh.dp, strat, R=8)
    got = _gpu.reconstruct("fggc", pk, grid, eps, _gpu.options("fp64", nq=nq, np_=np_))
    assert _gpu.rel_l2(got, ref) <= _fp64_fggc_tol(nq, np_)


@pytest.mark.parametrize("nq,np_", [(2, 4), (4, 4)])
def test_fggc_fp64_other_strategies(nq, np_):
    pk, grid, eps, mesh = _case(1, seed=5)
    strat = lsa.Strategy(nq=nq, np_=np_)
    ref = fggc.reconstruct(pk, grid, eps, mesh.dq, mesh.dp, strat, R=8)
    got = _gpu.reconstruct("fggc", pk, grid, eps, _gpu.options("fp64", nq=nq, np_=np_))
    # Q4P4 is rank-truncated (cond ~1e18): both sides carry ~1e-8 of truncation
    tol = 1e-7 if strat.pinv.rank < strat.n1 else _fp64_fggc_tol(nq, np_)
    assert _gpu.rel_l2(got, ref) <= tol


@pytest.mark.parametrize("d", [1, 2, 3])
def test_fggc_fp32_matches_oracle(d):
    pk, grid, eps, mesh = _case(d, seed=6)
    strat = lsa.Strategy(nq=4, np_=2)
    ref = fggc.reconstruct(pk, grid, eps, mesh.dq, mesh.dp, strat, R=6)
    got = _gpu.reconstruct("fggc", pk, grid, eps, _gpu.options("fp32"))
    assert got.dtype == np.complex64
    assert _gpu.rel_l2(got, ref) <= 1e-5


@pytest.mark.parametrize("d", [1, 2])
@pytest.mark.parametrize("nq,np_", [(2, 2), (2, 4), (4, 4)])
def test_fggc_fp32_other_strategies(d, nq, np_):
    pk, grid, eps, mesh = _case(d, seed=7)
    strat = lsa.Strategy(nq=nq, np_=np_)
    ref = fggc.reconstruct(pk, grid, eps, mesh.dq, mesh.dp, strat, R=6)
    got = _gpu.reconstruct("fggc", pk, grid, eps, _gpu.options("fp32", nq=nq, np_=np_))
    err = _gpu.rel_l2(got, ref)
    print("FP32 FGGC Q%dP%d d=%d: rel L2 %.3e" % (nq, np_, d, err))
    assert err <= 1e-5


def test_fggc_on_grid_packets_equal_direct_on_gpu():
    d = 2
    eps = 1 / 64
    mesh = mesh_for(d, eps)
    pk = random_packets(9, d, 200, q_range=(-2, 2), p_range=(-2, 2), mesh=mesh, on_node_fraction=1.0)
    grid = _grid(d, (65, 70))
    a = _gpu.reconstruct("fggc", pk, grid, eps, _gpu.options("fp64"))
    b = _gpu.reconstruct("direct", pk, grid, eps, _gpu.options("fp64"))
    assert _gpu.rel_l2(a, b) <= _fp64_fggc_tol(4, 2)


def test_fggc_wide_p_range_fp32():
    # large |P| / dp (|b| up to ~330) and |Q| beyond the grid: phases of 1e4 rad
    eps = 1 / 1024
    mesh = mesh_for(1, eps)
    pk = random_packets(10, 1, 3000, q_range=(-3.5, 3.5), p_range=(-4, 4), s_range=(-2, 2), mesh=mesh)
    grid = _grid(1, 32768)
    strat = lsa.Strategy(nq=4, np_=2)
    rng = np.random.default_rng(1)
    pts = rng.integers(0, 32768, size=(1, 1200))
    ref = fggc.reconstruct(pk, grid, eps, mesh.dq, mesh.dp, strat, R=6, points=pts)
    got = _gpu.reconstruct("fggc", pk, grid, eps, _gpu.options("fp32"))
    assert _gpu.rel_l2(got[tuple(pts)], ref) <= 1e-5


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("method", ["direct", "fggc"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_edge_cases(method, prec):
    eps = 1 / 64
    mesh = mesh_for(1, eps)
    grid = _grid(1, 517)
    R = 8 if prec == "fp64" else 6
    tol = 1e-12 if prec == "fp64" else 1e-5
    if method == "fggc" and prec == "fp64":
        tol = _fp64_fggc_tol(4, 2)
    strat = lsa.Strategy(nq=4, np_=2)

    def ref_of(pk):
        if method == "direct":
            return fga.direct_sum(pk, grid, eps, mesh.dq, mesh.dp, R=R)
        return fggc.reconstruct(pk, grid, eps, mesh.dq, mesh.dp, strat, R=R)

    # no packets
    empty = random_packets(1, 1, 0, mesh=mesh)
    assert np.all(_gpu.reconstruct(method, empty, grid, eps, _gpu.options(prec)) == 0)
    # every packet far outside the grid
    far = random_packets(2, 1, 50, q_range=(20, 30), mesh=mesh)
    assert np.all(_gpu.reconstruct(method, far, grid, eps, _gpu.options(prec)) == 0)
    # one packet, negative Q and P, half outside the grid edge
    one = {"q": np.array([[-math.pi + 0.05]]), "p": np.array([[-1.37]]), "s": np.array([0.3]),
           "a": np.array([[0.7], [-0.2]])}
    assert _gpu.rel_l2(_gpu.reconstruct(method, one, grid, eps, _gpu.options(prec)), ref_of(one)) <= tol
    # zero amplitudes mixed with others, packets exactly on nodes
    mixed = random_packets(3, 1, 300, q_range=(-3, 3), p_range=(-2, 2), mesh=mesh, on_node_fraction=0.5)
    mixed["a"][:, ::3] = 0.0
    got = _gpu.reconstruct(method, mixed, grid, eps, _gpu.options(prec))
    assert _gpu.rel_l2(got, ref_of(mixed)) <= tol
    # a one-point grid
    g1 = _grid(1, 1, -0.01, 0.01)
    pt = random_packets(4, 1, 20, q_range=(-0.1, 0.1), mesh=mesh)
    r1 = (fga.direct_sum(pt, g1, eps, mesh.dq, mesh.dp, R=R) if method == "direct"
          else fggc.reconstruct(pt, g1, eps, mesh.dq, mesh.dp, strat, R=R))
    assert _gpu.rel_l2(_gpu.reconstruct(method, pt, g1, eps, _gpu.options(prec)), r1) <= tol


def test_invalid_arguments_are_rejected():
    import paper_2504_21785_gb300 as fgr
    with pytest.raises(fgr.FgrError) as e:
        fgr.Context(4, _grid(1, 10), 0.1)
    assert e.value.status == fgr.fgr.FGR_E_INVALID
    with pytest.raises(fgr.FgrError):
        fgr.Context(1, _grid(1, 10), -1.0)
    with pytest.raises(fgr.FgrError):
        fgr.Context(1, dict(d=1, n=[0], lo=[0.0], hi=[1.0]), 0.1)
    with pytest.raises(fgr.FgrError):
        fgr.Context(1, _grid(1, 10), 0.1, fgr.make_options(nq=3))
    ctx = fgr.Context(1, _grid(1, 10), 0.1)
    bad = {"q": np.array([[np.nan]]), "p": np.zeros((1, 1)), "s": np.zeros(1), "a": np.zeros((2, 1))}
    host = [np.ascontiguousarray(bad[k]) for k in ("q", "p", "s", "a")]
    u = np.zeros(10, np.complex128)
    with pytest.raises(fgr.FgrError):
        fgr.fgr_reconstruct_direct(ctx.handle, fgr.make_packets(*host), u)
    with pytest.raises(fgr.FgrError):
        fgr.fgr_propagate(ctx.handle, fgr.make_packets(*host), fgr.make_potential("free"), 1.0, -1.0)
    ctx.close()


def test_context_eigenvalues_match_oracle():
    import paper_2504_21785_gb300 as fgr
    for nq, np_ in [(2, 2), (4, 2), (2, 4), (4, 4)]:
        with fgr.Context(1, _grid(1, 8), 0.01, fgr.make_options(nq=nq, np_=np_)) as ctx:
            info = ctx.info()
            strat = lsa.Strategy(nq=nq, np_=np_)
            ev = np.array(info.eigenvalues[: info.n1])
            sv = strat.pinv.singular_values
            assert np.max(np.abs(ev - sv)) <= 1e-14 * sv[0]
            assert info.rank == strat.pinv.rank


# ---------------------------------------------------------------------------
# the workloads at their full sizes
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def cfg1():
    from workloads import config_workload
    w = config_workload(1)
    w["prop"] = tr.propagate(w["packets"], w["potential"], w["t"], w["dt"])
    return w


def test_config1_direct_and_fggc_fp64(cfg1):
    w = cfg1
    mesh, eps, grid = w["mesh"], w["eps"], w["grid"]
    strat = lsa.Strategy(nq=4, np_=2)
    ref_d = fga.direct_sum(w["prop"], grid, eps, mesh.dq, mesh.dp, R=8)
    ref_f = fggc.reconstruct(w["prop"], grid, eps, mesh.dq, mesh.dp, strat, R=8)
    got_d = _gpu.reconstruct("direct", w["prop"], grid, eps, _gpu.options("fp64"))
    got_f = _gpu.reconstruct("fggc", w["prop"], grid, eps, _gpu.options("fp64"))
    assert _gpu.rel_l2(got_d, ref_d) <= 1e-12
    assert _gpu.rel_l2(got_f, ref_f) <= _fp64_fggc_tol(4, 2)
    # FGGC against the direct sum it replaces: the LSA error (Q4P2) is far below 1e-5
    assert _gpu.rel_l2(got_f, got_d) <= 1e-6


@pytest.fixture(scope="module")
def cfg2():
    from workloads import config_workload
    w = config_workload(2)
    w["prop"] = tr.propagate(w["packets"], w["potential"], w["t"], w["dt"])
    return w


def test_config2_full_size_fp32(cfg2):
    # 262144 packets propagated to t = 1 by the oracle; the GPU reconstructs the
    # full 32768-point grid in FP32; the oracle evaluates 2048 sampled points.
    w = cfg2
    mesh, eps, grid = w["mesh"], w["eps"], w["grid"]
    strat = lsa.Strategy(nq=4, np_=2)
    rng = np.random.default_rng(0)
    pts = np.sort(rng.choice(grid["n"][0], size=2048, replace=False))[None, :]
    ref_d = fga.direct_sum(w["prop"], grid, eps, mesh.dq, mesh.dp, R=6, points=pts)
    ref_f = fggc.reconstruct(w["prop"], grid, eps, mesh.dq, mesh.dp, strat, R=6, points=pts)
    got_d = _gpu.reconstruct("direct", w["prop"], grid, eps, _gpu.options("fp32"))
    got_f = _gpu.reconstruct("fggc", w["prop"], grid, eps, _gpu.options("fp32"))
    assert _gpu.rel_l2(got_d[tuple(pts)], ref_d) <= 1e-5
    assert _gpu.rel_l2(got_f[tuple(pts)], ref_f) <= 1e-5
    assert _gpu.rel_l2(got_f, got_d) <= 1e-5


def test_config2_propagation_sample(cfg2):
    # the GPU integrator on the full 262144-packet set, checked on a sample
    w = cfg2
    got = _gpu.propagate(w["packets"], 1, w["potential"], w["t"], w["dt"])
    rng = np.random.default_rng(3)
    idx = rng.choice(w["packets"]["s"].size, size=4096, replace=False)
    ref = w["prop"]
    assert np.max(np.abs(got["q"][:, idx] - ref["q"][:, idx])) <= 1e-12 * np.max(np.abs(ref["q"]))
    assert np.max(np.abs(got["p"][:, idx] - ref["p"][:, idx])) <= 1e-12 * np.max(np.abs(ref["p"]))
    assert np.max(np.abs(got["s"][idx] - ref["s"][idx])) <= 1e-12 * max(1.0, np.max(np.abs(ref["s"])))
    A = got["a"][0, idx] + 1j * got["a"][1, idx]
    Ar = ref["a"][0, idx] + 1j * ref["a"][1, idx]
    nz = np.abs(Ar) > 1e-200
    assert np.max(np.abs(A[nz] - Ar[nz]) / np.abs(Ar[nz])) <= 1e-12


def test_non_finite_host_packets_are_rejected_in_large_sets():
    # a non-finite value anywhere in a large host packet set (near the end of
    # the amplitudes, in P, in S) rejects the call before any kernel writes the
    # output: FGGC tests the copied values on the device in its bounds
    # reduction, the direct sum scans them with several host threads while
    # their copy runs
    import paper_2504_21785_gb300 as fgr
    m = (1 << 21) + 17
    rng = np.random.default_rng(8)
    pk = {"q": rng.uniform(-1, 1, (1, m)), "p": rng.uniform(-1, 1, (1, m)), "s": rng.uniform(-1, 1, m),
          "a": rng.standard_normal((2, m))}
    grid = _grid(1, 256)
    with fgr.Context(1, grid, 1 / 64, fgr.make_options(precision=fgr.FGR_FP32)) as ctx:
        for key, idx in (("a", (1, m - 3)), ("p", (0, m // 2 + 1)), ("s", (m - 5,))):
            bad = {k: np.array(v, copy=True) for k, v in pk.items()}
            bad[key][idx] = np.inf if key == "a" else np.nan
            host = [np.ascontiguousarray(bad[k]) for k in ("q", "p", "s", "a")]
            u = np.full(256, 7.0, np.complex64)
            for call in (fgr.fgr_reconstruct_fggc, fgr.fgr_reconstruct_direct):
                with pytest.raises(fgr.FgrError) as e:
                    call(ctx.handle, fgr.make_packets(*host), u)
                assert e.value.status == fgr.fgr.FGR_E_INVALID
                assert np.all(u == 7.0)
