"""Serving (fgr_submit / fgr_poll): results in a concurrent mix equal the same
requests run alone; admission under a memory budget; cancellation; errors."""

import math
import threading

import numpy as np
import pytest

from workloads import random_packets

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fgr():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2504_21785_gb300 as pkg
    pkg.fgr.load()
    return pkg


def _grid(d, n):
    return dict(d=d, n=[n] * d, lo=[-math.pi] * d, hi=[math.pi] * d)


def _requests(seed=0, count=24):
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(count):
        d = int(rng.integers(1, 3))
        eps = float(2.0 ** -rng.uniform(6, 10))
        n = int(2 ** rng.integers(10, 13)) if d == 1 else int(2 ** rng.integers(6, 8))
        reqs.append(dict(d=d, eps=eps, grid=_grid(d, n), method=int(rng.integers(0, 2)),
                         set=int(rng.integers(0, 3)) + (0 if d == 1 else 3)))
    return reqs


def _sets():
    out = []
    for d in (1, 1, 1, 2, 2, 2):
        k = len(out)
        m = [4000, 12000, 30000, 2000, 6000, 9000][k]
        out.append(random_packets(50 + k, d, m, q_range=(-2.5, 2.5), p_range=(-2, 2), s_range=(-1, 1)))
    return out


def _alone(fgr, pk, r):
    from . import _gpu
    opt = fgr.make_options(precision=fgr.FGR_FP32)
    return _gpu.reconstruct("fggc" if r["method"] else "direct", pk, r["grid"], r["eps"], opt)


def test_results_alone_equal_results_in_the_mix(fgr):
    import torch
    sets = _sets()
    srv = fgr.fgr_server_create(8 << 30, 4)
    try:
        ids = [fgr.fgr_register_packets(srv, pk["q"].shape[0],
                                        fgr.make_packets(*[np.ascontiguousarray(pk[k]) for k in "qpsa"]))
               for pk in sets]
        reqs = _requests()
        outs, tickets = [], []
        opt = fgr.make_options(precision=fgr.FGR_FP32)
        for r in reqs:
            shape = tuple(r["grid"]["n"][: r["d"]])
            u = torch.zeros(shape, dtype=torch.complex64, device="cuda")
            outs.append(u)
            tickets.append(fgr.fgr_submit(srv, fgr.make_request(r["method"], r["grid"], r["eps"], opt,
                                                                ids[r["set"]], u)))
        results = [fgr.fgr_poll(srv, t, -1) for t in tickets]
        assert all(res.status == 0 for res in results)
        # the mix really overlapped: some request started before another finished
        spans = sorted((res.t_start_ms, res.t_done_ms) for res in results)
        assert any(spans[i + 1][0] < spans[i][1] for i in range(len(spans) - 1))
        for r, u in zip(reqs, outs):
            ref = _alone(fgr, sets[r["set"]], r)
            got = u.cpu().numpy()
            den = max(np.linalg.norm(ref), 1e-300)
            assert np.linalg.norm(got - ref) / den <= 1e-5
    finally:
        fgr.fgr_server_destroy(srv)


def test_admission_by_budget_and_host_output(fgr):
    pk = random_packets(60, 1, 20000, q_range=(-2, 2), p_range=(-2, 2))
    arrs = [np.ascontiguousarray(pk[k]) for k in "qpsa"]
    n = 4096
    # budget fits the set and about one request at a time
    srv = fgr.fgr_server_create(24 << 20, 4)
    try:
        sid = fgr.fgr_register_packets(srv, 1, fgr.make_packets(*arrs))
        opt = fgr.make_options(precision=fgr.FGR_FP32)
        outs = [np.zeros(n, np.complex64) for _ in range(6)]
        ts = [fgr.fgr_submit(srv, fgr.make_request(0, _grid(1, n), 1 / 256, opt, sid, u)) for u in outs]
        res = [fgr.fgr_poll(srv, t, -1) for t in ts]
        assert all(r.status == 0 for r in res)
        # same request six times; atomics make the summation order (not the sum) vary
        for u in outs[1:]:
            assert np.linalg.norm(u - outs[0]) <= 1e-6 * np.linalg.norm(outs[0])
        # a request that can never fit is refused at submit
        big = np.zeros(1 << 22, np.complex64)
        with pytest.raises(fgr.FgrError) as e:
            fgr.fgr_submit(srv, fgr.make_request(1, _grid(1, 1 << 22), 1 / 256, opt, sid, big))
        assert e.value.status == fgr.fgr.FGR_E_CAPACITY
    finally:
        fgr.fgr_server_destroy(srv)


def test_cancel_unknown_ticket_and_shutdown(fgr):
    import torch
    pk = random_packets(61, 2, 30000, q_range=(-2, 2), p_range=(-2, 2))
    srv = fgr.fgr_server_create(16 << 30, 1)
    sid = fgr.fgr_register_packets(srv, 2, fgr.make_packets(*[np.ascontiguousarray(pk[k]) for k in "qpsa"]))
    opt = fgr.make_options(precision=fgr.FGR_FP32)
    outs = [torch.zeros((512, 512), dtype=torch.complex64, device="cuda") for _ in range(5)]
    ts = [fgr.fgr_submit(srv, fgr.make_request(0, _grid(2, 512), 1 / 256, opt, sid, u)) for u in outs]
    cancelled = 0
    for t in ts[1:]:
        try:
            fgr.fgr_cancel(srv, t)
            cancelled += 1
        except fgr.FgrError:
            pass  # already admitted
    statuses = [fgr.fgr_poll(srv, t, -1).status for t in ts]
    assert statuses[0] == 0
    assert statuses.count(fgr.fgr.FGR_E_CANCELLED) == cancelled
    with pytest.raises(fgr.FgrError):
        fgr.fgr_poll(srv, 987654, 0)
    bad = fgr.make_request(0, _grid(2, 64), 1 / 256, opt, 12345, outs[0])
    with pytest.raises(fgr.FgrError):
        fgr.fgr_submit(srv, bad)
    # destroy with work queued: queued requests end cancelled, running ones finish
    ts2 = [fgr.fgr_submit(srv, fgr.make_request(0, _grid(2, 512), 1 / 256, opt, sid, u)) for u in outs]
    fgr.fgr_server_destroy(srv)
    torch.cuda.synchronize()
    assert len(ts2) == 5


def test_many_client_threads(fgr):
    import torch
    pk = random_packets(62, 1, 5000, q_range=(-2, 2), p_range=(-2, 2))
    srv = fgr.fgr_server_create(4 << 30, 3)
    try:
        sid = fgr.fgr_register_packets(srv, 1, fgr.make_packets(*[np.ascontiguousarray(pk[k]) for k in "qpsa"]))
        opt = fgr.make_options(precision=fgr.FGR_FP32)
        errors = []

        def client(i):
            try:
                u = torch.zeros(2048, dtype=torch.complex64, device="cuda")
                t = fgr.fgr_submit(srv, fgr.make_request(i % 2, _grid(1, 2048), 1 / 512, opt, sid, u))
                r = None
                while r is None:
                    r = fgr.fgr_poll(srv, t, 50)
                if r.status != 0:
                    errors.append(r.status)
            except Exception as e:  # noqa: BLE001
                errors.append(e)

        th = [threading.Thread(target=client, args=(i,)) for i in range(12)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        assert not errors
    finally:
        fgr.fgr_server_destroy(srv)


def test_direct_requests_waiting_together_run_as_one_batch(fgr):
    import torch
    from . import _gpu
    sets = [random_packets(70 + k, 1, m, q_range=(-2.5, 2.5), p_range=(-2, 2), s_range=(-1, 1))
            for k, m in enumerate((3000, 8000))]
    big = random_packets(72, 2, 200000, q_range=(-2.5, 2.5), p_range=(-2, 2))
    srv = fgr.fgr_server_create(8 << 30, 1)
    try:
        fgr.fgr_server_set_max_batch(srv, 64)
        with pytest.raises(fgr.FgrError):
            fgr.fgr_server_set_max_batch(srv, 65)
        ids = [fgr.fgr_register_packets(srv, 1, fgr.make_packets(*[np.ascontiguousarray(pk[k]) for k in "qpsa"]))
               for pk in sets]
        big_id = fgr.fgr_register_packets(srv, 2, fgr.make_packets(*[np.ascontiguousarray(big[k]) for k in "qpsa"]))
        opt = fgr.make_options(precision=fgr.FGR_FP32)
        # a long 2-D request holds the only slot while the 1-D ones queue up
        ub = torch.zeros((1024, 1024), dtype=torch.complex64, device="cuda")
        tickets = [fgr.fgr_submit(srv, fgr.make_request(1, _grid(2, 1024), 1 / 1024, opt, big_id, ub))]
        rng = np.random.default_rng(5)
        reqs, outs = [], []
        for i in range(40):
            r = dict(set=int(rng.integers(0, 2)), n=int(2 ** rng.integers(9, 13)),
                     eps=float(2.0 ** -rng.uniform(6, 10)))
            u = torch.zeros(r["n"], dtype=torch.complex64, device="cuda")
            reqs.append(r)
            outs.append(u)
            tickets.append(fgr.fgr_submit(srv, fgr.make_request(0, _grid(1, r["n"]), r["eps"], opt,
                                                                ids[r["set"]], u)))
        res = [fgr.fgr_poll(srv, t, -1) for t in tickets]
        assert all(x.status == 0 for x in res)
        # a group shares its start and completion times
        groups = {}
        for x in res[1:]:
            groups.setdefault((x.t_start_ms, x.t_done_ms), []).append(x)
        assert max(len(g) for g in groups.values()) >= 2
        for r, u in zip(reqs, outs):
            ref = _gpu.reconstruct("direct", sets[r["set"]], _grid(1, r["n"]), r["eps"], opt)
            got = u.cpu().numpy()
            assert np.linalg.norm(got - ref) <= 1e-6 * max(np.linalg.norm(ref), 1e-300)
    finally:
        fgr.fgr_server_destroy(srv)


def test_fggc_requests_through_cached_plans_and_release(fgr):
    import torch
    from . import _gpu
    pk = random_packets(80, 1, 6000, q_range=(-2.5, 2.5), p_range=(-2, 2), s_range=(-1, 1))
    big = random_packets(81, 2, 200000, q_range=(-2.5, 2.5), p_range=(-2, 2))
    srv = fgr.fgr_server_create(8 << 30, 1)
    try:
        sid = fgr.fgr_register_packets(srv, 1, fgr.make_packets(*[np.ascontiguousarray(pk[k]) for k in "qpsa"]))
        big_id = fgr.fgr_register_packets(srv, 2, fgr.make_packets(*[np.ascontiguousarray(big[k]) for k in "qpsa"]))
        opt = fgr.make_options(precision=fgr.FGR_FP32)
        ub = torch.zeros((1024, 1024), dtype=torch.complex64, device="cuda")
        tickets = [fgr.fgr_submit(srv, fgr.make_request(1, _grid(2, 1024), 1 / 1024, opt, big_id, ub))]
        # two grids, each asked for several times: the second and later requests
        # of a (set, grid) reuse its plan; requests that wait together form groups
        reqs, outs = [], []
        for i in range(24):
            n = 2048 if i % 2 else 4096
            u = torch.full((n,), 9.0, dtype=torch.complex64, device="cuda")
            reqs.append(n)
            outs.append(u)
            tickets.append(fgr.fgr_submit(srv, fgr.make_request(1, _grid(1, n), 1 / 512, opt, sid, u)))
        res = [fgr.fgr_poll(srv, t, -1) for t in tickets]
        assert all(x.status == 0 for x in res)
        for n, u in zip(reqs, outs):
            ref = _gpu.reconstruct("fggc", pk, _grid(1, n), 1 / 512, opt)
            got = u.cpu().numpy()
            assert np.linalg.norm(got - ref) <= 1e-6 * np.linalg.norm(ref)
        # releasing the set frees its plans; new sets and requests still work
        fgr.fgr_release_packets(srv, sid)
        sid2 = fgr.fgr_register_packets(srv, 1, fgr.make_packets(*[np.ascontiguousarray(pk[k]) for k in "qpsa"]))
        u = torch.zeros(4096, dtype=torch.complex64, device="cuda")
        r = fgr.fgr_poll(srv, fgr.fgr_submit(srv, fgr.make_request(1, _grid(1, 4096), 1 / 512, opt, sid2, u)), -1)
        assert r.status == 0
        ref = _gpu.reconstruct("fggc", pk, _grid(1, 4096), 1 / 512, opt)
        assert np.linalg.norm(u.cpu().numpy() - ref) <= 1e-6 * np.linalg.norm(ref)
    finally:
        fgr.fgr_server_destroy(srv)


def test_cached_plans_give_way_to_a_request_that_needs_their_memory(fgr):
    # A small budget; FGGC requests on distinct grids each leave a cached plan
    # (resident memory); then a request whose footprint fitted only before
    # those plans existed.  The scheduler frees idle plans, least recently
    # used first, instead of waiting for memory that nothing would release.
    import torch
    from . import _gpu
    m = 4000
    pk = random_packets(82, 1, m, q_range=(-2.5, 2.5), p_range=(-2, 2), s_range=(-1, 1))
    n_big = 1 << 20
    set_bytes = m * 5 * 8
    big_footprint = m * 112 + (n_big // 64 + 1) * 16 + n_big * 8   # direct-sum footprint rule of the server
    srv = fgr.fgr_server_create(set_bytes + big_footprint + (3 << 19), 1)
    try:
        sid = fgr.fgr_register_packets(srv, 1, fgr.make_packets(*[np.ascontiguousarray(pk[k]) for k in "qpsa"]))
        opt = fgr.make_options(precision=fgr.FGR_FP32)
        grids = [1024 + 96 * i for i in range(12)]
        outs = []
        for n in grids:   # one at a time: every request creates and keeps its plan
            u = torch.zeros(n, dtype=torch.complex64, device="cuda")
            r = fgr.fgr_poll(srv, fgr.fgr_submit(srv, fgr.make_request(1, _grid(1, n), 1 / 512, opt, sid, u)),
                             60000)
            assert r.status == 0
            outs.append(u)
        ub = torch.zeros(n_big, dtype=torch.complex64, device="cuda")
        t = fgr.fgr_submit(srv, fgr.make_request(0, _grid(1, n_big), 1 / 512, opt, sid, ub))
        r = fgr.fgr_poll(srv, t, 60000)
        assert r.status == 0
        ref = _gpu.reconstruct("direct", pk, _grid(1, n_big), 1 / 512, opt)
        assert np.linalg.norm(ub.cpu().numpy() - ref) <= 1e-6 * np.linalg.norm(ref)
        # the evicted plans are rebuilt on demand
        u = torch.zeros(grids[0], dtype=torch.complex64, device="cuda")
        r = fgr.fgr_poll(srv, fgr.fgr_submit(srv, fgr.make_request(1, _grid(1, grids[0]), 1 / 512, opt, sid, u)),
                         60000)
        assert r.status == 0
        assert np.linalg.norm(u.cpu().numpy() - outs[0].cpu().numpy()) <= 1e-6 * np.linalg.norm(outs[0].cpu().numpy())
    finally:
        fgr.fgr_server_destroy(srv)


def test_small_requests_pass_a_large_direct_sum(fgr):
    # A 2-D direct sum of 2^21 packets on 1024^2 points (about 10 ms alone) is a
    # large request: it runs on a low-priority stream, leaves a worker slot to
    # small requests and, while they wait, gives up a CTA slot per SM between
    # its work items.  Small requests submitted right after it finish first,
    # and every result equals the same request run alone.
    import torch
    from . import _gpu
    big = random_packets(91, 2, 1 << 21, q_range=(-2.5, 2.5), p_range=(-2, 2), s_range=(-1, 1))
    small = [random_packets(92 + k, 1, 6000, q_range=(-2.5, 2.5), p_range=(-2, 2), s_range=(-1, 1))
             for k in range(2)]
    opt = fgr.make_options(precision=fgr.FGR_FP32)
    srv = fgr.fgr_server_create(8 << 30, 4)
    try:
        sid_big = fgr.fgr_register_packets(srv, 2, fgr.make_packets(*[np.ascontiguousarray(big[k]) for k in "qpsa"]))
        sids = [fgr.fgr_register_packets(srv, 1, fgr.make_packets(*[np.ascontiguousarray(p[k]) for k in "qpsa"]))
                for p in small]
        g_big = _grid(2, 1024)
        u_big = torch.zeros((1024, 1024), dtype=torch.complex64, device="cuda")
        reqs = [(k % 2, int(2 ** (10 + k % 3)), k % 2) for k in range(16)]   # (set, n, method)
        outs = [torch.zeros(n, dtype=torch.complex64, device="cuda") for (_, n, _) in reqs]
        t_big = fgr.fgr_submit(srv, fgr.make_request(0, g_big, 1 / 64, opt, sid_big, u_big))
        tickets = [fgr.fgr_submit(srv, fgr.make_request(mth, _grid(1, n), 1 / 256, opt, sids[s], u))
                   for (s, n, mth), u in zip(reqs, outs)]
        res = [fgr.fgr_poll(srv, t, 60000) for t in tickets]
        r_big = fgr.fgr_poll(srv, t_big, 60000)
        assert r_big.status == 0 and all(r.status == 0 for r in res)
        assert max(r.t_done_ms for r in res) < r_big.t_done_ms
        ref = _gpu.reconstruct("direct", big, g_big, 1 / 64, opt)
        # the server cuts the large sum into finer work items, so its FP32
        # partial sums meet in another order: equal to the FP32 tolerance
        assert _gpu.rel_l2(u_big.cpu().numpy(), ref) <= 1e-5
        for (s, n, mth), u in zip(reqs, outs):
            ref = _gpu.reconstruct("fggc" if mth else "direct", small[s], _grid(1, n), 1 / 256, opt)
            assert _gpu.rel_l2(u.cpu().numpy(), ref) <= 1e-6
    finally:
        fgr.fgr_server_destroy(srv)
