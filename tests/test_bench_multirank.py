"""The multi-rank path of bench.py on CPU: two gloo ranks (127.0.0.1), each with
its own batch; only the timing maximum crosses ranks, and rank 0 alone prints."""

import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    r, local, w = bench._rank_env()
    # each rank's own step time; the reported time is the slowest rank's
    got = bench.max_over_ranks(10.0 + 5.0 * rank, w)
    out.put((r, local, w, got))
    dist.destroy_process_group()


def test_max_over_ranks_with_gloo():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1]
    assert all(r[2] == 2 and r[3] == 15.0 for r in res)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5


def test_reference_arm_rank_nonzero_does_nothing(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        config = 2
        steps = 1
        warmup = 0
        ref_sample = 8
    assert bench.run_reference(A()) is None
