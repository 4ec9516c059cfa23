"""Multi-rank logic of bench.py on CPU (gloo, world size 2).

The solve shards over right-hand sides with no collective on the data path:
each rank solves its own source, and only the step time is reduced (max over
ranks).  These tests run that host logic in two spawned gloo processes.
"""
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.max_over_ranks(10.0 + rank, world)
    src = bench.source_for_rank((1023, 1023), rank)
    bench.barrier(world)
    q.put((rank, t, src))
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_time_and_take_distinct_sources():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert [o[1] for o in out] == [11.0, 11.0]          # max over ranks on every rank
    srcs = [o[2] for o in out]
    assert srcs[0] != srcs[1]
    for x, y in srcs:
        assert 0 <= x < 1023 and 0 <= y < 1023


def test_sources_distinct_for_eight_ranks():
    sys.path.insert(0, ROOT)
    import bench
    srcs = [bench.source_for_rank((1023, 1023), r) for r in range(8)]
    assert len(set(srcs)) == 8


def test_reference_arm_non_zero_rank_exits_without_work(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        steps, warmup = 1, 0
    assert bench.run_reference(Args()) == 0
    assert capsys.readouterr().out == ""
