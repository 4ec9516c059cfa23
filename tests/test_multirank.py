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


# ---------------------------------------------------------------------------
# the misfit gradient over source shards: one all-reduce of the interior grid
# ---------------------------------------------------------------------------

def _grad_problem():
    sys.path.insert(0, ROOT)
    from paper_1208_3956_gb300 import media
    n = (20, 16)
    w = 3
    h = 1.0 / 16
    c0 = media.smooth_medium(n, 2.0, 1.0, 2.0, 3)
    c = c0 * (1 + 0.1 * media.smooth_medium(n, 2.0, 0.0, 1.0, 4))
    omega = media.omega_for(c0, h, 8.0)
    src = [media.padded_index((x, 0), n, w) for x in (3, 9, 15)]
    rec = [media.padded_index((x, 0), n, w) for x in range(0, 20, 3)]
    return n, w, h, c0, c, omega, src, rec


class _OracleSolver:
    """Stands in for a rank's factored solver: the oracle's gradient of its shard."""

    def __init__(self, c, h, omega, w, c_ref):
        self.c, self.h, self.omega, self.w, self.c_ref = c, h, omega, w, c_ref
        self.n = tuple(reversed(c.shape))
        self.calls = []

    def gradient(self, src, rec, d, tol):
        from oracle.helm_oracle import misfit_and_gradient
        self.calls.append(list(src))
        return misfit_and_gradient(self.c, self.h, self.omega, self.w, list(src), rec, d, c_ref=self.c_ref)


def _grad_worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist

    from oracle.helm_oracle import receiver_data
    from paper_1208_3956_gb300 import sharded
    n, w, h, c0, c, omega, src, rec = _grad_problem()
    d = receiver_data(c0, h, omega, w, src, rec, c_ref=2.5)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    s = _OracleSolver(c, h, omega, w, 2.5)
    J, g = sharded.gradient_over_ranks(s, src, rec, d)
    q.put((rank, J, g, s.calls))
    dist.destroy_process_group()


def test_gradient_over_two_gloo_ranks_sums_the_source_shards():
    sys.path.insert(0, ROOT)
    import numpy as np

    from oracle.helm_oracle import misfit_and_gradient, receiver_data
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_grad_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=300) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort(key=lambda o: o[0])
    n, w, h, c0, c, omega, src, rec = _grad_problem()
    d = receiver_data(c0, h, omega, w, src, rec, c_ref=2.5)
    Jref, gref = misfit_and_gradient(c, h, omega, w, src, rec, d, c_ref=2.5)
    assert [o[3] for o in out] == [[src[:2]], [src[2:]]]   # 3 sources: shares of 2 and 1
    for _, J, g, _ in out:
        assert abs(J - Jref) <= 1e-12 * abs(Jref)
        assert np.linalg.norm(g - gref) <= 1e-12 * np.linalg.norm(gref)


def test_shard_is_balanced_and_covers_every_item():
    sys.path.insert(0, ROOT)
    from paper_1208_3956_gb300 import sharded
    for n in (0, 1, 3, 16, 17, 64):
        for world in (1, 2, 3, 8):
            parts = [sharded.shard(n, r, world) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == n
            assert all(parts[i][1] == parts[i + 1][0] for i in range(world - 1))
            sizes = [hi - lo for lo, hi in parts]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        sharded.shard(4, 2, 2)
