"""Host-side logic of the multi-rank benchmark on CPU ranks (gloo, world size 2).

Each rank owns independent solves (no data-path collective); the job time is
the maximum over ranks and the job rate sums every rank's updates.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, _ = bench.dist_env()
    mine = bench.shard(7, r, ws)
    t, u = bench.reduce_max_sum(1.0 + r, 100.0 * len(mine), dist)
    q.put((r, mine, t, u))
    dist.barrier()
    dist.destroy_process_group()


def test_sharding_is_a_partition():
    for n in (0, 1, 5, 8, 13):
        for world in (1, 2, 3, 8):
            units = [u for r in range(world) for u in bench.shard(n, r, world)]
            assert units == list(range(n))
            sizes = [len(bench.shard(n, r, world)) for r in range(world)]
            assert max(sizes) - min(sizes) <= 1


def test_two_gloo_ranks_max_time_and_total_updates():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, m0, t0, u0), (r1, m1, t1, u1) = out
    assert sorted(m0 + m1) == list(range(7))
    assert t0 == t1 == 2.0                 # max over ranks
    assert u0 == u1 == 700.0               # sum over ranks


def test_reference_arm_other_ranks_exit_without_work(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench.run_reference(type("A", (), {"warmup": 3, "steps": 1, "gpus": 2})()) == 0
