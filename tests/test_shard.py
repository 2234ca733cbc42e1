"""Multi-GPU host logic on CPU: batch sharding and the timing reductions, with world_size-2
gloo process groups (127.0.0.1 rendezvous)."""
import os
import socket

import numpy as np
import pytest

from paper_2510_09812_gb300.shard import batch_shard, max_over_ranks, sum_over_ranks

torch = pytest.importorskip("torch")


def test_batch_shard_partitions_and_balances():
    rng = np.random.default_rng(3)
    counts = rng.integers(2000, 200000, size=64)
    for world in (1, 2, 3, 8):
        parts = [batch_shard(counts, r, world) for r in range(world)]
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(64))
        for p in parts:
            assert p == sorted(p)
        loads = [counts[p].sum() for p in parts]
        # greedy LPT: no rank exceeds the mean by more than the largest mesh
        assert max(loads) - counts.sum() / world <= counts.max()


def test_batch_shard_edge_cases():
    assert batch_shard([], 0, 2) == []
    assert batch_shard([5], 1, 2) == []
    assert batch_shard([5, 5, 5], 0, 2) == [0, 2]
    with pytest.raises(ValueError):
        batch_shard([1], 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, counts, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = batch_shard(counts, rank, world)
    units = sum_over_ranks(float(len(mine)))
    t = max_over_ranks(1.0 + rank)
    dist.barrier()
    out.put((rank, mine, units, t))
    dist.destroy_process_group()


def test_two_rank_gloo_shard_and_reductions():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    counts = [7000, 150000, 3000, 42000, 99000, 2000, 64000]
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, counts, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, m0, u0, t0), (r1, m1, u1, t1) = res
    assert sorted(m0 + m1) == list(range(len(counts))) and not set(m0) & set(m1)
    assert u0 == u1 == len(counts)
    assert t0 == t1 == 2.0


def test_reductions_without_process_group():
    assert max_over_ranks(3.5) == 3.5 and sum_over_ranks(2.0) == 2.0
