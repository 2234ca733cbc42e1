"""Host-side logic of multi-GPU runs: one process per GPU, no data-path collective.

Independent meshes of a batch are the only units that shard: each rank steps its own share in
one batched context, and ranks meet only to time the run (a barrier on both sides and the
largest elapsed time).  A single mesh does not shard (it would need a halo exchange per SpMV and
reductions per CG iteration), so single-mesh runs on N GPUs are N independent replicas.
"""
from __future__ import annotations

import numpy as np


def batch_shard(node_counts, rank: int, world: int) -> list[int]:
    """Indices of the meshes that `rank` of `world` steps.

    Greedy longest-processing-time split by node count (a step's work is proportional to the
    nodes): meshes in decreasing size (ties by index) go to the rank with the fewest nodes so
    far (ties by rank).  Every mesh goes to exactly one rank; each rank's list is ascending.
    """
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    counts = np.asarray(node_counts, dtype=np.int64)
    load = np.zeros(world, dtype=np.int64)
    owner = np.empty(counts.size, dtype=np.int64)
    for i in sorted(range(counts.size), key=lambda k: (-counts[k], k)):
        r = int(np.argmin(load))
        owner[i] = r
        load[r] += counts[i]
    return [int(i) for i in np.flatnonzero(owner == rank)]


def max_over_ranks(value: float, device=None) -> float:
    """Largest `value` over the ranks of the default process group (the value itself without
    one).  `device`: where the reduction tensor lives (CUDA for NCCL, CPU for gloo)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    """Sum of `value` over the ranks (units processed by the whole job)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
