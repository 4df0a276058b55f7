"""Host logic of multi-GPU runs (one process per GPU, no data-path collective).

One design iteration of one grid does not shard in this build; N GPUs run N
independent replicas (the 3D cantilever) or independent shares of a batch of
instances. The only cross-rank communication is timing and bookkeeping:
the slowest rank's time, and whole-job throughput = all ranks' units / that
time.
"""
from __future__ import annotations


def env():
    """(rank, local_rank, world_size) from the launcher's environment."""
    import os
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def max_over_ranks(value, world, device=None):
    """The maximum of a float over all ranks (value itself when world == 1)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value, world, device=None):
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def whole_job_rate(units_all_ranks, max_seconds):
    """Throughput of the whole job: every rank's units over the slowest rank's time."""
    return units_all_ranks / max_seconds if max_seconds > 0 else 0.0


def shard(costs, world):
    """Assign items with the given costs to `world` ranks: longest item first to
    the least-loaded rank (ties to the lower rank). Returns one sorted index list
    per rank; every item appears exactly once."""
    loads = [0.0] * world
    parts = [[] for _ in range(world)]
    for i in sorted(range(len(costs)), key=lambda k: (-costs[k], k)):
        r = min(range(world), key=lambda q: (loads[q], q))
        parts[r].append(i)
        loads[r] += costs[i]
    return [sorted(p) for p in parts]
