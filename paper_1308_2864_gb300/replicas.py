"""Replica helpers for running independent systems on several GPUs.

One system does not shard across GPUs here; a multi-GPU job runs one replica
per rank (one process per GPU) over a disjoint share of independent jobs,
with no collective on the data path.  The only collective is the final
max-over-ranks of the elapsed time (and the gathering of counts), which
works with any torch.distributed backend.
"""
from __future__ import annotations


def shard(njobs: int, rank: int, world: int) -> list[int]:
    """Job indices of `rank`: round-robin, disjoint, covering all jobs."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    return list(range(rank, njobs, world))


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a float over all ranks (the float itself without a
    process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
