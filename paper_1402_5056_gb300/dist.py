"""Sharding of independent updates across ranks (one process per GPU).

Updates of an isolated batch are independent (each reads the same base
matrix), so ranks need no data exchange: under weak scaling every rank runs
a batch of its own (its own seed), under strong scaling the ranks split one
batch by index.  The only communication is the timing reduction of the
benchmark harness.  Works with any torch.distributed backend (NCCL on GPUs,
gloo on CPU).
"""
from __future__ import annotations


def shard_range(count: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous slice [begin, end) of ``count`` updates for ``rank`` of
    ``world``; the first ``count % world`` ranks take one more."""
    if world < 1 or not (0 <= rank < world) or count < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(count, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def rank_seed(seed: int, rank: int) -> int:
    """Seed of a rank's own batch under weak scaling."""
    return seed + rank


def reduce_max(value: float, dist=None, device=None) -> float:
    """Maximum of ``value`` over all ranks (``dist`` = torch.distributed or None)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(value: float, dist=None, device=None) -> float:
    """Sum of ``value`` over all ranks."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
