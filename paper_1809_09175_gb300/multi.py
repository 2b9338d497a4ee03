"""Multi-rank host logic (one process per GPU, launched by torchrun).

The MTTKRP / CP-ALS work of this library shards into independent problems:
every rank works on its own tensor (or on its share of a batch of tensors),
so ranks exchange nothing on the data path.  The only collectives are the
timing reductions of a measurement: the slowest rank's time and the sum of
the units processed (weak scaling: work per rank is fixed as ranks grow).
Works with any torch.distributed backend (nccl on GPUs, gloo on CPU).
"""
from __future__ import annotations

from typing import List, Sequence, TypeVar

T = TypeVar("T")


def rank_seed(seed: int, rank: int) -> int:
    """Seed of rank `rank`'s independent problem."""
    return seed + 7919 * rank


def shard(items: Sequence[T], rank: int, world: int) -> List[T]:
    """Round-robin share of `items` for `rank` (disjoint, covers all)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    return [x for i, x in enumerate(items) if i % world == rank]


def reduce_timing(local_seconds: float, local_units: float, device=None):
    """(max seconds over ranks, sum of units over ranks); no-op without a
    process group."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return local_seconds, local_units
    t = torch.tensor([local_seconds], dtype=torch.float64, device=device)
    u = torch.tensor([local_units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def aggregate_throughput(local_seconds: float, local_units: float, device=None) -> float:
    """Whole-job throughput: all ranks' units over the slowest rank's time."""
    t, u = reduce_timing(local_seconds, local_units, device)
    return u / t if t > 0 else 0.0
