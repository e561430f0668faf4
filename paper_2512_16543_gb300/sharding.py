"""Instance sharding across ranks (one process per GPU).

Instances are independent, so each rank owns a disjoint, contiguous range of global instance
identities and runs them with no communication on the data path.  The identities feed the
Philox counters of Algorithm 1, so an instance's results do not depend on which rank (or which
batch position) computes it.  The only cross-rank operation is the timing reduction: the job
time is the maximum of the per-rank times.
"""
from __future__ import annotations

import torch


def shard_ids(rank: int, world: int, per_rank: int) -> list[int]:
    """Global instance identities owned by `rank` when every rank runs `per_rank` instances."""
    if not (0 <= rank < world) or per_rank < 1:
        raise ValueError("bad rank / world / per_rank")
    return list(range(rank * per_rank, (rank + 1) * per_rank))


def max_over_ranks(value: float, device: torch.device | str = "cpu") -> float:
    """Maximum of `value` over the default process group (the value itself without one)."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device: torch.device | str = "cpu") -> float:
    """Sum of `value` over the default process group (units processed by the whole job)."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
