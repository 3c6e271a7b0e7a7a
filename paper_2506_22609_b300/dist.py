"""Multi-GPU sharding for playout batches (weak scaling, no data-path collective).

Envs are independent and every random draw is keyed by the GLOBAL env index,
so rank r of a world of W ranks simply plays the env range
[r * n_per_rank, (r + 1) * n_per_rank) through env_offset: the union of the
ranks' results equals one big batch played on one GPU.  The only collective
is the end-of-run reduction of timing (max over ranks) and work done (sum).
"""
from __future__ import annotations

import os


def world_info():
    """(rank, world_size, local_rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard_offset(rank: int, n_per_rank: int) -> int:
    """Global index of this rank's first env."""
    return rank * n_per_rank


def aggregate(total_ms: float, units: float, device=None):
    """(max over ranks of the timed milliseconds, sum over ranks of the work
    units); identity when torch.distributed is not initialised."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(total_ms), float(units)
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())
