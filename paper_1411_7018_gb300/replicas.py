"""Replica execution over ranks: one process per GPU, each solving its own
instance (weak scaling).  The method has no data-path exchange between
replicas; the only collectives are the timing barrier and the max-over-ranks
reduction of the measured time.  Works with any torch.distributed backend
(NCCL on GPUs, gloo on the CPU)."""
from __future__ import annotations

import os


def rank_info(env=None):
    """(rank, local_rank, world_size) from the launcher's environment."""
    env = os.environ if env is None else env
    return int(env.get("RANK", "0")), int(env.get("LOCAL_RANK", "0")), int(env.get("WORLD_SIZE", "1"))


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def max_over_ranks(value: float, device=None) -> float:
    """The largest value over all ranks (the job's time is its slowest rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, max_seconds: float, world: int) -> float:
    """Units all ranks processed per second of the slowest rank."""
    return world * units_per_rank / max_seconds


def shard(items, rank: int, world: int):
    """The items rank `rank` of `world` takes (round robin): independent
    instances spread over replicas with nothing shared between them."""
    return list(items)[rank::world]
