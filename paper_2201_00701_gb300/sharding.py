"""Host-side logic of the multi-GPU run: one process per GPU, each projecting
its own shard of points with the same landmarks (Section 3.1: points are
independent, so there is no exchange on the data path).

Weak scaling: every rank holds `n` points of its own (drawn with a
rank-specific seed), so the job's throughput is the points of all ranks over
the slowest rank's time.  The only collectives are the barriers around the
timed region, the broadcast of rank 0's plan choice and the maximum of the
ranks' times; they run on whatever process group is initialised (NCCL on
GPUs, gloo in the CPU tests).
"""
from __future__ import annotations

import os


def env_ranks() -> tuple[int, int, int]:
    """(world size, rank, local rank) from the torchrun environment."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(values, device="cpu"):
    """Element-wise maximum of a list of floats over all ranks (identity
    without a process group)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def broadcast_choice(value: int, device="cpu") -> int:
    """Rank 0's integer choice on every rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1):
        return int(value)
    t = torch.tensor([int(value)], dtype=torch.int64, device=device)
    dist.broadcast(t, 0)
    return int(t[0])


def job_throughput(points_per_rank: int, world: int, steps: int, max_seconds: float) -> float:
    """Units of all ranks over the slowest rank's time (weak scaling)."""
    return world * points_per_rank * steps / max_seconds
