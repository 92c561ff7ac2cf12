"""Host-side logic of the multi-GPU run: one process per GPU, each projecting
its own contiguous row range of one point set X with the same landmarks
(Section 3.1: points are independent, so there is no exchange on the data
path).

* ``row_range`` splits the n rows of X into one contiguous range per rank;
  each rank writes the coordinates of its own rows, so the ranks' outputs
  concatenated in rank order are the projection of X.
* ``LandmarkSync`` replicates the landmarks (L and l): one broadcast of
  L (d + 2) floats from rank 0 per landmark version, nothing while the
  version is unchanged.
* Weak scaling: X has n points per rank, so the job's throughput is the
  points of all ranks over the slowest rank's time.

The only collectives are the landmark broadcast, the barriers around the
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


def _group_size() -> int:
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        return dist.get_world_size()
    return 1


def row_range(n: int, world: int, rank: int) -> tuple[int, int]:
    """[start, stop) of the rows of an n-row X that `rank` projects: contiguous
    ranges in rank order, sizes differing by at most one (the first n % world
    ranks take one more)."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError(f"row_range(n={n}, world={world}, rank={rank})")
    base, extra = divmod(n, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


class LandmarkSync:
    """Keeps every rank's copy of the landmarks equal to rank 0's.

    ``sync(version, hi, lo)`` takes rank 0's landmark version and, on every
    rank, tensors of the landmarks' shapes (L x d and L x 2; their contents
    matter only on rank 0).  When rank 0's version differs from the last one
    synchronised, rank 0's (hi, lo) are broadcast as one packed buffer of
    L (d + 2) floats and written into every rank's tensors; otherwise
    nothing is sent.  Returns True when a broadcast happened.  Without a
    process group (one rank) it only records the version."""

    def __init__(self, device="cpu"):
        self.device = device
        self.version = None
        self.broadcasts = 0

    def sync(self, version: int, hi, lo) -> bool:
        import torch
        import torch.distributed as dist
        version = broadcast_choice(int(version), device=self.device)
        if version == self.version:
            return False
        self.version = version
        if _group_size() > 1:
            packed = torch.cat([hi.reshape(-1), lo.reshape(-1)]).to(self.device)
            dist.broadcast(packed, 0)
            hi.copy_(packed[:hi.numel()].view_as(hi))
            lo.copy_(packed[hi.numel():].view_as(lo))
            self.broadcasts += 1
        return True


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
