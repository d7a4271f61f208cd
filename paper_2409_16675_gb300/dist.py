"""One process per GPU: the host-side logic of a multi-GPU run.

The linear layers shard without any exchange step: every rank owns whole
images (or whole jobs / requests) and its own keys, so the data path has no
collective.  The only collectives are the timing barrier and the max over
ranks of the timed region, which make the reported rate a whole-job figure
(weak scaling: per-rank work is fixed as the number of ranks grows).
"""
from __future__ import annotations

import os

RANK_STRIDE = 100003   # spacing of per-rank seeds (prime, far above any per-step offset)


def world():
    """(world_size, rank, local_rank) from the torchrun environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_seed(base: int, rank: int) -> int:
    """Seed of rank `rank`'s own inputs: distinct per rank, rank 0 keeps `base`."""
    return base + RANK_STRIDE * rank


def shard(n: int, rank: int, world_size: int) -> range:
    """Contiguous, balanced share of n independent units: the first n % W
    ranks take one unit more; every unit lands on exactly one rank."""
    q, r = divmod(n, world_size)
    lo = rank * q + min(rank, r)
    return range(lo, lo + q + (1 if rank < r else 0))


def reduce_max(value: float, device=None) -> float:
    """Max over ranks of a host float (identity when no process group is up)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def whole_job_rate(units_per_rank: float, world_size: int, max_seconds: float) -> float:
    """Units processed by all ranks per second of the slowest rank."""
    return units_per_rank * world_size / max_seconds
