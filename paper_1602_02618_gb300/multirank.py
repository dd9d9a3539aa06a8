"""Multi-GPU form: independent replicas, one process per GPU.

Transforms are independent (each output depends on one input vector and one
plan), so a job of many transforms splits over ranks with no exchange on the
data path.  Rank r draws its own items from seeded streams offset by r, i.e. it
runs the r-th shard of a job `world` times as large as the one-GPU workload, on
its own GPU.  Per-rank work is fixed as the number of ranks grows (weak scaling).

The only collectives are host-side bookkeeping around a timed region: a barrier
before and after it, a maximum over ranks of the measured time, and a sum over
ranks of the units processed.  They work on any torch.distributed backend
(NCCL on GPUs, gloo on CPU) and are no-ops when `dist` is None (one process).

Environment: RANK, LOCAL_RANK and WORLD_SIZE as set by torchrun; a missing
variable means a single process.
"""
from __future__ import annotations

import os

# Seed offset between ranks.  Item t of a workload draws from stream seed + t (and
# small fixed offsets), with t below 2^20 in every workload here, so the streams of
# different ranks never coincide.
RANK_SEED_STRIDE = 1 << 24


def env():
    """(world, rank, local_rank) from the torchrun environment."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    if world < 1 or not 0 <= rank < world:
        raise ValueError("inconsistent WORLD_SIZE=%d, RANK=%d" % (world, rank))
    return world, rank, local


def rank_seed(seed: int, rank: int) -> int:
    """Base seed of rank `rank`'s shard; rank 0 keeps `seed` (the one-GPU workload)."""
    if rank < 0:
        raise ValueError("rank must be >= 0")
    return int(seed) + RANK_SEED_STRIDE * int(rank)


def _reduce(x: float, dist, device, op_name: str) -> float:
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=getattr(dist.ReduceOp, op_name))
    return float(t.item())


def max_over_ranks(x: float, dist=None, device="cpu") -> float:
    """Maximum of x over all ranks (x itself for one process)."""
    return _reduce(x, dist, device, "MAX")


def sum_over_ranks(x: float, dist=None, device="cpu") -> float:
    """Sum of x over all ranks (x itself for one process)."""
    return _reduce(x, dist, device, "SUM")


def barrier(dist=None):
    if dist is not None:
        dist.barrier()


def job_rate(units_all_ranks: float, max_seconds: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    if max_seconds <= 0:
        raise ValueError("time must be positive")
    return float(units_all_ranks) / float(max_seconds)
