"""Sharding a trajectory workload across ranks (one process per GPU).

Trajectories are independent and every random number of a lane is keyed by
its global id (Philox counter = id), so a workload splits into contiguous
id ranges with no data-path exchange; results do not depend on the split.
The one exchange a caller may want is the sum of the per-cell int64
histograms, which is exact (bit-identical in any order and for any number of
ranks).  torch.distributed provides the collective (NCCL on GPUs, gloo on
CPUs); a rank that has died shows up as an error of that collective within
the process group's timeout.
"""
from __future__ import annotations

import datetime

import torch


def shard_range(n: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous [lo, hi) slice of n lanes for `rank` of `world`
    (sizes differ by at most one)."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError(f"bad shard request n={n} rank={rank} world={world}")
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def merge_histograms(hist: torch.Tensor, group=None) -> torch.Tensor:
    """In-place sum of the int64 histograms over all ranks."""
    if hist.dtype != torch.int64:
        raise TypeError("histograms are int64 (exact sums)")
    torch.distributed.all_reduce(hist, op=torch.distributed.ReduceOp.SUM, group=group)
    return hist


def init_process_group(backend: str, timeout_s: float = 60.0):
    """torch.distributed init from the usual environment (RANK, WORLD_SIZE,
    MASTER_ADDR, MASTER_PORT) with a bounded collective timeout."""
    torch.distributed.init_process_group(backend, timeout=datetime.timedelta(seconds=timeout_s))
