"""Sharding of Monte Carlo work across ranks (one process per GPU).

Photons are independent, and their random numbers depend only on (seed, item id,
photon id), so a batch can be split across ranks by photon ranges of each item with no
exchange during the walk; the only collective is an exact int64 sum of the count table
at the end (associative, hence bit-identical to a single-rank run).  Each rank passes
its `photon_first` / `photons_per_item` to fos_mc_spectrum and then calls
`allreduce_counts`.
"""
from __future__ import annotations

import numpy as np


def photon_range(n_photons: int, rank: int, world: int):
    """The photon ids [first, first + count) of `rank` among `world` ranks: contiguous,
    disjoint, covering [0, n_photons), sizes differing by at most one."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    base, extra = divmod(int(n_photons), int(world))
    first = rank * base + min(rank, extra)
    count = base + (1 if rank < extra else 0)
    return first, count


def photon_ranges(n_photons, rank: int, world: int):
    """Per-item version: arrays (first [n_items], count [n_items]) for int64 budgets."""
    n = np.asarray(n_photons, np.int64)
    base, extra = np.divmod(n, world)
    first = rank * base + np.minimum(rank, extra)
    count = base + (rank < extra).astype(np.int64)
    return first, count


def allreduce_counts(counts, group=None):
    """Exact int64 sum of count tables over the ranks of torch.distributed (gloo on CPU,
    NCCL on GPU)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(counts, op=dist.ReduceOp.SUM, group=group)
    return counts
