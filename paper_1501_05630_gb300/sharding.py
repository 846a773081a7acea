"""Instance sharding across GPUs (one process per GPU).

Disorder instances are independent: PT and the cluster moves stay inside an
instance, so a multi-GPU run gives every rank a disjoint range of instance
ids and needs no collective on the data path.  The only exchange is a
host-side gather of per-instance results when a caller wants disorder
averages over all ranks.
"""
from __future__ import annotations

import numpy as np


def instance_range(rank: int, world: int, n_per_rank: int, first: int = 0) -> np.ndarray:
    """Instance ids of `rank` under weak scaling (n_per_rank per rank)."""
    if not (0 <= rank < world) or n_per_rank < 0:
        raise ValueError("bad rank/world/n_per_rank")
    start = first + rank * n_per_rank
    return np.arange(start, start + n_per_rank, dtype=np.uint32)


def split_instances(n_total: int, rank: int, world: int) -> np.ndarray:
    """Instance ids of `rank` when n_total instances are split (strong scaling):
    contiguous blocks whose sizes differ by at most one."""
    if not (0 <= rank < world) or n_total < 0:
        raise ValueError("bad rank/world/n_total")
    base, extra = divmod(n_total, world)
    start = rank * base + min(rank, extra)
    return np.arange(start, start + base + (rank < extra), dtype=np.uint32)


def gather_rows(local: np.ndarray, ids: np.ndarray, group=None):
    """Concatenate per-instance rows from all ranks, ordered by instance id
    (torch.distributed all_gather_object; any backend)."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    parts = [None] * world
    dist.all_gather_object(parts, (np.asarray(ids), np.asarray(local)), group=group)
    all_ids = np.concatenate([p[0] for p in parts])
    rows = np.concatenate([p[1] for p in parts])
    order = np.argsort(all_ids, kind="stable")
    return all_ids[order], rows[order]
