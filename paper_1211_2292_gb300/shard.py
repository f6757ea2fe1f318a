"""Sharding of independent systems across ranks (one process per GPU).

The batched workload is many independent systems, so it partitions with no
exchange at all: each rank owns whole systems.  Systems are dealt largest
cost first (cost = N_k^2 pairs) to the rank with the least work so far, the
longest-processing-time rule -- the multi-process analogue of the paper's
dynamic scheduling of uneven work (Sec. V-C, Table VI).  The single-system
workload is not sharded: ranks run independent replicas.
"""
from __future__ import annotations

import heapq

import numpy as np


def shard_systems(sizes, world_size: int, rank: int):
    """Indices (ascending) of the systems rank `rank` owns."""
    sizes = np.asarray(sizes, dtype=np.int64)
    if world_size < 1 or not 0 <= rank < world_size:
        raise ValueError("bad world_size/rank")
    order = sorted(range(sizes.size), key=lambda k: (-int(sizes[k]) ** 2, k))
    heap = [(0, r) for r in range(world_size)]
    owner = np.empty(sizes.size, dtype=np.int64)
    for k in order:
        load, r = heapq.heappop(heap)
        owner[k] = r
        heapq.heappush(heap, (load + int(sizes[k]) ** 2, r))
    return np.flatnonzero(owner == rank)


def gather_rows(offsets, systems):
    """(body indices of the given systems in order, their local offsets)."""
    offsets = np.asarray(offsets, dtype=np.int64)
    parts = [np.arange(offsets[k], offsets[k + 1]) for k in systems]
    idx = np.concatenate(parts) if parts else np.zeros(0, dtype=np.int64)
    local = np.zeros(len(systems) + 1, dtype=np.int64)
    local[1:] = np.cumsum([offsets[k + 1] - offsets[k] for k in systems])
    return idx, local


def max_over_ranks(value: float, dist=None) -> float:
    """The slowest rank's time (the bench's timing rule); identity when alone."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
