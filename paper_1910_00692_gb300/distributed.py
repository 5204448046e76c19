"""Multi-GPU exact top-k: each rank answers one shard of the query on its own
GPU (wtri_topk_shard), then one all-gather of the k best per shard and a
host merge (wtri_merge_topk) give the global answer.  The graph is
replicated on every rank (it fits: 84 bytes per edge).

The exchange step uses torch.distributed (NCCL or gloo, whichever the group
was created with); nothing else crosses ranks.
"""
from __future__ import annotations

from . import wtri


def merge_across_ranks(local_part, k: int, group=None):
    """All-gathers each rank's (tris, weights, keys) and merges them on every
    rank; returns the global (tris, weights, keys)."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    parts = [None] * world
    dist.all_gather_object(parts, tuple(x.tolist() for x in local_part), group=group)
    import numpy as np
    arrays = [(np.array(t, dtype=np.int32).reshape(-1, 3), np.array(w, dtype=np.float64),
               np.array(kk, dtype=np.uint64)) for t, w, kk in parts]
    return wtri.merge_topk(arrays, k)


def topk_distributed(graph: "wtri.Graph", p: float, k: int, group=None):
    """Exact top-k of a replicated graph, split across the group's ranks."""
    import torch.distributed as dist
    rank = dist.get_rank(group)
    world = dist.get_world_size(group)
    local = wtri.topk_shard(graph, p, k, rank, world)
    return merge_across_ranks(local, k, group)
