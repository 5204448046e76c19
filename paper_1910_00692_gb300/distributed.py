"""Multi-GPU exact top-k: each rank answers one shard of the query on its own
GPU (wtri_topk_shard: the owning edges split into round-robin chunks), then
one all-gather of the k best per shard and a host merge (wtri_merge_topk)
give the global answer.  The graph is replicated on every rank (48 bytes
per edge and 16 per vertex).

The exchange is a single torch.distributed all_gather of one fixed-size
int64 tensor per rank: 1 + 5k words (the count; k vertex triples; k fp64
weights and k 64-bit keys, bit for bit), on the current CUDA device for an
NCCL group and on the host for gloo.  Nothing else crosses ranks.
"""
from __future__ import annotations

import numpy as np

from . import wtri


def pack_part(local_part, k: int) -> np.ndarray:
    """(tris, weights, keys) of one shard -> the 1 + 5k int64 words sent."""
    tris, w, keys = local_part
    cnt = len(w)
    if cnt > k:
        raise ValueError("a shard holds more than k results")
    buf = np.zeros(1 + 5 * k, dtype=np.int64)
    buf[0] = cnt
    buf[1:1 + 3 * cnt] = np.asarray(tris, dtype=np.int64).reshape(-1)[:3 * cnt]
    buf[1 + 3 * k:1 + 3 * k + cnt] = np.asarray(w, dtype=np.float64).view(np.int64)
    buf[1 + 4 * k:1 + 4 * k + cnt] = np.asarray(keys, dtype=np.uint64).view(np.int64)
    return buf


def unpack_part(buf: np.ndarray, k: int):
    cnt = int(buf[0])
    tris = buf[1:1 + 3 * cnt].astype(np.int32).reshape(-1, 3)
    w = buf[1 + 3 * k:1 + 3 * k + cnt].copy().view(np.float64)
    keys = buf[1 + 4 * k:1 + 4 * k + cnt].copy().view(np.uint64)
    return tris, w, keys


def merge_across_ranks(local_part, k: int, group=None):
    """All-gathers each rank's (tris, weights, keys) as one fixed-size tensor
    and merges them on every rank; returns the global (tris, weights, keys)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    nccl = dist.get_backend(group) == "nccl"
    dev = torch.device("cuda", torch.cuda.current_device()) if nccl else torch.device("cpu")
    mine = torch.from_numpy(pack_part(local_part, k)).to(dev)
    parts = [torch.empty_like(mine) for _ in range(world)]
    dist.all_gather(parts, mine, group=group)
    arrays = [unpack_part(t.cpu().numpy(), k) for t in parts]
    return wtri.merge_topk(arrays, k)


def topk_distributed(graph: "wtri.Graph", p: float, k: int, group=None):
    """Exact top-k of a replicated graph, split across the group's ranks."""
    import torch.distributed as dist
    rank = dist.get_rank(group)
    world = dist.get_world_size(group)
    local = wtri.topk_shard(graph, p, k, rank, world)
    return merge_across_ranks(local, k, group)
