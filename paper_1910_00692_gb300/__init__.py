"""Exact top-k weighted triangles on GB300 (sm_103a).

A thin ctypes binding over ``libwtri.so`` (C ABI in ``include/wtri.h``).  The
binding only marshals arguments: every step of the path runs in the
library's CUDA kernels.  Importing this package does not need a GPU; calling
into it does, and a missing library raises ``WtriUnavailable`` instead of
falling back to anything else.
"""
from __future__ import annotations

from .wtri import (  # noqa: F401
    ARRAYS,
    Graph,
    Server,
    WtriError,
    WtriUnavailable,
    autotune_buckets,
    build_csr,
    debug_set_wait_limit,
    lib,
    lib_path,
    merge_topk,
    sample_cliques,
    sample_edges,
    sample_topk,
    sample_wedges,
    topk,
    topk_batch,
    topk_device,
    topk_device_noalloc,
    topk_shard,
    wedge_topk,
)

__all__ = ["ARRAYS", "Graph", "Server", "WtriError", "WtriUnavailable", "autotune_buckets", "build_csr",
           "debug_set_wait_limit", "lib", "lib_path", "merge_topk", "topk_shard",
           "sample_cliques", "sample_edges", "sample_topk", "sample_wedges", "topk", "topk_batch", "topk_device",
           "topk_device_noalloc", "wedge_topk"]
