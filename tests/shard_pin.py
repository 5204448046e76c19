"""Hand-built graph that pins the shard ownership rule of the split query.

Rule: edges are dealt to shards by their position r in the edge order
(weight descending, input index ascending) in chunks of 1024 positions,
round-robin: chunk c = r // 1024 belongs to shard c % nshards.  A triangle
belongs to the shard that owns its FIRST edge in the edge order.

The graph has 2208 edges with distinct weights 5000 - r, so the edge at
position r is the one of weight 5000 - r.  Five triangles have their edges
at chosen positions; every other position holds an edge of a perfect
matching on fresh vertices (no triangles):

  triangle     positions of its edges   first edge -> chunk
  {0, 1, 2}    0, 2200, 2201            0
  {3, 4, 5}    1500, 2202, 2203         1
  {6, 7, 8}    2100, 2204, 2205         2
  {9, 10, 11}  1023, 1024, 2206         0
  {12, 13, 14} 1025, 1026, 2207         1

Expected triangles per shard (written out by hand from the chunks above):
  2 shards: shard 0 {0,1,2} {6,7,8} {9,10,11}; shard 1 {3,4,5} {12,13,14}
  3 shards: shard 0 {0,1,2} {9,10,11}; shard 1 {3,4,5} {12,13,14}; shard 2 {6,7,8}
A rule that gave a triangle to its last edge's shard would move {0,1,2}
(last edge at 2201, chunk 2) and fail the 3-shard case.
"""
import numpy as np

M = 2208
TRIANGLE_EDGES = {
    (0, 1, 2): [(0, 1, 0), (1, 2, 2200), (0, 2, 2201)],
    (3, 4, 5): [(3, 4, 1500), (4, 5, 2202), (3, 5, 2203)],
    (6, 7, 8): [(6, 7, 2100), (7, 8, 2204), (6, 8, 2205)],
    (9, 10, 11): [(9, 10, 1023), (10, 11, 1024), (9, 11, 2206)],
    (12, 13, 14): [(12, 13, 1025), (13, 14, 1026), (12, 14, 2207)],
}
EXPECTED = {
    2: {0: [(0, 1, 2), (6, 7, 8), (9, 10, 11)], 1: [(3, 4, 5), (12, 13, 14)]},
    3: {0: [(0, 1, 2), (9, 10, 11)], 1: [(3, 4, 5), (12, 13, 14)], 2: [(6, 7, 8)]},
}


def graph():
    """(n, u, v, w): edge i of the arrays sits at edge-order position pos[i];
    the arrays are shuffled so that input order says nothing."""
    u = np.full(M, -1, np.int64)
    v = np.full(M, -1, np.int64)
    for edges in TRIANGLE_EDGES.values():
        for a, b, r in edges:
            u[r], v[r] = a, b
    nxt = 100
    for r in range(M):
        if u[r] < 0:
            u[r], v[r] = nxt, nxt + 1
            nxt += 2
    w = 5000 - np.arange(M)
    perm = np.random.default_rng(5).permutation(M)
    return int(nxt), u[perm].astype(np.int32), v[perm].astype(np.int32), w[perm].astype(np.int32)
