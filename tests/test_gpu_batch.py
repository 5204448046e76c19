"""Batched exact top-k (wtri_topk_batch) against the oracle, query by query.

The batch mixes graphs of very different sizes (n log-uniform, as in the
batch workload but with a smaller upper end so that the oracle finishes in
seconds), per-query p and k, an empty graph, a triangle-free graph and one
graph queried at every supported p (including p = 0).
"""
import math

import numpy as np
import pytest

import oracle
import synth
from wtri_testutil import assert_topk_equal

pytestmark = pytest.mark.gpu

wt = pytest.importorskip("paper_1910_00692_gb300")


def test_batch_vs_oracle():
    graphs = [synth.batch_graph(i, seed=3, n_hi=8000) for i in range(96)]
    ps, ks = synth.batch_queries(len(graphs), seed=3)
    ps, ks = list(ps), list(ks)
    # degenerate members: empty graph, triangle-free star, one graph at all p
    graphs.append(synth.Graph(7, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int32)))
    ps.append(1.0)
    ks.append(5)
    graphs.append(synth.Graph(6, np.zeros(5, np.int32), np.arange(1, 6, dtype=np.int32),
                              np.arange(1, 6, dtype=np.int32)))
    ps.append(2.0)
    ks.append(3)
    for p in (-math.inf, 0.0, 1.0, 2.0, math.inf):
        graphs.append(graphs[5])
        ps.append(p)
        ks.append(777)
    dev = {}
    handles = []
    for g in graphs:
        if id(g) not in dev:
            dev[id(g)] = wt.build_csr(g.n, g.u, g.v, g.w)
        handles.append(dev[id(g)])
    try:
        for rep in range(2):
            res = wt.topk_batch(handles, ps, ks)
            for i, (g, p, k) in enumerate(zip(graphs, ps, ks)):
                want = oracle.topk(g.n, g.u, g.v, g.w, p, int(k))
                assert_topk_equal(res[i][0], res[i][1], want, p, f"rep={rep} query {i} n={g.n} p={p} k={k}")
    finally:
        for d in dev.values():
            d.free()


def test_batch_matches_plain_calls():
    graphs = [synth.batch_graph(i, seed=4, n_hi=30000) for i in range(40)]
    ps, ks = synth.batch_queries(len(graphs), seed=4)
    handles = [wt.build_csr(g.n, g.u, g.v, g.w) for g in graphs]
    try:
        res = wt.topk_batch(handles, ps, ks)
        for i, h in enumerate(handles):
            t, w = h.topk(ps[i], int(ks[i]))
            assert np.array_equal(res[i][0], t), i
            assert np.array_equal(res[i][1], w), i
    finally:
        for h in handles:
            h.free()


def test_batch_errors():
    g = synth.tiny_graph(0)
    d = wt.build_csr(g.n, g.u, g.v, g.w)
    try:
        with pytest.raises(wt.WtriError) as ei:
            wt.topk_batch([d, d], [1.0, 0.5], [10, 10])
        assert ei.value.code == -5
        with pytest.raises(wt.WtriError) as ei:
            wt.topk_batch([d], [1.0], [0])
        assert ei.value.code == -1
        assert wt.topk_batch([], [], []) == []
    finally:
        d.free()
