"""GPU shards of one query (the multi-GPU split, run here one after another
on one GPU): each shard equals the oracle's top-k of the triangles it owns,
and the merged shards equal the whole query."""
import math

import numpy as np
import pytest

import oracle
import synth
from wtri_testutil import PS, assert_topk_equal

pytestmark = pytest.mark.gpu

wt = pytest.importorskip("paper_1910_00692_gb300")


@pytest.mark.parametrize("n,m,seed", [(2000, 20000, 0), (100000, 1000000, 12)])
@pytest.mark.parametrize("nshards", [2, 3])
def test_shards(n, m, seed, nshards):
    g = synth.tiny_graph(0) if n == 2000 else synth.scaled_mid_graph(n, m, seed=seed)
    d = wt.build_csr(g.n, g.u, g.v, g.w)
    try:
        for p in PS:
            k = 500
            parts = []
            for sh in range(nshards):
                t, w, kk = wt.topk_shard(d, p, k, sh, nshards)
                want = oracle.topk_shard(g.n, g.u, g.v, g.w, p, k, sh, nshards)
                assert_topk_equal(t, w, want, p, f"shard {sh}/{nshards} p={p}")
                assert np.array_equal(kk, want["key"])
                parts.append((t, w, kk))
            mt, mw, mk = wt.merge_topk(parts, k)
            ft, fw = d.topk(p, k)
            assert np.array_equal(mt, ft) and np.array_equal(mw, fw)
    finally:
        d.free()
