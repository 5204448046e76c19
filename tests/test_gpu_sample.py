"""GPU weighted edge sampling (Algorithm 3) against the oracle.

The draws are compared bit for bit (same Philox4x64-10 words, same integer
inverse CDF over the edge order), and the top-k of the sampled triangle set
T is compared element by element with the oracle's brute force over T.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from wtri_testutil import assert_topk_equal

pytestmark = pytest.mark.gpu

wt = pytest.importorskip("paper_1910_00692_gb300")


@pytest.fixture(scope="module")
def graphs():
    out = {"tiny": synth.tiny_graph(0), "scaled": synth.scaled_mid_graph(100_000, 1_000_000, seed=12)}
    dev = {k: wt.build_csr(g.n, g.u, g.v, g.w) for k, g in out.items()}
    yield out, dev
    for d in dev.values():
        d.free()


@pytest.mark.parametrize("name", ["tiny", "scaled"])
@pytest.mark.parametrize("p", [1.0, 2.0, 0.0])
@pytest.mark.parametrize("nsamples,seed", [(1, 0), (1000, 7), (200_000, 7), (50_000, 2**64 - 1)])
def test_draws_bit_identical(graphs, name, p, nsamples, seed):
    g, d = graphs[0][name], graphs[1][name]
    _, hits = oracle.sample_edges(g.w, p, nsamples, seed)
    got = wt.sample_edges(d, p, nsamples, seed)
    assert np.array_equal(got, hits > 0)


@pytest.mark.parametrize("name", ["tiny", "scaled"])
@pytest.mark.parametrize("p", [1.0, 2.0, 0.0])
@pytest.mark.parametrize("k,nsamples", [(10, 500), (100, 20_000), (1000, 300_000)])
def test_sample_topk_vs_oracle(graphs, name, p, k, nsamples):
    g, d = graphs[0][name], graphs[1][name]
    want = oracle.sample_topk(g.n, g.u, g.v, g.w, p, k, nsamples, 7)
    tris, wts = d.sample_topk(p, k, nsamples, 7)
    assert_topk_equal(tris, wts, want, p, f"{name} p={p} k={k} s={nsamples}")


def test_sample_errors(graphs):
    d = graphs[1]["tiny"]
    for p in (math.inf, -math.inf, -1.0, 3.0):
        with pytest.raises(wt.WtriError) as ei:
            d.sample_topk(p, 10, 100, 1)
        assert ei.value.code == -5
    with pytest.raises(wt.WtriError) as ei:
        d.sample_topk(1.0, 10, -1, 1)
    assert ei.value.code == -1
    tris, _ = d.sample_topk(1.0, 10, 0, 1)
    assert tris.shape[0] == 0


def test_sample_mid_full():
    """Full mid graph (n=1e6, m=2e7): 1e6 draws, top-1000 of T equals the
    oracle's; recall against the exact top-1000 is reported."""
    g = synth.mid_graph(1)
    d = wt.build_csr(g.n, g.u, g.v, g.w)
    try:
        want = oracle.sample_topk(g.n, g.u, g.v, g.w, 1.0, 1000, 1_000_000, 7)
        tris, wts = d.sample_topk(1.0, 1000, 1_000_000, 7)
        assert_topk_equal(tris, wts, want, 1.0, "mid sample")
        exact = oracle.topk(g.n, g.u, g.v, g.w, 1.0, 1000)
        recall = len(set(map(tuple, exact["tri"].tolist())) & set(map(tuple, tris.tolist()))) / 1000
        print(f"mid ES recall@1000 with 1e6 draws: {recall:.3f}")
    finally:
        d.free()
