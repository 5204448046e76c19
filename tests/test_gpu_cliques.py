"""Top weighted 4- and 5-cliques on the GPU (Section 4.5, Appendix A)
against the oracle: the exact mode (every edge) and edge sampling (the
oracle's cliques on the edges Algorithm 3's draws select), element by
element (ids, keys, fp64 weights)."""
import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

wt = pytest.importorskip("paper_1910_00692_gb300")

PS = [-math.inf, 1.0, 2.0, math.inf]


def _same(got, want, ctx):
    ids, w, kk = got
    assert ids.shape[0] == want["count"], f"{ctx}: count {ids.shape[0]} != {want['count']}"
    assert np.array_equal(ids, want["ids"]), ctx
    assert np.array_equal(kk, want["key"]), ctx
    assert np.array_equal(w, want["value"]), ctx


@pytest.fixture(scope="module")
def dense():
    g = synth.clique_graph(243, 8300)
    d = wt.build_csr(g.n, g.u, g.v, g.w)
    yield g, d
    d.free()


@pytest.mark.parametrize("q", [4, 5])
def test_exact_vs_oracle_ties(q):
    """Small dense graphs with weights 1..4 (ties everywhere): the exact mode
    equals the oracle's full top-k at every p and k."""
    for seed in range(3):
        g = synth.random_small_graph(40 + 10 * seed, 0.45, 4, 200 + seed)
        d = wt.build_csr(g.n, g.u, g.v, g.w)
        try:
            for p in PS:
                for k in (1, 37, 5000):
                    want = oracle.clique_topk(g.n, g.u, g.v, g.w, q, p, k)
                    _same(wt.sample_cliques(d, q, p, k, -1, 0), want, f"seed={seed} q={q} p={p} k={k}")
        finally:
            d.free()


@pytest.mark.parametrize("q", [4, 5])
def test_exact_dense_graph(dense, q):
    g, d = dense
    for p in PS:
        want = oracle.clique_topk(g.n, g.u, g.v, g.w, q, p, 1000)
        _same(wt.sample_cliques(d, q, p, 1000, -1, 0), want, f"dense q={q} p={p}")


@pytest.mark.parametrize("q", [4, 5])
@pytest.mark.parametrize("p", [1.0, 2.0])
@pytest.mark.parametrize("nsamples,seed", [(200, 1), (3000, 2), (40000, 3)])
def test_sampled_vs_oracle(dense, q, p, nsamples, seed):
    """Edge sampling: the draws are the sampler's (seeded Philox), the
    cliques those with a drawn edge; equal to the oracle over the same set."""
    g, d = dense
    flags = oracle.sampled_edge_flags(g.w, p, nsamples, seed)
    want = oracle.clique_topk(g.n, g.u, g.v, g.w, q, p, 500, edge_sampled=flags)
    _same(wt.sample_cliques(d, q, p, 500, nsamples, seed), want, f"q={q} p={p} s={nsamples}")


def test_complete_graph():
    n = 30
    iu, ju = np.triu_indices(n, 1)
    u, v = iu.astype(np.int32), ju.astype(np.int32)
    w = (u + v).astype(np.int32)
    d = wt.build_csr(n, u, v, w)
    try:
        for q in (4, 5):
            ids, ws, kk = wt.sample_cliques(d, q, 1.0, 3, -1, 0)
            assert tuple(ids[0]) == tuple(range(n - q, n))
            assert int(kk[0]) == (q - 1) * sum(range(n - q, n))
            want = oracle.clique_topk(n, u, v, w, q, math.inf, 200)
            _same(wt.sample_cliques(d, q, math.inf, 200, -1, 0), want, f"K30 q={q} +inf")
    finally:
        d.free()


def test_moderate_graph_5_cliques():
    """The email-Eu-sized stand-in (979 vertices, 29,000 edges, 1.8M
    5-cliques): exact mode and a 20,000-draw sample against the oracle."""
    g = synth.clique_graph(979, 29000)
    d = wt.build_csr(g.n, g.u, g.v, g.w)
    try:
        want = oracle.clique_topk(g.n, g.u, g.v, g.w, 5, 1.0, 2000)
        _same(wt.sample_cliques(d, 5, 1.0, 2000, -1, 0), want, "979/29000 exact")
        flags = oracle.sampled_edge_flags(g.w, 1.0, 20000, 9)
        want = oracle.clique_topk(g.n, g.u, g.v, g.w, 5, 1.0, 2000, edge_sampled=flags)
        _same(wt.sample_cliques(d, 5, 1.0, 2000, 20000, 9), want, "979/29000 sampled")
    finally:
        d.free()


def test_errors(dense):
    g, d = dense
    for args, code in [((3, 1.0, 10, -1), -1), ((4, 0.0, 10, -1), -5), ((4, -1.0, 10, -1), -5),
                       ((4, math.inf, 10, 100), -5), ((4, 1.0, 0, -1), -1), ((4, 1.0, 70000, -1), -1)]:
        with pytest.raises(wt.WtriError) as ei:
            wt.sample_cliques(d, *args, 0)
        assert ei.value.code == code, args
    # an edge whose endpoints share 1,100 neighbours: above the shared-memory list
    leaves = np.arange(2, 1102, dtype=np.int32)
    u = np.concatenate([[0], np.zeros(1100, np.int32), np.ones(1100, np.int32)]).astype(np.int32)
    v = np.concatenate([[1], leaves, leaves]).astype(np.int32)
    dd = wt.build_csr(1102, u, v, np.ones(u.shape[0], np.int32))
    try:
        with pytest.raises(wt.WtriError) as ei:
            wt.sample_cliques(dd, 4, 1.0, 10, -1, 0)
        assert ei.value.code == -5
    finally:
        dd.free()
