"""Pins of the clique oracle (Section 4.5, Appendix A: a clique weighs the
p-mean of its edge weights): closed forms on K_n, clique counts from
networkx's independent enumeration, and a brute force over every vertex
subset on tiny graphs full of ties."""
import itertools
import math

import numpy as np
import pytest

import oracle
import synth

PS = [-math.inf, 1.0, 2.0, math.inf]


def _kn(n):
    iu, ju = np.triu_indices(n, 1)
    u, v = iu.astype(np.int32), ju.astype(np.int32)
    return u, v, (u + v).astype(np.int32)


@pytest.mark.parametrize("q", [4, 5])
@pytest.mark.parametrize("n", [5, 8, 13])
def test_complete_graph_closed_forms(n, q):
    u, v, w = _kn(n)
    top = tuple(range(n - q, n))
    # every q-subset is a clique
    r = oracle.clique_topk(n, u, v, w, q, 1.0, 1)
    assert r["ncliques"] == math.comb(n, q)
    # p = 1: each vertex lies on q - 1 edges of the clique, so the sum of the
    # edge weights u + v is (q - 1) times the sum of the ids: the q largest ids win
    assert tuple(r["ids"][0]) == top and int(r["key"][0]) == (q - 1) * sum(top)
    assert r["value"][0] == (q - 1) * sum(top) / (q * (q - 1) / 2)
    # p = -inf: the lightest edge joins the two smallest ids
    r = oracle.clique_topk(n, u, v, w, q, -math.inf, 1)
    assert tuple(r["ids"][0]) == top and int(r["key"][0]) == 2 * (n - q) + 1
    # p = +inf: every clique holding n-2 and n-1 ties at 2n - 3; the tuple
    # order puts the smallest other ids first
    r = oracle.clique_topk(n, u, v, w, q, math.inf, 2)
    assert tuple(r["ids"][0]) == tuple(range(q - 2)) + (n - 2, n - 1)
    assert int(r["key"][0]) == 2 * n - 3
    # p = 2: the q largest ids (u + v grows with both ids)
    r = oracle.clique_topk(n, u, v, w, q, 2.0, 1)
    assert tuple(r["ids"][0]) == top


@pytest.mark.parametrize("seed", range(6))
def test_counts_match_networkx(seed):
    nx = pytest.importorskip("networkx")
    g = synth.random_small_graph(12 + 3 * seed, 0.5 + 0.05 * seed, 5, seed)
    G = nx.Graph()
    G.add_nodes_from(range(g.n))
    G.add_edges_from(zip(g.u.tolist(), g.v.tolist()))
    sizes = [len(c) for c in nx.enumerate_all_cliques(G)]
    for q in (4, 5):
        r = oracle.clique_topk(g.n, g.u, g.v, g.w, q, 1.0, 1)
        assert r["ncliques"] == sizes.count(q)


def _brute(n, u, v, w, q, p, flags=None):
    wt = {}
    eid = {}
    for i, (a, b, c) in enumerate(zip(u.tolist(), v.tolist(), w.tolist())):
        wt[(min(a, b), max(a, b))] = c
        eid[(min(a, b), max(a, b))] = i
    out = []
    for s in itertools.combinations(range(n), q):
        pairs = list(itertools.combinations(s, 2))
        if not all(pr in wt for pr in pairs):
            continue
        if flags is not None and not any(flags[eid[pr]] for pr in pairs):
            continue
        ws = [wt[pr] for pr in pairs]
        if p == 1.0:
            key, val = sum(ws), sum(ws) / len(ws)
        elif p == 2.0:
            key = sum(x * x for x in ws)
            val = math.sqrt(key / len(ws))
        elif p == math.inf:
            key = val = max(ws)
        else:
            key = val = min(ws)
        out.append((-key, s, val))
    out.sort()
    return out


@pytest.mark.parametrize("seed", range(10))
@pytest.mark.parametrize("q", [4, 5])
def test_brute_force_with_ties(seed, q):
    g = synth.random_small_graph(9 + seed % 5, 0.55 + 0.04 * seed, 3, seed)
    for p in PS:
        want = _brute(g.n, g.u, g.v, g.w, q, p)
        for k in (1, 5, 1000):
            r = oracle.clique_topk(g.n, g.u, g.v, g.w, q, p, k)
            exp = want[:k]
            assert r["count"] == len(exp) and r["ncliques"] == len(want)
            assert [tuple(int(x) for x in t) for t in r["ids"]] == [e[1] for e in exp]
            assert [int(x) for x in r["key"]] == [-e[0] for e in exp]
            assert [float(x) for x in r["value"]] == [e[2] for e in exp]


@pytest.mark.parametrize("seed", range(5))
def test_sampled_set_is_the_cliques_on_sampled_edges(seed):
    g = synth.random_small_graph(13, 0.6, 4, 100 + seed)
    rng = np.random.default_rng(seed)
    flags = (rng.random(g.m) < 0.2).astype(np.uint8)
    for q in (4, 5):
        for p in (1.0, 2.0):
            want = _brute(g.n, g.u, g.v, g.w, q, p, flags)
            r = oracle.clique_topk(g.n, g.u, g.v, g.w, q, p, 10_000, edge_sampled=flags)
            assert r["ncliques"] == len(want)
            assert [tuple(int(x) for x in t) for t in r["ids"]] == [e[1] for e in want]


def test_sampled_flags_follow_the_draws():
    g = synth.random_small_graph(20, 0.4, 9, 3)
    flags = oracle.sampled_edge_flags(g.w, 1.0, 50, 11)
    perm, hits = oracle.sample_edges(g.w, 1.0, 50, 11)
    assert flags.sum() == (hits > 0).sum() and flags[perm[hits > 0]].all()


def test_invalid():
    u, v, w = _kn(6)
    for q in (3, 6):
        with pytest.raises(oracle.OracleError):
            oracle.clique_topk(6, u, v, w, q, 1.0, 3)
    for p in (0.0, -1.0, 3.0):
        with pytest.raises(oracle.OracleError):
            oracle.clique_topk(6, u, v, w, 4, p, 3)
    big = w.copy()
    big[0] = oracle.CLIQUE_P2_WMAX + 1
    with pytest.raises(oracle.OracleError):
        oracle.clique_topk(6, u, v, big, 4, 2.0, 3)
    oracle.clique_topk(6, u, v, big, 4, 1.0, 3)  # the sum still fits
