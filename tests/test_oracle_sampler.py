"""Pins for the oracle's weighted edge sampler (Algorithm 3, Proposition 4.1,
Section 4.1), independent of the oracle's own code:

* Philox4x64-10 words equal numpy's Philox bit generator (a library run);
* the draw frequencies of edges match w^p / Z (chi-square);
* the triangle set T for hand-chosen marked edges on a bowtie;
* an independent Python sampler (numpy Philox + Python integer CDF) with an
  itertools brute force gives the same top-k of T;
* T only grows with more samples (the s-th sample uses counter s), so recall
  of the exact top-k is monotone in the sample count (Section 4.4).
"""
import itertools
import math

import numpy as np
import pytest

import oracle
import synth


def numpy_philox_block(s, seed):
    # numpy's generator emits the block of counter+1 first.
    bg = np.random.Philox(counter=(s - 1) % (1 << 256), key=np.array([seed, 0], dtype=np.uint64))
    return bg.random_raw(4)


@pytest.mark.parametrize("s,seed", [(0, 0), (1, 7), (2, 7), (12345, 99), (2**40 + 3, 2**63 + 5)])
def test_philox_matches_numpy(s, seed):
    mine = oracle.philox4x64_10([s, 0, 0, 0], [seed, 0])
    assert np.array_equal(mine, numpy_philox_block(s, seed))


@pytest.mark.parametrize("p", [1.0, 2.0, 0.0])
def test_edge_draws_follow_w_to_the_p(p):
    stats = pytest.importorskip("scipy.stats")
    w = np.array([1, 2, 3, 5, 8, 13, 21, 1, 1, 4, 30, 7], np.int32)
    perm, hits = oracle.sample_edges(w, p, 400_000, 11)
    wp = w[perm].astype(np.float64) ** p
    expect = wp / wp.sum() * hits.sum()
    chi = stats.chisquare(hits, expect)
    assert chi.pvalue > 1e-4, chi
    assert hits.sum() == 400_000


def test_marked_set_on_bowtie():
    # bowtie: 012 weights (2,2,2), 034 weights (1,6,1); edges in input order
    u = np.array([0, 1, 2, 0, 4, 0], np.int32)
    v = np.array([1, 2, 0, 3, 3, 4], np.int32)
    w = np.array([2, 2, 2, 1, 6, 1], np.int32)
    none = oracle.topk_of_marked(5, u, v, w, np.zeros(6, np.uint8), 1.0, 10)
    assert none["count"] == 0
    only34 = oracle.topk_of_marked(5, u, v, w, np.array([0, 0, 0, 0, 1, 0], np.uint8), 1.0, 10)
    assert only34["tri"].tolist() == [[0, 3, 4]] and only34["key"].tolist() == [8]
    only01 = oracle.topk_of_marked(5, u, v, w, np.array([1, 0, 0, 0, 0, 0], np.uint8), 2.0, 10)
    assert only01["tri"].tolist() == [[0, 1, 2]] and only01["key"].tolist() == [12]
    both = oracle.topk_of_marked(5, u, v, w, np.array([0, 0, 1, 1, 0, 0], np.uint8), 1.0, 10)
    assert both["tri"].tolist() == [[0, 3, 4], [0, 1, 2]]


def _python_sample_topk(n, u, v, w, p, k, nsamples, seed):
    m = len(u)
    order = sorted(range(m), key=lambda i: (-int(w[i]), i))
    C, acc = [], 0
    for i in order:
        acc += int(w[i]) ** int(p)
        C.append(acc)
    Z = acc
    marked = set()
    bg_first = None
    for s in range(nsamples):
        x = int(numpy_philox_block(s, seed)[0])
        t = (x * Z) >> 64
        lo, hi = 0, m
        while lo < hi:
            mid = (lo + hi) // 2
            if C[mid] > t:
                hi = mid
            else:
                lo = mid + 1
        marked.add(order[lo])
    del bg_first
    adj = {}
    for i, (a, b) in enumerate(zip(u.tolist(), v.tolist())):
        adj[(min(a, b), max(a, b))] = i
    out = []
    for a, b, c in itertools.combinations(range(n), 3):
        e = [adj.get((a, b)), adj.get((b, c)), adj.get((a, c))]
        if None in e or not any(x in marked for x in e):
            continue
        ws = [int(w[x]) for x in e]
        key = sum(ws) if p == 1.0 else sum(x * x for x in ws)
        out.append((key, (a, b, c)))
    out.sort(key=lambda t: (-t[0], t[1]))
    return out[:k]


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("p", [1.0, 2.0])
def test_sampled_topk_matches_python(seed, p):
    g = synth.random_small_graph(28, 0.35, 9, 500 + seed)
    nsamples = 25
    want = _python_sample_topk(g.n, g.u, g.v, g.w, p, 40, nsamples, seed)
    got = oracle.sample_topk(g.n, g.u, g.v, g.w, p, 40, nsamples, seed)
    assert [(int(k_), tuple(int(x) for x in t)) for k_, t in zip(got["key"], got["tri"])] == want


def test_recall_monotone_in_samples():
    g = synth.tiny_graph(0)
    exact = oracle.topk(g.n, g.u, g.v, g.w, 1.0, 100)
    ref = set(map(tuple, exact["tri"].tolist()))
    prev = -1.0
    for ns in (100, 1000, 10_000, 100_000, 400_000):
        r = oracle.sample_topk(g.n, g.u, g.v, g.w, 1.0, 100, ns, 7)
        got = set(map(tuple, r["tri"].tolist()))
        # T grows with ns; recall of the exact top-k counts exact members found
        # anywhere in the sampled top-k list
        recall = len(ref & got) / 100.0
        assert recall >= prev - 1e-12
        prev = recall
    assert prev >= 0.9
