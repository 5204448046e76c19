"""Pins for the oracle's weighted wedge sampler (Algorithm 4, Eqs. 6-8,
Proposition 4.2, Section 4.2), independent of its own code.

Reading of Proposition 4.2: an iteration draws a center a, then b and c in
N(a) one after the other, so each unordered wedge {ab, ac} arises in two
orders and an iteration closes triangle {a, b, c} with probability
2 w_p(a,b,c) / Z~, Z~ = sum_v d_v D(v), not w_p / Z~ as printed (the proof
counts one order of each wedge).  On a triangle with unit weights the
closing probability is exactly 1/2 (a hand count: a is any vertex, c must
differ from b, each of the two neighbours equally likely), which the first
pin checks; the printed form would give 1/4.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
import synth
from golden_io import load_all


def _adj(n, u, v, w):
    nb = [dict() for _ in range(n)]
    for a, b, x in zip(u.tolist(), v.tolist(), w.tolist()):
        nb[a][b] = x
        nb[b][a] = x
    return nb


def test_unit_triangle_closes_half_the_time():
    u = np.array([0, 1, 0], np.int32)
    v = np.array([1, 2, 2], np.int32)
    w = np.ones(3, np.int32)
    for p in (0.0, 1.0, 2.0):
        _, _, _, tri = oracle.wedge_samples(3, u, v, w, p, 200_000, 3)
        hits = int((tri[:, 0] >= 0).sum())
        # binomial(200000, 1/2): 4.5 standard deviations = 1006
        assert abs(hits - 100_000) < 1006, (p, hits)


@pytest.mark.parametrize("p", [0.0, 1.0, 2.0])
def test_ordered_wedge_law(p):
    """Eqs. 6-8 jointly: an ordered draw (a, b, c) with b, c in N(a) (b = c
    allowed) has probability (w_ab^p + w_ac^p) / Z1, Z1 = sum_v 2 d_v D(v).
    Chi-square over every (a, b, c) of a small weighted graph."""
    stats = pytest.importorskip("scipy.stats")
    # a triangle with a pendant path and a hub, distinct weights
    edges = [(0, 1, 3), (1, 2, 1), (0, 2, 2), (2, 3, 4), (3, 4, 1), (0, 5, 2), (0, 6, 1), (2, 6, 5)]
    e = np.array(edges, np.int32)
    n = 7
    u, v, w = e[:, 0], e[:, 1], e[:, 2]
    nb = _adj(n, u, v, w)
    wp = lambda x: float(x) ** p  # noqa: E731
    Z1 = sum(2 * len(nb[a]) * sum(wp(x) for x in nb[a].values()) for a in range(n))
    # the oracle reports b and c as positions in a's weight-sorted row
    order = np.argsort(-w, kind="stable")
    rows = [[] for _ in range(n)]
    for r in order:
        rows[u[r]].append(int(v[r]))
        rows[v[r]].append(int(u[r]))
    cells, expect = [], []
    for a in range(n):
        for jb, b in enumerate(rows[a]):
            for jc, c in enumerate(rows[a]):
                cells.append((a, jb, jc))
                expect.append((wp(nb[a][b]) + wp(nb[a][c])) / Z1)
    ns = 300_000
    center, jb, jc, _ = oracle.wedge_samples(n, u, v, w, p, ns, 17)
    idx = {c: i for i, c in enumerate(cells)}
    counts = np.zeros(len(cells))
    for a, x, y in zip(center.tolist(), jb.tolist(), jc.tolist()):
        counts[idx[(a, x, y)]] += 1
    expect = np.array(expect) * ns
    assert abs(expect.sum() - ns) < 1e-6 * ns
    chi = stats.chisquare(counts, expect)
    assert chi.pvalue > 1e-4, chi


def test_triangle_probability_reading():
    """Per-iteration closing probability of each triangle = 2 w_p / Z~
    (Proposition 4.2 as read above), by chi-square on a graph with several
    triangles of different weights."""
    stats = pytest.importorskip("scipy.stats")
    fx = [f for f in load_all() if f["name"] == "k4_distinct.json"][0]
    n, u, v, w = fx["n"], fx["u"], fx["v"], fx["w"]
    nb = _adj(n, u, v, w)
    p = 1.0
    Zt = sum(len(nb[a]) * sum(nb[a].values()) for a in range(n))
    tris = [t for t in itertools.combinations(range(n), 3)]
    probs = [2 * (nb[a][b] + nb[b][c] + nb[a][c]) / Zt for a, b, c in tris]
    ns = 400_000
    _, _, _, tri = oracle.wedge_samples(n, u, v, w, p, ns, 5)
    counts = [int(np.all(tri == np.array(t), axis=1).sum()) for t in tris]
    openc = ns - sum(counts)
    chi = stats.chisquare(counts + [openc], [q * ns for q in probs] + [(1 - sum(probs)) * ns])
    assert chi.pvalue > 1e-4, chi


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("p", [0.0, 1.0, 2.0])
def test_wedge_topk_is_topk_of_closed_set(seed, p):
    """The top-k is the exact top-k (by Eq. 1's keys) of the distinct closed
    triangles the draws produced, computed here in Python."""
    g = synth.random_small_graph(25 + seed, 0.4, 6, seed)
    if g.m == 0:
        return
    nb = _adj(g.n, g.u, g.v, g.w)
    _, _, _, tri = oracle.wedge_samples(g.n, g.u, g.v, g.w, p, 3000, 9 + seed)
    closed = sorted({tuple(t) for t in tri.tolist() if t[0] >= 0})

    def key(t):
        a, b, c = t
        ws = [nb[a][b], nb[b][c], nb[a][c]]
        return {0.0: ws[0] * ws[1] * ws[2], 1.0: sum(ws), 2.0: sum(x * x for x in ws)}[p]
    want = sorted(closed, key=lambda t: (-key(t), t))[:15]
    r = oracle.wedge_topk(g.n, g.u, g.v, g.w, p, 15, 3000, 9 + seed)
    assert r["ntri"] == len(closed)
    assert [tuple(int(x) for x in t) for t in r["tri"]] == want


def test_wedge_more_samples_find_more():
    g = synth.tiny_graph(0)
    prev = -1
    for ns in (1000, 10_000, 100_000):
        r = oracle.wedge_topk(g.n, g.u, g.v, g.w, 1.0, 100, ns, 1)
        assert r["ntri"] >= prev
        prev = r["ntri"]
    assert prev > 0
