"""The paper's dynamic heavy-light algorithm (Algorithm 2) and Auto-HL
(Section 3.3), run on the CPU as the prior-art baseline.

Section 3.2's correctness argument makes the answer independent of the
promotion rule, so every alpha (and Auto-HL) must return exactly what the
brute-force oracle returns: the hand-enumerated fixtures, closed forms on
K_n, random small graphs full of ties, and the tiny and scaled Chung-Lu
workloads.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from golden_io import P_OF, closed_form, load_all

PS = [-math.inf, 0.0, 1.0, 2.0, math.inf]
ALPHAS = [None, 1.0, 3.0, 0.0]  # alpha_p(beta=2), two fixed rules, Auto-HL


def _same(got, want):
    return (got["count"] == want["count"] and np.array_equal(got["tri"], want["tri"])
            and np.array_equal(got["key"], want["key"]) and np.array_equal(got["value"], want["value"]))


def test_alpha_closed_form():
    # alpha_p = 2 - p / (p - 1 + beta)
    assert oracle.dhl_alpha(1.0, 2.0) == pytest.approx(1.5)
    assert oracle.dhl_alpha(2.0, 2.0) == pytest.approx(4.0 / 3.0)
    assert oracle.dhl_alpha(1.0, 3.0) == pytest.approx(5.0 / 3.0)
    assert oracle.dhl_alpha(math.inf, 2.0) == 1.0
    assert oracle.dhl_alpha(-math.inf, 2.0) == 1.0
    assert oracle.dhl_alpha(0.0, 2.0) == 2.0


@pytest.mark.parametrize("fx", load_all(), ids=lambda d: d["name"])
def test_dhl_golden(fx):
    for pname, rows in fx["expected"].items():
        if rows and rows[0][3] is None:
            continue  # fp64-keyed p: the CPU DHL takes the five exact-key p only
        for a in ALPHAS:
            r = oracle.dhl_topk(fx["n"], fx["u"], fx["v"], fx["w"], P_OF[pname], fx["k"], alpha=a)
            assert r["count"] == len(rows)
            for i, row in enumerate(rows):
                assert tuple(int(x) for x in r["tri"][i]) == tuple(row[:3])
                assert int(r["key"][i]) == row[3]
                assert abs(r["value"][i] - closed_form(row[4])) <= 1e-15 * max(1.0, closed_form(row[4]))


@pytest.mark.parametrize("n", [5, 12, 30])
def test_dhl_complete_graph(n):
    # K_n with w(u, v) = u + v: every triple is a triangle; at p = 1 the key
    # of {a, b, c} is 2 (a + b + c), so the top-1 is {n-3, n-2, n-1}
    iu, ju = np.triu_indices(n, 1)
    u, v = iu.astype(np.int32), ju.astype(np.int32)
    w = (u + v).astype(np.int32)
    r = oracle.dhl_topk(n, u, v, w, 1.0, math.comb(n, 3) + 5)
    assert r["count"] == math.comb(n, 3)
    assert tuple(r["tri"][0]) == (n - 3, n - 2, n - 1)
    assert int(r["key"][0]) == 2 * (3 * n - 6)


@pytest.mark.parametrize("n", [5, 300])
def test_dhl_wheel(n):
    # hub n, rim 0..n-1: n triangles {i, i+1, hub}; spokes 2i+2, rim edges 1
    u = np.array(list(range(n)) * 2, np.int32)
    v = np.array([n] * n + [(i + 1) % n for i in range(n)], np.int32)
    w = np.array([2 * i + 2 for i in range(n)] + [1] * n, np.int32)
    tris = [tuple(sorted((i, (i + 1) % n, n))) for i in range(n)]
    key = {t: 2 * t[0] + 2 * t[1] + 5 for t in tris}
    for a in ALPHAS:
        r = oracle.dhl_topk(n + 1, u, v, w, 1.0, n, alpha=a)
        assert [tuple(x) for x in r["tri"]] == sorted(tris, key=lambda t: (-key[t], t))


@pytest.mark.parametrize("seed", range(60))
def test_dhl_random_small(seed):
    g = synth.random_small_graph(6 + seed % 40, 0.15 + 0.8 * ((seed * 37) % 100) / 100, 1 + seed % 9, seed)
    for p in PS:
        k = 1 + (seed * 13) % 40
        want = oracle.topk(g.n, g.u, g.v, g.w, p, k)
        for a in ALPHAS:
            assert _same(oracle.dhl_topk(g.n, g.u, g.v, g.w, p, k, alpha=a), want), (seed, p, a)


@pytest.mark.parametrize("p", PS)
def test_dhl_tiny_workload(p):
    g = synth.tiny_graph(0)
    want = oracle.topk(g.n, g.u, g.v, g.w, p, 100)
    for a in ALPHAS:
        assert _same(oracle.dhl_topk(g.n, g.u, g.v, g.w, p, 100, alpha=a), want), a


def test_dhl_scaled_workload():
    g = synth.scaled_mid_graph(20_000, 200_000, seed=1)
    for p in PS:
        want = oracle.topk(g.n, g.u, g.v, g.w, p, 1000)
        got = oracle.dhl_topk(g.n, g.u, g.v, g.w, p, 1000)
        assert _same(got, want), p
        # the heavy-first stop: far fewer edges reach S u H than the graph has
        if p != -math.inf:
            assert got["stats"]["l"] < g.m // 4


def test_dhl_degenerate():
    empty = np.zeros(0, np.int32)
    assert oracle.dhl_topk(4, empty, empty, empty, 1.0, 3)["count"] == 0
    star_u = np.zeros(5, np.int32)
    star_v = np.arange(1, 6, dtype=np.int32)
    assert oracle.dhl_topk(6, star_u, star_v, star_v, 2.0, 3)["count"] == 0
    # k above the number of triangles returns all of them
    g = synth.tiny_graph(0)
    ntri = oracle.topk(g.n, g.u, g.v, g.w, 1.0, 1)["ntri"]
    r = oracle.dhl_topk(g.n, g.u, g.v, g.w, 1.0, ntri + 100)
    assert r["count"] == ntri


@pytest.mark.parametrize("edges", [
    [(0, 0, 1)],            # self-loop
    [(0, 1, 1), (1, 0, 2)],  # repeated pair
    [(0, 1, 0)],            # weight <= 0
    [(0, 9, 1)],            # id out of range
])
def test_dhl_invalid(edges):
    e = np.array(edges, np.int32)
    with pytest.raises(oracle.OracleError):
        oracle.dhl_topk(4, e[:, 0], e[:, 1], e[:, 2], 1.0, 3)
