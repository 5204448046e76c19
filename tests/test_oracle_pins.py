"""Pins for the CPU oracle against facts fixed by the paper and by
mathematics, independent of the oracle's own code:

* closed forms on complete graphs (C(n,3) triangles; K_n with w(u,v)=u+v);
* an independent triangle count, trace(A^3)/6 with a BLAS matmul;
* hand-enumerated graphs in tests/golden/ (Eq. 1 worked by hand);
* a Python itertools brute force over vertex triples on random small graphs;
* invariants (sorted output, prefix property, relabelling).
"""
import itertools
import math

import numpy as np
import pytest

import oracle
import synth
from golden_io import P_OF, closed_form, load_all

PS = [-math.inf, 0.0, 1.0, 2.0, math.inf]


def complete_graph(n, wfun):
    iu, ju = np.triu_indices(n, 1)
    w = np.array([wfun(a, b) for a, b in zip(iu, ju)], dtype=np.int32)
    return iu.astype(np.int32), ju.astype(np.int32), w


@pytest.mark.parametrize("n", [3, 4, 5, 7, 12, 31, 60])
def test_complete_graph_counts(n):
    u, v, w = complete_graph(n, lambda a, b: 1 + (a * 7 + b * 3) % 11)
    expect = n * (n - 1) * (n - 2) // 6
    assert oracle.count_triangles(n, u, v, w) == expect
    for p in PS:
        r = oracle.topk(n, u, v, w, p, 5)
        assert r["ntri"] == expect
        assert r["count"] == min(5, expect)


@pytest.mark.parametrize("n", [4, 9, 16])
def test_complete_graph_sum_weights_closed_form(n):
    # w(u,v) = u + v: each vertex of {a<b<c} lies on two of its edges, so the
    # p=1 key is 2(a+b+c); the max edge is b+c and the min edge is a+b.
    u, v, w = complete_graph(n, lambda a, b: a + b + 1)  # +1 keeps weights positive
    triples = list(itertools.combinations(range(n), 3))
    N = len(triples)
    want = {
        1.0: sorted(triples, key=lambda t: (-(2 * sum(t) + 3), t)),
        math.inf: sorted(triples, key=lambda t: (-(t[1] + t[2] + 1), t)),
        -math.inf: sorted(triples, key=lambda t: (-(t[0] + t[1] + 1), t)),
    }
    for p, order in want.items():
        r = oracle.topk(n, u, v, w, p, N)
        assert r["count"] == N
        assert [tuple(x) for x in r["tri"]] == order
        # max edge b+c ties across every a < n-2, so +inf starts at a = 0
        top = (0, n - 2, n - 1) if p == math.inf else (n - 3, n - 2, n - 1)
        assert tuple(r["tri"][0]) == top
    r = oracle.topk(n, u, v, w, 1.0, N)
    assert [int(x) for x in r["key"]] == [2 * sum(t) + 3 for t in want[1.0]]
    r2 = oracle.topk(n, u, v, w, 2.0, 1)
    assert tuple(r2["tri"][0]) == (n - 3, n - 2, n - 1)
    # p = 0: key (a+b+1)(a+c+1)(b+c+1), the full order by that product
    geo = sorted(triples, key=lambda t: (-(t[0] + t[1] + 1) * (t[0] + t[2] + 1) * (t[1] + t[2] + 1), t))
    r0 = oracle.topk(n, u, v, w, 0.0, N)
    assert [tuple(x) for x in r0["tri"]] == geo
    assert tuple(r0["tri"][0]) == (n - 3, n - 2, n - 1)


@pytest.mark.parametrize("n", [5, 17, 300])
def test_wheel_closed_form(n):
    """Wheel: hub h = n joined to rim vertices 0..n-1, rim cycle i -- i+1
    (mod n).  Exactly n triangles {i, i+1, hub}.  Spokes weigh 2 i + 2 and rim
    edges 1, so triangle {i, i+1 mod n, hub} has p = 1 key
    (2 i + 2) + (2 (i+1 mod n) + 2) + 1 and min key 1: the p = 1 order is by
    that sum, the p = -inf order (all keys 1) is the triple order."""
    hub = n
    u = np.array(list(range(n)) + list(range(n)), np.int32)
    v = np.array([hub] * n + [(i + 1) % n for i in range(n)], np.int32)
    w = np.array([2 * i + 2 for i in range(n)] + [1] * n, np.int32)
    tris = [tuple(sorted((i, (i + 1) % n, hub))) for i in range(n)]
    key1 = {t: (2 * t[0] + 2) + (2 * t[1] + 2) + 1 for t in tris}
    r = oracle.topk(n + 1, u, v, w, 1.0, n + 3)
    assert r["ntri"] == n and r["count"] == n
    assert [tuple(x) for x in r["tri"]] == sorted(tris, key=lambda t: (-key1[t], t))
    assert [int(k) for k in r["key"]] == sorted(key1.values(), reverse=True)
    r = oracle.topk(n + 1, u, v, w, -math.inf, n)
    assert [tuple(x) for x in r["tri"]] == sorted(tris) and set(int(k) for k in r["key"]) == {1}
    r = oracle.topk(n + 1, u, v, w, math.inf, 1)
    assert int(r["key"][0]) == 2 * (n - 1) + 2


def test_trace_a_cubed_count():
    for g in [synth.tiny_graph(0), synth.scaled_mid_graph(3000, 30000, seed=5)]:
        A = np.zeros((g.n, g.n), dtype=np.float64)
        A[g.u, g.v] = 1.0
        A[g.v, g.u] = 1.0
        tr = float(np.sum((A @ A) * A))
        expect = int(round(tr)) // 6
        assert oracle.count_triangles(g.n, g.u, g.v, g.w) == expect
        assert oracle.topk(g.n, g.u, g.v, g.w, 1.0, 10)["ntri"] == expect


@pytest.mark.parametrize("fx", load_all(), ids=lambda d: d["name"])
def test_golden_hand_enumerated(fx):
    for pname, rows in fx["expected"].items():
        r = oracle.topk(fx["n"], fx["u"], fx["v"], fx["w"], P_OF[pname], fx["k"])
        assert r["ntri"] == fx["ntri"]
        assert r["count"] == len(rows)
        for i, row in enumerate(rows):
            assert tuple(int(x) for x in r["tri"][i]) == tuple(row[:3])
            if row[3] is not None:  # exact integer key (p in {-inf, 0, 1, 2, +inf})
                assert int(r["key"][i]) == row[3]
            want = closed_form(row[4])
            assert abs(r["value"][i] - want) <= 4e-16 * max(1.0, abs(want))


def test_score_closed_forms():
    assert oracle.score(1.0, 1, 2, 2) == (5, 5.0 / 3.0)
    k, val = oracle.score(2.0, 1, 2, 2)
    assert k == 9 and val == math.sqrt(3.0)
    assert oracle.score(math.inf, 1, 2, 2) == (2, 2.0)
    assert oracle.score(-math.inf, 1, 2, 2) == (1, 1.0)
    # p = 0: the geometric mean (2 * 4 * 8)^(1/3) = 4, ranked by the product
    k, val = oracle.score(0.0, 2, 4, 8)
    assert k == 64 and abs(val - 4.0) <= 4e-16 * 4.0
    W = 2**21 - 1
    assert oracle.score(0.0, W, W, W)[0] == W**3
    # Largest int32 weights: the p=2 key must not wrap (3 * (2^31-1)^2 < 2^64).
    W = 2**31 - 1
    k, val = oracle.score(2.0, W, W, W)
    assert k == 3 * W * W
    assert abs(val - W) <= 1e-12 * W
    k, val = oracle.score(1.0, W, W, W)
    assert k == 3 * W and val == float(W)


def test_score_general_p_closed_forms():
    """Any other finite p ranks by the fp64 p-mean of Eq. 1; values against
    closed forms worked here with exact fractions."""
    from fractions import Fraction as F

    def harmonic(a, b, c):
        return 3 / (F(1, a) + F(1, b) + F(1, c))
    for a, b, c in [(1, 2, 4), (2, 3, 6), (4, 5, 6), (1, 1, 1), (7, 1000000, 3)]:
        want = float(harmonic(a, b, c))
        for perm in itertools.permutations((a, b, c)):
            k, val = oracle.score(-1.0, *perm)
            assert abs(val - want) <= 4e-16 * want, (a, b, c, perm)
            assert k == oracle.score(-1.0, a, b, c)[0]  # equal multisets: equal keys
    # p = -2: ((1 + 1 + 1/4) / 3)^(-1/2) = (3/4)^(-1/2) = 2/sqrt(3)
    assert abs(oracle.score(-2.0, 1, 1, 2)[1] - 2 / math.sqrt(3)) <= 4e-16 * 2
    # p = 3: ((1 + 8 + 64) / 3)^(1/3); p = 1/2: ((1 + 2 + 3) / 3)^2 = 4
    assert abs(oracle.score(3.0, 1, 2, 4)[1] - (73 / 3) ** (1 / 3)) <= 1e-15 * 3
    assert abs(oracle.score(0.5, 1, 4, 9)[1] - 4.0) <= 1e-15 * 4
    # equal weights: every mean is that weight exactly
    for p in (-7.5, -1.0, 0.25, 3.0, 40.0):
        assert oracle.score(p, 9, 9, 9)[1] == 9.0
    # the limits p -> +-inf: max and min (Section 1)
    assert abs(oracle.score(400.0, 3, 5, 11)[1] - 11.0) <= 11.0 * 3e-3
    assert abs(oracle.score(-400.0, 3, 5, 11)[1] - 3.0) <= 3.0 * 3e-3
    # weights near 2^31 and large |p|: no overflow (the largest or smallest
    # weight is factored out)
    W = 2**31 - 1
    for p in (-60.0, 60.0):
        val = oracle.score(p, W, W - 1, 5)[1]
        assert math.isfinite(val) and 5 <= val <= W


def _python_bruteforce(n, u, v, w, p):
    adj = {}
    for a, b, x in zip(u.tolist(), v.tolist(), w.tolist()):
        adj[(min(a, b), max(a, b))] = x
    out = []
    for a, b, c in itertools.combinations(range(n), 3):
        if (a, b) in adj and (b, c) in adj and (a, c) in adj:
            ws = [adj[(a, b)], adj[(b, c)], adj[(a, c)]]
            if p == 1.0:
                key = sum(ws)
            elif p == 2.0:
                key = sum(x * x for x in ws)
            elif p == math.inf:
                key = max(ws)
            elif p == 0.0:
                key = ws[0] * ws[1] * ws[2]
            else:
                key = min(ws)
            out.append((key, (a, b, c)))
    out.sort(key=lambda t: (-t[0], t[1]))
    return out


@pytest.mark.parametrize("seed", range(40))
def test_python_bruteforce_random_small(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(3, 36))
    g = synth.random_small_graph(n, float(rng.uniform(0.1, 0.9)), int(rng.integers(1, 6)), seed)
    if g.m == 0:
        return
    for p in PS:
        want = _python_bruteforce(g.n, g.u, g.v, g.w, p)
        k = max(1, len(want))
        r = oracle.topk(g.n, g.u, g.v, g.w, p, k)
        assert r["ntri"] == len(want)
        got = [(int(key), tuple(int(x) for x in t)) for key, t in zip(r["key"], r["tri"])]
        assert got == want[: r["count"]]


def _exact_mean(p, ws):
    """m_p with exact rationals where p is an integer (p = -1, -2, 3 are
    rational; the cube root of p = 3 is taken on the float of the exact
    power mean)."""
    from fractions import Fraction as F
    if p == -1.0:
        return 3 / sum(F(1, x) for x in ws)
    if p == 3.0:
        return float(sum(F(x) ** 3 for x in ws) / 3) ** (1.0 / 3.0)
    raise ValueError(p)


@pytest.mark.parametrize("seed", range(24))
@pytest.mark.parametrize("p", [-1.0, 3.0])
def test_python_bruteforce_general_p(seed, p):
    """Any other finite p: the oracle's top-k against a Python itertools brute
    force over vertex triples with exact rational harmonic means (p = -1) or
    exact power sums (p = 3), under the fp64-key comparison rule."""
    from wtri_testutil import assert_topk_close
    rng = np.random.default_rng(500 + seed)
    n = int(rng.integers(3, 30))
    g = synth.random_small_graph(n, float(rng.uniform(0.2, 0.9)), int(rng.integers(2, 9)), seed)
    if g.m == 0:
        return
    adj = {}
    for a, b, x in zip(g.u.tolist(), g.v.tolist(), g.w.tolist()):
        adj[(min(a, b), max(a, b))] = x
    tris = []
    for a, b, c in itertools.combinations(range(g.n), 3):
        if (a, b) in adj and (b, c) in adj and (a, c) in adj:
            tris.append((_exact_mean(p, [adj[(a, b)], adj[(b, c)], adj[(a, c)]]), (a, b, c)))
    tris.sort(key=lambda t: (-t[0], t[1]))
    k = max(1, min(len(tris), int(rng.integers(1, 40))))
    r = oracle.topk(g.n, g.u, g.v, g.w, p, k)
    assert r["ntri"] == len(tris)
    want = tris[:k]
    assert_topk_close(r["tri"], r["value"], np.array([t for _, t in want], np.int32).reshape(-1, 3),
                      np.array([float(v) for v, _ in want]), f"seed={seed} p={p}")


@pytest.mark.parametrize("n", [5, 13, 40])
@pytest.mark.parametrize("p", [-1.0, -2.0, 0.5, 3.0])
def test_complete_graph_general_p_top1(n, p):
    """K_n with w(u, v) = u + v: the mean is increasing in each weight, so the
    heaviest triangle {n-3, n-2, n-1} is first for every p."""
    u, v, w = complete_graph(n, lambda a, b: a + b)
    r = oracle.topk(n, u, v, w, p, 3)
    assert tuple(int(x) for x in r["tri"][0]) == (n - 3, n - 2, n - 1)
    ws = [2 * n - 5, 2 * n - 4, 2 * n - 3]
    want = (sum(x ** p for x in ws) / 3) ** (1 / p)
    assert abs(r["value"][0] - want) <= 1e-13 * want


def test_invariants_tiny():
    g = synth.tiny_graph(0)
    adj = {}
    for a, b, x in zip(g.u.tolist(), g.v.tolist(), g.w.tolist()):
        adj[(min(a, b), max(a, b))] = x
    for p in PS:
        r = oracle.topk(g.n, g.u, g.v, g.w, p, 300)
        r2 = oracle.topk(g.n, g.u, g.v, g.w, p, 301)
        # prefix property
        assert np.array_equal(r["tri"], r2["tri"][:300])
        # sorted by (key desc, triple asc), each a real triangle with its key
        prev = None
        for t, key, val in zip(r["tri"].tolist(), r["key"].tolist(), r["value"].tolist()):
            a, b, c = t
            assert a < b < c
            ws = [adj[(a, b)], adj[(b, c)], adj[(a, c)]]
            kk, vv = oracle.score(p, *ws)
            assert kk == key and vv == val
            if prev is not None:
                assert (-prev[0], prev[1]) < (-key, tuple(t))
            prev = (key, tuple(t))
    # relabelling vertices keeps the multiset of the top keys
    perm = np.random.default_rng(3).permutation(g.n).astype(np.int32)
    for p in PS:
        a = oracle.topk(g.n, g.u, g.v, g.w, p, 500)
        b = oracle.topk(g.n, perm[g.u], perm[g.v], g.w, p, 500)
        assert np.array_equal(a["key"], b["key"])


@pytest.mark.parametrize("bad", ["self_loop", "out_of_range", "zero_weight", "negative_weight", "duplicate"])
def test_invalid_inputs_rejected(bad):
    u = np.array([0, 1, 2], np.int32)
    v = np.array([1, 2, 0], np.int32)
    w = np.array([1, 2, 3], np.int32)
    n = 3
    if bad == "self_loop":
        v[1] = 1
    elif bad == "out_of_range":
        v[1] = 3
    elif bad == "zero_weight":
        w[2] = 0
    elif bad == "negative_weight":
        w[2] = -4
    elif bad == "duplicate":
        u = np.array([0, 1, 2, 1], np.int32)
        v = np.array([1, 2, 0, 0], np.int32)
        w = np.array([1, 2, 3, 4], np.int32)
    with pytest.raises(oracle.OracleError):
        oracle.topk(n, u, v, w, 1.0, 3)
    with pytest.raises(oracle.OracleError):
        oracle.sym_csr(n, u, v, w)


def test_edge_order_matches_stable_argsort():
    g = synth.tiny_graph(0)
    perm = oracle.edge_order(g.w)
    assert np.array_equal(perm, np.argsort(-g.w.astype(np.int64), kind="stable"))


def test_sym_csr_matches_scipy():
    sp = pytest.importorskip("scipy.sparse")
    g = synth.tiny_graph(0)
    rowptr, col, wt, eid = oracle.sym_csr(g.n, g.u, g.v, g.w)
    A = sp.coo_matrix((np.concatenate([g.w, g.w]), (np.concatenate([g.u, g.v]), np.concatenate([g.v, g.u]))),
                      shape=(g.n, g.n)).tocsr()
    A.sort_indices()
    assert np.array_equal(rowptr, A.indptr.astype(np.int64))
    assert np.array_equal(col, A.indices)
    assert np.array_equal(wt, A.data)


def test_oriented_csr_structure():
    g = synth.tiny_graph(0)
    orow, ocol, owt, oeid = oracle.oriented_csr(g.n, g.u, g.v, g.w)
    deg = np.bincount(np.concatenate([g.u, g.v]), minlength=g.n)
    src = np.repeat(np.arange(g.n), np.diff(orow))
    # each undirected edge exactly once, from lower (degree, id) to higher
    assert np.array_equal(np.sort(oeid), np.arange(g.m))
    assert np.all((deg[src] < deg[ocol]) | ((deg[src] == deg[ocol]) & (src < ocol)))
    lo = np.minimum(g.u[oeid], g.v[oeid])
    hi = np.maximum(g.u[oeid], g.v[oeid])
    assert np.array_equal(np.minimum(src, ocol), lo) and np.array_equal(np.maximum(src, ocol), hi)
    assert np.array_equal(owt, g.w[oeid])
    for a in range(g.n):
        row = ocol[orow[a]:orow[a + 1]]
        assert np.all(np.diff(row) > 0)


def test_weight_sorted_rows():
    g = synth.tiny_graph(0)
    rowptr, col, wt, rank = oracle.weight_sorted_rows(g.n, g.u, g.v, g.w)
    perm = oracle.edge_order(g.w)
    for a in range(0, g.n, 7):
        s, e = rowptr[a], rowptr[a + 1]
        assert np.all(np.diff(wt[s:e]) <= 0)
        assert np.all(np.diff(rank[s:e]) > 0)
        assert np.array_equal(g.w[perm[rank[s:e]]], wt[s:e])
