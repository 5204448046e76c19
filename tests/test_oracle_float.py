"""Pins of the oracle's real-weight top-k (Eq. 1 over positive reals):
integer-valued weights give the integer oracle's answer, scaling every
weight by a power of two scales every mean exactly, closed forms on K_n,
a subset brute force on tiny graphs, and bad weights rejected."""
import itertools
import math

import numpy as np
import pytest

import oracle
import synth

PS = [-math.inf, 0.0, 1.0, 2.0, math.inf, -1.0, 3.0]


@pytest.mark.parametrize("p", PS)
def test_integer_valued_weights_match_the_integer_oracle(p):
    for seed in range(3):
        g = synth.random_small_graph(40, 0.3, 50, 300 + seed)
        a = oracle.topk(g.n, g.u, g.v, g.w, p, 200)
        b = oracle.topk_real(g.n, g.u, g.v, g.w.astype(np.float32), p, 200)
        assert a["ntri"] == b["ntri"] and np.array_equal(a["tri"], b["tri"])
        assert np.allclose(a["value"], b["value"], rtol=1e-12, atol=0)


@pytest.mark.parametrize("p", PS)
def test_power_of_two_scaling(p):
    rng = np.random.default_rng(5)
    g = synth.random_small_graph(30, 0.4, 9, 7)
    w = rng.lognormal(0.0, 1.0, g.m).astype(np.float32)
    a = oracle.topk_real(g.n, g.u, g.v, w, p, 500)
    b = oracle.topk_real(g.n, g.u, g.v, w * np.float32(4.0), p, 500)
    assert np.array_equal(a["tri"], b["tri"])
    if p == 0.0:  # cbrt is not correctly rounded: a few ulps
        assert np.allclose(b["value"], 4.0 * a["value"], rtol=1e-15, atol=0)
    else:  # every other mean scales exactly (the power of two factors out)
        assert np.array_equal(b["value"], 4.0 * a["value"])


def test_complete_graph():
    n = 12
    iu, ju = np.triu_indices(n, 1)
    u, v = iu.astype(np.int32), ju.astype(np.int32)
    w = ((u + v) / 8.0).astype(np.float32)
    for p in (-math.inf, 0.0, 1.0, 2.0, -1.0, 3.0):
        r = oracle.topk_real(n, u, v, w, p, 1)
        assert tuple(r["tri"][0]) == (n - 3, n - 2, n - 1)
    r = oracle.topk_real(n, u, v, w, 1.0, 1)
    assert r["value"][0] == (2 * (3 * n - 6) / 8.0) / 3.0
    assert r["ntri"] == math.comb(n, 3)


def test_subset_brute_force():
    rng = np.random.default_rng(9)
    g = synth.random_small_graph(14, 0.5, 3, 11)
    w = rng.choice(np.array([0.5, 1.25, 3.0], np.float32), g.m)  # ties
    wt = {(min(a, b), max(a, b)): float(x) for a, b, x in zip(g.u.tolist(), g.v.tolist(), w.tolist())}
    for p in (-math.inf, 1.0, math.inf):
        want = []
        for t in itertools.combinations(range(g.n), 3):
            es = [(t[0], t[1]), (t[0], t[2]), (t[1], t[2])]
            if all(e in wt for e in es):
                xs = [wt[e] for e in es]
                m = min(xs) if p == -math.inf else (max(xs) if p == math.inf else sum(sorted(xs)) / 3.0)
                want.append((-m, t))
        want.sort()
        r = oracle.topk_real(g.n, g.u, g.v, w, p, 10_000)
        assert r["ntri"] == len(want)
        assert [tuple(int(x) for x in t) for t in r["tri"]] == [e[1] for e in want]
        assert [float(x) for x in r["value"]] == [-e[0] for e in want]


@pytest.mark.parametrize("bad", [0.0, -1.0, math.inf, math.nan])
def test_bad_weights(bad):
    u = np.array([0, 1, 0], np.int32)
    v = np.array([1, 2, 2], np.int32)
    w = np.array([1.0, 2.0, bad], np.float32)
    with pytest.raises(oracle.OracleError):
        oracle.topk_real(3, u, v, w, 1.0, 3)
