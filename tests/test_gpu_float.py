"""Real (fp32) edge weights on the GPU against the oracle's real-weight
top-k: exact at p = -inf and +inf (min and max of the weights), within the
fp64 set-equality rule at every other p (0 included)."""
import math

import numpy as np
import pytest

import oracle
import synth
from wtri_testutil import GEN_TOL, assert_topk_close

pytestmark = pytest.mark.gpu

wt = pytest.importorskip("paper_1910_00692_gb300")

PS = [-math.inf, 0.0, 1.0, 2.0, math.inf, -1.0, 3.0]


def _check(g, w, p, k, ctx):
    d = wt.build_csr(g.n, g.u, g.v, w)
    try:
        _check_built(g, d, w, p, k, ctx)
    finally:
        d.free()


def _check_built(g, d, w, p, k, ctx):
    want = oracle.topk_real(g.n, g.u, g.v, w, p, k)
    tris, wts = d.topk(p, k)
    if math.isinf(p):
        assert np.array_equal(tris, want["tri"]), ctx
        assert np.array_equal(wts, want["value"]), ctx
    else:
        assert_topk_close(tris, wts, want["tri"], want["value"], ctx, rel=GEN_TOL)


@pytest.mark.parametrize("p", PS)
def test_tiny_lognormal(p):
    g = synth.tiny_graph(0)
    w = np.random.default_rng(1).lognormal(0.0, 2.0, g.m).astype(np.float32)
    d = wt.build_csr(g.n, g.u, g.v, w)
    try:
        for k in (1, 100, 5000):
            _check_built(g, d, w, p, k, f"tiny p={p} k={k}")
    finally:
        d.free()


@pytest.mark.parametrize("seed", range(8))
def test_random_small_with_ties(seed):
    g = synth.random_small_graph(30 + 5 * seed, 0.3, 5, 400 + seed)
    w = np.random.default_rng(seed).choice(np.array([0.25, 1.5, 1.5, 7.0, 1e-3], np.float32), g.m)
    d = wt.build_csr(g.n, g.u, g.v, w)
    try:
        for p in PS:
            _check_built(g, d, w, p, 50, f"seed={seed} p={p}")
    finally:
        d.free()


def test_scaled_graph_and_structures():
    g = synth.scaled_mid_graph(100_000, 1_000_000, seed=13)
    w = np.random.default_rng(2).lognormal(3.0, 1.5, g.m).astype(np.float32)
    d = wt.build_csr(g.n, g.u, g.v, w)
    try:
        perm = np.lexsort((np.arange(g.m), -w.astype(np.float64)))  # weight desc, index asc
        assert np.array_equal(d.array("order_w").view(np.float32), w[perm])
        assert np.array_equal(d.array("order_u"), g.u[perm])
        for p in PS:
            _check_built(g, d, w, p, 1000, f"scaled p={p}")
    finally:
        d.free()


@pytest.mark.parametrize("p", [-math.inf, 1.0, 2.0, math.inf])
def test_integer_valued_floats_match_the_integer_build(p):
    """The same graph built from int32 and from float32 weights."""
    g = synth.tiny_graph(0)
    di = wt.build_csr(g.n, g.u, g.v, g.w)
    df = wt.build_csr(g.n, g.u, g.v, g.w.astype(np.float32))
    try:
        ti, wi = di.topk(p, 500)
        tf, wf = df.topk(p, 500)
        if math.isinf(p):  # min and max are exact either way
            assert np.array_equal(ti, tf) and np.array_equal(wi, wf)
        else:  # fp64 means of tied integer sums may differ in the last bit
            assert_topk_close(tf, wf, ti, wi, f"p={p}", rel=GEN_TOL)
    finally:
        di.free()
        df.free()


@pytest.mark.parametrize("bad", [0.0, -2.0, math.inf, math.nan])
def test_bad_weights_rejected(bad):
    g = synth.tiny_graph(0)
    w = g.w.astype(np.float32)
    w[17] = bad
    with pytest.raises(wt.WtriError) as ei:
        wt.build_csr(g.n, g.u, g.v, w)
    assert ei.value.code == -1 and "17" in str(ei.value)


def test_integer_only_paths_refuse():
    g = synth.tiny_graph(0)
    d = wt.build_csr(g.n, g.u, g.v, g.w.astype(np.float32))
    try:
        with pytest.raises(wt.WtriError) as ei:
            d.sample_topk(1.0, 10, 1000, 1)
        assert ei.value.code == -5
        with pytest.raises(wt.WtriError) as ei:
            wt.topk_batch([d], [1.0], [10])
        assert ei.value.code == -5
        with pytest.raises(wt.WtriError) as ei:
            wt.sample_cliques(d, 4, 1.0, 10, -1, 0)
        assert ei.value.code == -5
    finally:
        d.free()
