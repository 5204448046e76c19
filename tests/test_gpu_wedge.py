"""GPU weighted wedge sampling (Algorithm 4) against the oracle: every draw
(center, positions of b and c, closed triangle) bit-identical for the same
seed, and the top-k of the triangle set T element by element."""
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
    gs = {"tiny": synth.tiny_graph(0), "scaled": synth.scaled_mid_graph(100_000, 1_000_000, seed=12)}
    ds = {k: wt.build_csr(g.n, g.u, g.v, g.w) for k, g in gs.items()}
    yield gs, ds
    for d in ds.values():
        d.free()


@pytest.mark.parametrize("name", ["tiny", "scaled"])
@pytest.mark.parametrize("p", [0.0, 1.0, 2.0])
@pytest.mark.parametrize("nsamples,seed", [(1, 0), (5000, 7), (200_000, 2**64 - 1)])
def test_wedge_draws_bit_identical(graphs, name, p, nsamples, seed):
    g, d = graphs[0][name], graphs[1][name]
    got = wt.sample_wedges(d, p, nsamples, seed)
    want = oracle.wedge_samples(g.n, g.u, g.v, g.w, p, nsamples, seed)
    for a, b, what in zip(got, want, ("center", "jb", "jc", "tri")):
        mism = np.nonzero(np.any(np.asarray(a).reshape(nsamples, -1) != np.asarray(b).reshape(nsamples, -1),
                                 axis=1))[0]
        assert mism.size == 0, f"{name} p={p}: {what} differs first at sample {mism[0]}"


@pytest.mark.parametrize("name", ["tiny", "scaled"])
@pytest.mark.parametrize("p", [0.0, 1.0, 2.0])
@pytest.mark.parametrize("k,nsamples", [(10, 2000), (100, 50_000), (1000, 500_000)])
def test_wedge_topk_vs_oracle(graphs, name, p, k, nsamples):
    g, d = graphs[0][name], graphs[1][name]
    want = oracle.wedge_topk(g.n, g.u, g.v, g.w, p, k, nsamples, 7)
    tris, wts = wt.wedge_topk(d, p, k, nsamples, 7)
    assert_topk_equal(tris, wts, want, p, f"{name} p={p} k={k} s={nsamples}")


def test_wedge_errors(graphs):
    d = graphs[1]["tiny"]
    for p in (math.inf, -math.inf, -1.0, 3.0):
        with pytest.raises(wt.WtriError) as ei:
            wt.wedge_topk(d, p, 10, 100, 1)
        assert ei.value.code == -5
    with pytest.raises(wt.WtriError) as ei:
        wt.wedge_topk(d, 1.0, 10, -1, 1)
    assert ei.value.code == -1
    tris, _ = wt.wedge_topk(d, 1.0, 10, 0, 1)
    assert tris.shape[0] == 0
