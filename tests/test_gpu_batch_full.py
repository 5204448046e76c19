"""The batched query at the batch workload's full size: 4,096 Chung-Lu
graphs, n log-uniform in [100, 2e5], m = 10 n (1.12e9 edges in all),
exponent 2.2, Zipf(2) weights, drawn on the device; per-graph k in
[10, 1000] and p in {-inf, 1, 2, +inf}.

* Every query's batched answer equals the plain wtri_topk answer bit for bit.
* A spread of graphs (the smallest, the largest and every 128th) is checked
  against the oracle.
"""
import numpy as np
import pytest

import oracle
import synth
from wtri_testutil import assert_topk_equal

pytestmark = pytest.mark.gpu

wt = pytest.importorskip("paper_1910_00692_gb300")
torch = pytest.importorskip("torch")

COUNT = 4096


@pytest.fixture(scope="module")
def batch():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    b = synth.batch_graphs_device(COUNT, seed=3, n_hi=200_000)
    ds = [wt.build_csr(*b.graph(i)) for i in range(COUNT)]
    ps, ks = synth.batch_queries(COUNT, seed=3)
    yield b, ds, ps, ks
    for d in ds:
        d.free()
    del b
    torch.cuda.empty_cache()


def test_full_batch_matches_plain(batch):
    b, ds, ps, ks = batch
    assert int(b.ms.sum()) > 1_000_000_000
    res = wt.topk_batch(ds, ps, ks)
    for i, d in enumerate(ds):
        t, w = d.topk(ps[i], int(ks[i]))
        assert np.array_equal(res[i][0], t), i
        assert np.array_equal(res[i][1], w), i


def test_full_batch_vs_oracle_sample(batch):
    b, ds, ps, ks = batch
    pick = sorted(set([int(np.argmin(b.ns)), int(np.argmax(b.ns))] + list(range(0, COUNT, 128))))
    res = wt.topk_batch([ds[i] for i in pick], ps[pick], ks[pick])
    for j, i in enumerate(pick):
        n, u, v, w = b.graph(i)
        want = oracle.topk(n, u.cpu().numpy(), v.cpu().numpy(), w.cpu().numpy(), ps[i], int(ks[i]))
        assert_topk_equal(res[j][0], res[j][1], want, ps[i], f"graph {i} n={n} p={ps[i]} k={ks[i]}")
