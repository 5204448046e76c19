"""The device-drawn batch workload (run here on the CPU device): every graph
is simple, has exactly the size batch_graph gives it, starts on a 16-byte
boundary, and has weights in [1, 1e6]."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")


def test_batch_graphs_device_valid():
    b = synth.batch_graphs_device(48, seed=3, n_hi=3000, device="cpu")
    ns, ms = synth.batch_sizes(48, 3, 3000)
    assert np.array_equal(b.ns, ns) and np.array_equal(b.ms, ms)
    for g in range(b.count):
        n, u, v, w = b.graph(g)
        host = synth.batch_graph(g, seed=3, n_hi=3000)
        assert (n, u.shape[0]) == (host.n, host.m)
        u = u.numpy().astype(np.int64)
        v = v.numpy().astype(np.int64)
        w = w.numpy()
        assert b.offs[g] % 4 == 0
        assert np.all(u != v) and u.min() >= 0 and v.min() >= 0 and max(u.max(), v.max()) < n
        key = np.minimum(u, v) * n + np.maximum(u, v)
        assert np.unique(key).shape[0] == u.shape[0]
        assert w.min() >= 1 and w.max() <= 1_000_000


def test_batch_graphs_device_seeded():
    a = synth.batch_graphs_device(8, seed=5, n_hi=1000, device="cpu")
    b = synth.batch_graphs_device(8, seed=5, n_hi=1000, device="cpu")
    assert torch.equal(a.u, b.u) and torch.equal(a.v, b.v) and torch.equal(a.w, b.w)


def test_large_recipe_device_draw_small():
    """The billion-edge recipe (and the serving pool's exponent) drawn at a
    small size on the CPU device: simple graph, exactly m edges, the lookup
    arrays consistent with the edge list, and none kept when not asked for."""
    g = synth.large_graph_device(9, n=200_000, m=400_000, device="cpu", gamma=2.1)
    u = g.u.numpy().astype(np.int64)
    v = g.v.numpy().astype(np.int64)
    assert u.shape[0] == 400_000 and np.all(u != v)
    key = np.minimum(u, v) * g.n + np.maximum(u, v)
    assert np.unique(key).shape[0] == 400_000
    order = np.argsort(key)
    assert np.array_equal(g.keys.numpy(), key[order])
    assert np.array_equal(g.w_by_key.numpy(), g.w.numpy()[order])
    bare = synth.large_graph_device(9, n=200_000, m=400_000, device="cpu", gamma=2.1, lookup=False)
    assert bare.keys is None and bare.w_by_key is None
    assert torch.equal(bare.u, g.u) and torch.equal(bare.w, g.w)
