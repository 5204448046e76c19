"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Triangle sets and order are compared element by element (bit-exact ids);
weights bit-exact for p in {-inf, 1, +inf} and within 1e-12 relative at
p = 2 and p = 0.  Inputs are the seeded synthetic graphs of synth/.
"""
import ctypes
import math

import numpy as np
import pytest

import oracle
import synth
from golden_io import P_OF, closed_form, load_all
from wtri_testutil import PS, assert_topk_equal, check_structures

pytestmark = pytest.mark.gpu

wt = pytest.importorskip("paper_1910_00692_gb300")


@pytest.fixture(scope="module")
def tiny():
    return synth.tiny_graph(0)


@pytest.fixture(scope="module")
def tiny_dev(tiny):
    g = wt.build_csr(tiny.n, tiny.u, tiny.v, tiny.w)
    yield g
    g.free()


@pytest.mark.parametrize("fx", load_all(), ids=lambda d: d["name"])
def test_golden(fx):
    g = wt.build_csr(fx["n"], fx["u"], fx["v"], fx["w"])
    try:
        for pname, rows in fx["expected"].items():
            tris, wts = g.topk(P_OF[pname], fx["k"])
            assert tris.shape[0] == len(rows), pname
            for i, row in enumerate(rows):
                assert tuple(int(x) for x in tris[i]) == tuple(row[:3]), (pname, i)
                want = closed_form(row[4])
                assert abs(wts[i] - want) <= 1e-15 * max(1.0, abs(want)), (pname, i)
    finally:
        g.free()


@pytest.mark.parametrize("p", PS)
@pytest.mark.parametrize("k", [1, 100, 777, 20000])
def test_tiny_vs_oracle(tiny, tiny_dev, p, k):
    want = oracle.topk(tiny.n, tiny.u, tiny.v, tiny.w, p, k)
    tris, wts = tiny_dev.topk(p, k)
    assert_topk_equal(tris, wts, want, p, f"tiny p={p} k={k}")


def test_tiny_structures(tiny, tiny_dev):
    check_structures(tiny, tiny_dev)
    # array ids 8..10 are unused (no symmetric id-sorted rows are kept)
    nb = ctypes.c_int64()
    for which in (8, 9, 10, 99):
        assert wt.lib().wtri_graph_copy_array(tiny_dev._h, which, None, 0, ctypes.byref(nb)) == -1


@pytest.mark.parametrize("n,m,seed", [(20000, 200000, 11), (100000, 1000000, 12)])
def test_scaled_structures(n, m, seed):
    """Graphs with rows longer than the block-orientation threshold."""
    g = synth.scaled_mid_graph(n, m, seed=seed)
    d = wt.build_csr(g.n, g.u, g.v, g.w)
    try:
        check_structures(g, d)
    finally:
        d.free()


def _cliques_graph(sizes, seed, wmax=9):
    """Disjoint cliques K_{s+1} for s in sizes: equal degrees inside a clique,
    so the (degree, id) order gives its vertices the oriented degrees s,
    s - 1, ..., 0 -- every size class of the per-row sort up to s; random
    weights 1..wmax, edges shuffled and flipped."""
    rng = np.random.default_rng(seed)
    us, vs = [], []
    base = 0
    for s_ in sizes:
        iu, ju = np.triu_indices(s_ + 1, 1)
        us.append(iu + base)
        vs.append(ju + base)
        base += s_ + 1
    u = np.concatenate(us)
    v = np.concatenate(vs)
    perm = rng.permutation(u.shape[0])
    u, v = u[perm], v[perm]
    flip = rng.random(u.shape[0]) < 0.5
    u2 = np.where(flip, v, u).astype(np.int32)
    v2 = np.where(flip, u, v).astype(np.int32)
    w = rng.integers(1, wmax + 1, u.shape[0]).astype(np.int32)
    return synth.Graph(n=int(base), u=u2, v=v2, w=w, name="cliques")


def test_oriented_row_classes_topk():
    """Oriented rows of the sub-warp and warp classes (cliques up to 129):
    structures and the top-k against the oracle."""
    g = _cliques_graph([5, 8, 9, 16, 17, 32, 33, 64, 65, 129], seed=7)
    d = wt.build_csr(g.n, g.u, g.v, g.w)
    try:
        check_structures(g, d)
        for p in PS:
            want = oracle.topk(g.n, g.u, g.v, g.w, p, 300)
            tris, wts = d.topk(p, 300)
            assert_topk_equal(tris, wts, want, p, f"cliques p={p}")
    finally:
        d.free()


@pytest.mark.parametrize("sizes", [[256, 257, 512, 513, 1024, 1025], [4000], [8193]],
                         ids=["warp-block", "block-smem", "block-global"])
def test_oriented_row_classes_structures(sizes):
    """Oriented rows at the boundaries of the per-row sort's size classes (one
    warp up to 1024, one block up to 8192 in shared memory, global merges
    beyond): every device structure against the oracle's construction; on
    the warp/block boundary case also the top-k at p = 1."""
    g = _cliques_graph(sizes, seed=sum(sizes), wmax=1_000_000)
    d = wt.build_csr(g.n, g.u, g.v, g.w)
    try:
        check_structures(g, d)
        if max(sizes) <= 1025:
            want = oracle.topk(g.n, g.u, g.v, g.w, 1.0, 300)
            tris, wts = d.topk(1.0, 300)
            assert_topk_equal(tris, wts, want, 1.0, f"cliques {sizes}")
    finally:
        d.free()


@pytest.mark.parametrize("dgr", [6, 14, 27, 200, 3000, 9000])
def test_repeated_pair_in_long_row(dgr):
    """A repeated undirected pair inside an oriented row of each size class is
    rejected (WTRI_EINVAL naming the pair).  Vertex 0 joins every vertex of
    a clique K_{dgr} whose vertices also hold two leaves each, so vertex 0
    has the lowest degree and its oriented row holds the whole clique and
    the repeat."""
    iu, ju = np.triu_indices(dgr, 1)
    cu, cv = iu + 1, ju + 1
    star = np.arange(1, dgr + 1)
    leaves = dgr + 1 + np.arange(2 * dgr)
    u = np.concatenate([cu, np.zeros(dgr, np.int64), np.repeat(star, 2), [dgr // 2 + 1]]).astype(np.int32)
    v = np.concatenate([cv, star, leaves, [0]]).astype(np.int32)
    w = np.full(u.shape[0], 3, np.int32)
    with pytest.raises(wt.WtriError) as ei:
        wt.build_csr(3 * dgr + 1, u, v, w)
    assert ei.value.code == -1
    assert "repeated" in str(ei.value) and "{0, %d}" % (dgr // 2 + 1) in str(ei.value)


@pytest.mark.parametrize("seed", range(24))
def test_random_small_graphs(seed):
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(3, 80))
    g = synth.random_small_graph(n, float(rng.uniform(0.05, 0.9)), int(rng.integers(1, 7)), seed)
    if g.m == 0:
        return
    d = wt.build_csr(g.n, g.u, g.v, g.w)
    try:
        for p in PS:
            for k in (1, 3, 50, 100000 // 2):
                k = min(k, 65536)
                want = oracle.topk(g.n, g.u, g.v, g.w, p, k)
                tris, wts = d.topk(p, k)
                assert_topk_equal(tris, wts, want, p, f"seed={seed} n={n} p={p} k={k}")
    finally:
        d.free()


@pytest.mark.parametrize("n,m,seed", [(20000, 200000, 11), (100000, 1000000, 12)])
def test_scaled_mid_vs_oracle(n, m, seed):
    g = synth.scaled_mid_graph(n, m, seed=seed)
    d = wt.build_csr(g.n, g.u, g.v, g.w)
    try:
        for p in PS:
            for k in (10, 1000, 5000):
                want = oracle.topk(g.n, g.u, g.v, g.w, p, k)
                tris, wts = d.topk(p, k)
                assert_topk_equal(tris, wts, want, p, f"n={n} p={p} k={k}")
    finally:
        d.free()


def test_device_inputs_and_device_outputs(tiny):
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda:0")
    u = torch.from_numpy(tiny.u).to(dev)
    v = torch.from_numpy(tiny.v).to(dev)
    w = torch.from_numpy(tiny.w).to(dev)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        d = wt.build_csr(tiny.n, u, v, w, stream=s)
    try:
        k = 500
        for p in PS:
            ot = torch.zeros((k, 3), dtype=torch.int32, device=dev)
            ow = torch.zeros(k, dtype=torch.float64, device=dev)
            oc = torch.zeros(1, dtype=torch.int32, device=dev)
            wt.topk_device(d, p, k, ot, ow, oc, stream=s)
            s.synchronize()
            cnt = int(oc.item())
            want = oracle.topk(tiny.n, tiny.u, tiny.v, tiny.w, p, k)
            assert_topk_equal(ot[:cnt].cpu().numpy(), ow[:cnt].cpu().numpy(), want, p, f"device p={p}")
    finally:
        d.free()


@pytest.mark.parametrize("bad", ["self_loop", "out_of_range", "zero_weight", "negative_weight", "duplicate",
                                 "duplicate_flipped"])
def test_invalid_inputs(bad):
    u = np.array([0, 1, 2, 3], np.int32)
    v = np.array([1, 2, 0, 0], np.int32)
    w = np.array([1, 2, 3, 4], np.int32)
    n = 4
    if bad == "self_loop":
        v[1] = 1
    elif bad == "out_of_range":
        v[1] = 4
    elif bad == "zero_weight":
        w[2] = 0
    elif bad == "negative_weight":
        w[2] = -1
    elif bad == "duplicate":
        u[3], v[3] = 1, 2
    elif bad == "duplicate_flipped":
        u[3], v[3] = 2, 1
    with pytest.raises(wt.WtriError) as ei:
        wt.build_csr(n, u, v, w)
    assert ei.value.code == -1


def test_bad_queries(tiny_dev):
    with pytest.raises(wt.WtriError) as ei:
        tiny_dev.topk(float("nan"), 10)
    assert ei.value.code == -1
    with pytest.raises(wt.WtriError) as ei:
        tiny_dev.topk(float("inf") * 0.0, 10)  # NaN again, by arithmetic
    assert ei.value.code == -1
    with pytest.raises(wt.WtriError) as ei:
        tiny_dev.topk(1.0, 0)
    assert ei.value.code == -1


def test_geometric_mean_weight_limit():
    """p = 0 ranks by the exact product of the weights, which fits 63 bits
    only for weights below 2^21; heavier graphs are refused, not rounded."""
    u = np.array([0, 1, 0], np.int32)
    v = np.array([1, 2, 2], np.int32)
    for wmax, ok in ((2**21 - 1, True), (2**21, False)):
        w = np.array([wmax, 3, 5], np.int32)
        d = wt.build_csr(3, u, v, w)
        try:
            if ok:
                t, x = d.topk(0.0, 1)
                assert t.tolist() == [[0, 1, 2]]
                assert abs(x[0] - (wmax * 15) ** (1 / 3)) <= 1e-12 * x[0]
            else:
                with pytest.raises(wt.WtriError) as ei:
                    d.topk(0.0, 1)
                assert ei.value.code == -5
                assert d.topk(1.0, 1)[0].tolist() == [[0, 1, 2]]
        finally:
            d.free()


def test_empty_and_degenerate():
    d = wt.build_csr(5, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int32))
    try:
        for p in PS:
            tris, wts = d.topk(p, 10)
            assert tris.shape[0] == 0
    finally:
        d.free()
    # a single edge, a path: no triangle
    d = wt.build_csr(3, np.array([0, 1], np.int32), np.array([1, 2], np.int32), np.array([5, 6], np.int32))
    try:
        assert d.topk(1.0, 3)[0].shape[0] == 0
    finally:
        d.free()
    # maximum int32 weights at p = 2 (key 3 * (2^31-1)^2 must not wrap)
    W = 2**31 - 1
    d = wt.build_csr(4, np.array([0, 1, 0, 2], np.int32), np.array([1, 2, 2, 3], np.int32),
                     np.array([W, W, W, 1], np.int32))
    try:
        for p in PS:
            if p == 0.0:  # the product key of such weights would not fit: refused
                with pytest.raises(wt.WtriError) as ei:
                    d.topk(p, 2)
                assert ei.value.code == -5
                continue
            want = oracle.topk(4, np.array([0, 1, 0, 2], np.int32), np.array([1, 2, 2, 3], np.int32),
                               np.array([W, W, W, 1], np.int32), p, 2)
            tris, wts = d.topk(p, 2)
            assert_topk_equal(tris, wts, want, p, "max weights")
    finally:
        d.free()


@pytest.mark.parametrize("p", [1.0, -math.inf])
def test_largest_k(p):
    """k at the library's limit (65536) on a graph with more triangles than
    that, against the oracle; one more is refused."""
    g = synth.scaled_mid_graph(100_000, 1_000_000, seed=31)
    d = wt.build_csr(g.n, g.u, g.v, g.w)
    try:
        want = oracle.topk(g.n, g.u, g.v, g.w, p, 65536)
        assert want["count"] == 65536
        t, w = d.topk(p, 65536)
        assert_topk_equal(t, w, want, p, f"k=65536 p={p}")
        with pytest.raises(wt.WtriError) as ei:
            d.topk(p, 65537)
        assert ei.value.code == -5
    finally:
        d.free()


def test_huge_sparse_vertex_range():
    """5e7 vertex ids (26-bit row keys: three radix passes per row sort) and
    two triangles at the two ends of the id range, the rest isolated."""
    n = 50_000_000
    a, b, c = n - 3, n - 2, n - 1
    u = np.array([a, b, a, 0, 1, 0, 7], np.int32)
    v = np.array([b, c, c, 1, 2, 2, a], np.int32)
    w = np.array([5, 6, 7, 1, 1, 1, 9], np.int32)
    d = wt.build_csr(n, u, v, w)
    try:
        t, x = d.topk(1.0, 5)
        assert t.tolist() == [[a, b, c], [0, 1, 2]]
        assert x.tolist() == [18 / 3.0, 1.0]
        t, x = d.topk(-math.inf, 1)
        assert t.tolist() == [[a, b, c]] and x.tolist() == [5.0]
    finally:
        d.free()


@pytest.mark.parametrize("n", [5, 300, 5000])
def test_wheel_closed_form(n):
    """A hub joined to every vertex of a rim cycle: n triangles {i, i+1, hub},
    spokes weigh 2i+2 and rim edges 1, so the p = 1 order is by 2i+2j+5 and
    every p = -inf key is 1 (triple order)."""
    u = np.array(list(range(n)) * 2, np.int32)
    v = np.array([n] * n + [(i + 1) % n for i in range(n)], np.int32)
    w = np.array([2 * i + 2 for i in range(n)] + [1] * n, np.int32)
    tris = [tuple(sorted((i, (i + 1) % n, n))) for i in range(n)]
    key = {t: 2 * t[0] + 2 * t[1] + 5 for t in tris}
    d = wt.build_csr(n + 1, u, v, w)
    try:
        t1, w1 = d.topk(1.0, n)
        assert [tuple(x) for x in t1] == sorted(tris, key=lambda t: (-key[t], t))
        np.testing.assert_array_equal(w1, np.array(sorted(key.values(), reverse=True)) / 3.0)
        tm, wm = d.topk(-math.inf, n)
        assert [tuple(x) for x in tm] == sorted(tris) and np.all(wm == 1.0)
    finally:
        d.free()


def test_complete_graph_closed_form():
    n = 40
    iu, ju = np.triu_indices(n, 1)
    u, v = iu.astype(np.int32), ju.astype(np.int32)
    w = (iu + ju + 1).astype(np.int32)
    d = wt.build_csr(n, u, v, w)
    try:
        N = n * (n - 1) * (n - 2) // 6
        tris, wts = d.topk(1.0, N)
        assert tris.shape[0] == N
        sums = tris.sum(axis=1)
        # p = 1 key is 2(a+b+c)+3: non-increasing sums, ties by triple
        assert np.all(np.diff(sums) <= 0)
        assert tuple(tris[0]) == (n - 3, n - 2, n - 1)
        np.testing.assert_array_equal(wts, (2 * sums + 3) / 3.0)
    finally:
        d.free()


@pytest.mark.parametrize("p", [-1.0, -2.0, 0.5, 3.0])
@pytest.mark.parametrize("k", [1, 100, 2000])
def test_general_p_tiny(tiny, tiny_dev, p, k):
    """Finite p outside {0, 1, 2}: ranked by the fp64 mean; the GPU answer
    equals the oracle's under the fp64 rule (values within 1e-12 relative,
    membership may differ only within 1e-12 of the k-th value)."""
    from wtri_testutil import assert_topk_close
    want = oracle.topk(tiny.n, tiny.u, tiny.v, tiny.w, p, k)
    tris, wts = tiny_dev.topk(p, k)
    assert_topk_close(tris, wts, want["tri"], want["value"], f"tiny p={p} k={k}")


@pytest.mark.parametrize("seed", range(8))
def test_general_p_random_small(seed):
    from wtri_testutil import assert_topk_close
    rng = np.random.default_rng(7000 + seed)
    n = int(rng.integers(4, 60))
    g = synth.random_small_graph(n, float(rng.uniform(0.1, 0.9)), int(rng.integers(1, 9)), seed)
    if g.m == 0:
        return
    d = wt.build_csr(g.n, g.u, g.v, g.w)
    try:
        for p in (-1.0, -3.0, 0.5, 3.0):
            for k in (1, 7, 200):
                want = oracle.topk(g.n, g.u, g.v, g.w, p, k)
                tris, wts = d.topk(p, k)
                assert_topk_close(tris, wts, want["tri"], want["value"], f"seed={seed} p={p} k={k}")
    finally:
        d.free()


@pytest.mark.parametrize("p", [-1.0, 3.0])
def test_general_p_scaled(p):
    """A 1e6-edge Chung-Lu graph with Zipf(2) weights up to 1e6."""
    from wtri_testutil import assert_topk_close
    g = synth.scaled_mid_graph(100000, 1000000, seed=12)
    d = wt.build_csr(g.n, g.u, g.v, g.w)
    try:
        for k in (1000, 5000):
            want = oracle.topk(g.n, g.u, g.v, g.w, p, k)
            tris, wts = d.topk(p, k)
            assert_topk_close(tris, wts, want["tri"], want["value"], f"scaled p={p} k={k}")
    finally:
        d.free()


def test_general_p_refused_where_not_offered(tiny_dev):
    """The samplers and the batched call take the exact-key p only."""
    with pytest.raises(wt.WtriError) as ei:
        tiny_dev.sample_topk(-1.0, 10, 1000, 1)
    assert ei.value.code == -5
    with pytest.raises(wt.WtriError) as ei:
        wt.topk_batch([tiny_dev], [-1.0], [10])
    assert ei.value.code == -5
