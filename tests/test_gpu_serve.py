"""Serving with continuous batching: every result equals the same query run
alone (wtri_topk), whether submitted in one burst, in waves while earlier
requests are still on the device, or through a small slot limit."""
import math
import threading
import time

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

wt = pytest.importorskip("paper_1910_00692_gb300")

PS = [-math.inf, 1.0, 2.0, math.inf]


@pytest.fixture(scope="module")
def graphs():
    gs = [synth.tiny_graph(0), synth.scaled_mid_graph(20000, 200000, seed=11),
          synth.scaled_mid_graph(100000, 1000000, seed=12)]
    ds = [wt.build_csr(g.n, g.u, g.v, g.w) for g in gs]
    yield gs, ds
    for d in ds:
        d.free()


def _alone(ds, gid, p, k, cache):
    key = (gid, p, k)
    if key not in cache:
        cache[key] = ds[gid].topk(p, k)
    return cache[key]


def _drain(srv, pending, timeout=120.0):
    out = {}
    t0 = time.time()
    while pending:
        for t in list(pending):
            r = srv.poll(t, pending[t][2])
            if r is not None:
                out[t] = r
                del pending[t]
        assert time.time() - t0 < timeout, "requests did not finish"
        time.sleep(0.0005)
    return out


def test_burst_and_waves_equal_alone(graphs):
    gs, ds = graphs
    srv = wt.Server(8 << 30, 64)
    gids = [srv.add_graph(d) for d in ds]
    rng = np.random.default_rng(5)
    cache = {}
    pending = {}
    # a burst, then waves submitted from another thread while it runs
    for _ in range(120):
        gid = int(rng.integers(0, 3))
        p = PS[int(rng.integers(0, 4))]
        k = int(rng.integers(1, 1200))
        pending[srv.submit(gids[gid], p, k)] = (gid, p, k)

    lock = threading.Lock()
    later = {}

    def waves():
        r2 = np.random.default_rng(6)
        for _ in range(6):
            time.sleep(0.01)
            for _ in range(20):
                gid = int(r2.integers(0, 3))
                p = PS[int(r2.integers(0, 4))]
                k = int(r2.integers(1, 1200))
                t = srv.submit(gids[gid], p, k)
                with lock:
                    later[t] = (gid, p, k)

    th = threading.Thread(target=waves)
    th.start()
    res = _drain(srv, dict(pending))
    th.join()
    res.update(_drain(srv, dict(later)))
    allq = dict(pending)
    allq.update(later)
    for t, (gid, p, k) in allq.items():
        tris, w, lat = res[t]
        at, aw = _alone(ds, gid, p, k, cache)
        assert np.array_equal(tris, at), (gid, p, k)
        assert np.array_equal(w, aw), (gid, p, k)
        assert lat >= 0
    st = srv.stats()
    assert st["admitted"] == len(allq)
    assert st["batches"] > 1          # requests were admitted in several micro-batches
    assert st["waiting"] == 0 and st["running"] == 0
    srv.free()


@pytest.mark.parametrize("coalesce", [True, False])
def test_same_graph_and_p_share_a_query(graphs, coalesce):
    """Requests on one graph with one p and many k (some above the number of
    triangles) submitted together: each gets exactly its own top-k, the
    prefix of the shared query's answer -- or, with coalescing off
    (WTRI_SERVER_COALESCE = 0), the answer of its own query."""
    gs, ds = graphs
    srv = wt.Server(8 << 30, 256)
    srv.set_coalesce(coalesce)
    gid = srv.add_graph(ds[0])
    ntri = len(ds[0].topk(1.0, 60000)[0])
    assert ntri < 20000
    ks = [1, 7, 100, 999, ntri - 1, ntri, ntri + 50, 20000, 3, 100]
    cache = {}
    for p in (1.0, 0.0, -math.inf):
        pending = {srv.submit(gid, p, k): (0, p, k) for k in ks}
        res = _drain(srv, dict(pending))
        for t, (g, pp, k) in pending.items():
            at, aw = _alone(ds, g, pp, k, cache)
            assert res[t][0].shape[0] == min(k, ntri)
            assert np.array_equal(res[t][0], at), (pp, k)
            assert np.array_equal(res[t][1], aw), (pp, k)
    srv.free()


def test_small_slot_limit(graphs):
    gs, ds = graphs
    srv = wt.Server(8 << 30, 3)
    gid = srv.add_graph(ds[1])
    pending = {srv.submit(gid, PS[i % 4], 50 + i): (1, PS[i % 4], 50 + i) for i in range(40)}
    res = _drain(srv, dict(pending))
    cache = {}
    for t, (g, p, k) in pending.items():
        at, _ = _alone(ds, g, p, k, cache)
        assert np.array_equal(res[t][0], at)
    assert srv.stats()["batches"] >= 40 // 3
    srv.free()


def test_server_errors(graphs):
    gs, ds = graphs
    srv = wt.Server(1 << 18, 8)          # 256 KB: no graph fits
    with pytest.raises(wt.WtriError) as ei:
        srv.add_graph(ds[0])
    assert ei.value.code == -2
    srv.free()
    srv = wt.Server(ds[0].info()["device_bytes"] + (20 << 20), 8)
    gid = srv.add_graph(ds[0])
    with pytest.raises(wt.WtriError) as ei:
        srv.submit(gid + 5, 1.0, 10)
    assert ei.value.code == -6
    with pytest.raises(wt.WtriError) as ei:
        srv.submit(gid, 0.5, 10)
    assert ei.value.code == -5
    with pytest.raises(wt.WtriError) as ei:
        srv.submit(gid, 1.0, 60000)          # scratch for k=60000 exceeds the budget
    assert ei.value.code == -2
    with pytest.raises(wt.WtriError) as ei:
        srv.poll(12345, 10)
    assert ei.value.code == -6
    t = srv.submit(gid, 1.0, 10)
    r = None
    t0 = time.time()
    while r is None and time.time() - t0 < 30:
        r = srv.poll(t, 10)
    assert r is not None and r[0].shape[0] == 10
    with pytest.raises(wt.WtriError):
        srv.poll(t, 10)                    # retired
    srv.free()
