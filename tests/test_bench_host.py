"""Host-side logic of bench.py (no GPU): the serving queue arithmetic with
stand-in server and graphs, the measured-peak lookup, and the rule that the
committed ncu traffic is only reported while the kernel sources match."""
import importlib.util
import json
import os
import time
import types

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


class _FakeServer:
    """Completes every request 1 ms after submission."""

    def __init__(self, *_):
        self.n = 0
        self.coalesce = True

    def set_coalesce(self, on):
        self.coalesce = on

    def add_graph(self, d):
        return 0

    def submit(self, gid, p, k):
        self.n += 1
        return self.n

    def poll(self, ticket, k):
        return (None, None, 0.001)

    def stats(self):
        return {"batches": 7, "retries": 0}

    def free(self):
        pass


class _FakeGraph:
    def __init__(self, service_s):
        self.service_s = service_s

    def topk(self, p, k):
        time.sleep(self.service_s)


def test_serve_run_queue_arithmetic():
    b = _bench()
    wt = types.SimpleNamespace(Server=_FakeServer)
    # service 2 ms per request at 1,000 req/s offered: the sequential loop is
    # over capacity, so its latency grows along the stream
    r = b.serve_run(wt, [_FakeGraph(0.002)], [10], 1000.0, 300, 200, "test")
    assert r["requests"] == 300 and r["sequential_requests"] == 200
    assert r["p50_ms"] == 1.0 and r["p99_ms"] == 1.0
    assert r["sequential_mean_service_ms"] >= 2.0
    assert r["sequential_p99_ms"] > r["sequential_p50_ms"] > 2.0
    assert r["sequential_qps"] < 1000.0
    assert r["server_first_requests_p50_ms"] == 1.0
    json.dumps(r)


def test_serve_run_without_coalescing_or_baseline():
    b = _bench()
    wt = types.SimpleNamespace(Server=_FakeServer)
    r = b.serve_run(wt, [_FakeGraph(0.001)], [10], 5000.0, 100, 0, "test", coalesce=False)
    assert r["coalesce"] is False and r["requests"] == 100
    assert "sequential_requests" not in r and "server_first_requests_p50_ms" not in r
    json.dumps(r)


def test_serve_run_sequential_budget():
    b = _bench()
    wt = types.SimpleNamespace(Server=_FakeServer)
    r = b.serve_run(wt, [_FakeGraph(0.001)], [10], 5000.0, 400, 400, "test", seq_budget_s=0.02)
    assert 1 <= r["sequential_requests"] < 400


def test_measured_peak_reads_the_file():
    b = _bench()
    peak, kind = b.measured_peak()
    if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")):
        assert kind == "measured" and peak > 1000
    else:
        assert kind == "fallback" and peak == b.FALLBACK_HBM_GBS


def test_ncu_traffic_tracks_the_sources(tmp_path):
    import hashlib
    b = _bench()
    src = "bench.py"
    digest = hashlib.sha256(open(os.path.join(ROOT, src), "rb").read()).hexdigest()
    cap = tmp_path / "radix_downsweep_traffic_large.txt"
    cap.write_text(f"how: test capture\ndram_bytes_per_launch: 123.0\nsources: {src}\n"
                   f"source_sha256: {digest}\n")
    traffic, why = b.ncu_traffic("radix_downsweep", "large", str(tmp_path))
    assert traffic == 123.0 and why == "test capture"
    cap.write_text(f"dram_bytes_per_launch: 123.0\nsources: {src}\nsource_sha256: {'0' * 64}\n")
    traffic, why = b.ncu_traffic("radix_downsweep", "large", str(tmp_path))
    assert traffic is None and "changed" in why
    traffic, why = b.ncu_traffic("radix_downsweep", "mid", str(tmp_path))
    assert traffic is None and "no capture" in why


def test_host_arrays_prefix():
    b = _bench()
    g = types.SimpleNamespace(u=np.arange(10, dtype=np.int32), v=np.arange(10, dtype=np.int32) + 1,
                              w=np.ones(10, np.int32), m=10)
    u, v, w = b.host_arrays(g, 4)
    assert u.tolist() == [0, 1, 2, 3] and v.tolist() == [1, 2, 3, 4]
