"""wtri_topk_device_noalloc: the top-k query for callers that cannot allocate
device memory while running (the scratch is a fixed array inside the
library).  Called through the C ABI, its output must match the allocating
wtri_topk_device on the same graph and query, on two calls in a row (the
second call reuses the array the first one left behind).

This file is collected last on purpose: it must pass alone in a fresh
process and after every other test.
"""

import numpy as np
import pytest

import synth
from wtri_testutil import PS, REL_TOL

pytestmark = pytest.mark.gpu

wt = pytest.importorskip("paper_1910_00692_gb300")
torch = pytest.importorskip("torch")


def _outputs(k, dev):
    return (torch.zeros((k, 3), dtype=torch.int32, device=dev),
            torch.zeros(k, dtype=torch.float64, device=dev),
            torch.zeros(1, dtype=torch.int32, device=dev))


def _read(t, w, c):
    n = int(c.item())
    assert n >= 0, f"device status {n}"
    return t[:n].cpu().numpy(), w[:n].cpu().numpy()


@pytest.mark.parametrize("graph", ["tiny", "scaled"])
def test_noalloc_matches_allocating_query(graph):
    dev = torch.device("cuda:0")
    g = synth.tiny_graph(0) if graph == "tiny" else synth.scaled_mid_graph(100_000, 1_000_000, seed=21)
    s = torch.cuda.Stream(device=dev)
    d = wt.build_csr(g.n, g.u, g.v, g.w, stream=s)
    try:
        for p in PS:
            for k in (1, 100, 1000):
                ref = _outputs(k, dev)
                wt.topk_device(d, p, k, *ref, stream=s)
                s.synchronize()
                rt, rw = _read(*ref)
                for call in range(2):
                    out = _outputs(k, dev)
                    wt.topk_device_noalloc(d, p, k, *out, stream=s)
                    s.synchronize()
                    ot, ow = _read(*out)
                    ctx = f"{graph} p={p} k={k} call={call}"
                    assert ot.shape == rt.shape, ctx
                    assert np.array_equal(ot, rt), ctx
                    tol = REL_TOL[p]
                    assert np.all(np.abs(ow - rw) <= tol * np.abs(rw)), ctx
    finally:
        d.free()


def test_noalloc_rejects_k_above_limit():
    g = synth.tiny_graph(0)
    d = wt.build_csr(g.n, g.u, g.v, g.w)
    try:
        out = _outputs(16385, torch.device("cuda:0"))
        with pytest.raises(wt.WtriError) as ei:
            wt.topk_device_noalloc(d, 1.0, 16385, *out)
        assert ei.value.code == -1
        assert "16384" in str(ei.value)
    finally:
        d.free()


def test_noalloc_overflow_reports_enomem_then_recovers():
    """K_300 with equal weights: every one of its 4,455,100 triangles ties at
    the k-th key, so a top-16384 query needs more candidate slots than the
    fixed array's 1,048,576.  The status word reports WTRI_ENOMEM (-2)
    instead of writing past the array; the call allocates no device memory;
    and the next call, on another graph, is correct."""
    dev = torch.device("cuda:0")
    s = torch.cuda.Stream(device=dev)
    n = 300
    iu, iv = np.triu_indices(n, 1)
    u, v = iu.astype(np.int32), iv.astype(np.int32)
    w = np.ones(u.shape[0], np.int32)
    dense = wt.build_csr(n, u, v, w, stream=s)
    g = synth.tiny_graph(0)
    d = wt.build_csr(g.n, g.u, g.v, g.w, stream=s)
    try:
        out = _outputs(16384, dev)
        wt.topk_device_noalloc(dense, 1.0, 16384, *out, stream=s)  # first call on the device
        s.synchronize()
        assert int(out[2].item()) == -2
        free0 = torch.cuda.mem_get_info(dev)[0]
        wt.topk_device_noalloc(dense, 1.0, 16384, *out, stream=s)
        s.synchronize()
        free1 = torch.cuda.mem_get_info(dev)[0]
        assert int(out[2].item()) == -2
        assert free1 == free0, (free0, free1)
        ref = _outputs(1000, dev)
        wt.topk_device(d, 1.0, 1000, *ref, stream=s)
        got = _outputs(1000, dev)
        wt.topk_device_noalloc(d, 1.0, 1000, *got, stream=s)
        s.synchronize()
        rt, rw = _read(*ref)
        gt, gw = _read(*got)
        assert np.array_equal(gt, rt) and np.array_equal(gw, rw)
    finally:
        dense.free()
        d.free()
