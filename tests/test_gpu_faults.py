"""Failure detection on the GPU without a GPU fault: a bounded device-side
wait is made to run out on purpose (the test hook sets its poll bound to 0),
the query reports WTRI_ETIMEOUT through the C ABI, the copy it was waiting
for is drained before its block moves on, and the next query on the same
graph, with the default bound, is exact."""
import numpy as np
import pytest

import oracle
import synth
from wtri_testutil import assert_topk_equal

pytestmark = pytest.mark.gpu

wt = pytest.importorskip("paper_1910_00692_gb300")


@pytest.fixture(scope="module")
def scaled():
    g = synth.scaled_mid_graph(100_000, 1_000_000, seed=12)
    d = wt.build_csr(g.n, g.u, g.v, g.w)
    # every edge with more than one wedge goes to the long-scan kernel, whose
    # staged rows wait on an mbarrier
    d.set_tune(64, 8, 1)
    yield g, d
    d.free()


@pytest.mark.parametrize("p", [1.0, np.inf])  # p values whose query runs the long-scan kernel
def test_bounded_wait_times_out_then_recovers(scaled, p):
    g, d = scaled
    try:
        wt.debug_set_wait_limit(0)
        with pytest.raises(wt.WtriError) as ei:
            d.topk(p, 1000)
        assert ei.value.code == -4  # WTRI_ETIMEOUT
    finally:
        wt.debug_set_wait_limit(-1)
    want = oracle.topk(g.n, g.u, g.v, g.w, p, 1000)
    tris, wts = d.topk(p, 1000)
    assert_topk_equal(tris, wts, want, p, f"after timeout p={p}")


def test_device_query_reports_timeout_status(scaled):
    """The device-output query writes the status into d_count (no host
    round trip), and the graph stays usable."""
    torch = pytest.importorskip("torch")
    g, d = scaled
    dev = torch.device("cuda:0")
    t = torch.zeros((100, 3), dtype=torch.int32, device=dev)
    w = torch.zeros(100, dtype=torch.float64, device=dev)
    c = torch.zeros(1, dtype=torch.int32, device=dev)
    try:
        wt.debug_set_wait_limit(0)
        wt.topk_device(d, 2.0, 100, t, w, c)
        torch.cuda.synchronize()
        assert int(c.item()) == -4
    finally:
        wt.debug_set_wait_limit(-1)
    wt.topk_device(d, 2.0, 100, t, w, c)
    torch.cuda.synchronize()
    assert int(c.item()) == 100
    want = oracle.topk(g.n, g.u, g.v, g.w, 2.0, 100)
    assert np.array_equal(t.cpu().numpy(), want["tri"])
