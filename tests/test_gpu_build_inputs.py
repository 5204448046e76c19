"""The build's input handling on the GPU: device-resident edge arrays that
start on a 16-byte boundary (four edges per load) and arrays that do not
(one edge at a time) give the same structures as the oracle's, for edge
counts with every remainder mod 4; a bad edge is reported by its smallest
index on both paths, wherever it sits (a full quad or the ragged tail)."""
import numpy as np
import pytest

import oracle
import synth
from wtri_testutil import check_structures

pytestmark = pytest.mark.gpu

wt = pytest.importorskip("paper_1910_00692_gb300")
torch = pytest.importorskip("torch")


def _device(arrs, shift):
    """The arrays as CUDA tensors whose data start `shift` int32 past a fresh
    allocation (shift 0: 16-byte aligned; 1..3: not)."""
    out = []
    for a in arrs:
        buf = torch.zeros(a.shape[0] + 4, dtype=torch.int32, device="cuda")
        t = buf[shift:shift + a.shape[0]]
        t.copy_(torch.from_numpy(np.ascontiguousarray(a)))
        out.append(t)
    return out


@pytest.mark.parametrize("shift", [0, 1, 3])
@pytest.mark.parametrize("drop", [0, 1, 2, 3])
def test_device_inputs_every_alignment(shift, drop):
    g0 = synth.random_small_graph(60, 0.3, 9, 77)
    m = g0.m - drop
    g = synth.Graph(g0.n, g0.u[:m].copy(), g0.v[:m].copy(), g0.w[:m].copy()) if drop else g0
    u, v, w = _device((g.u, g.v, g.w), shift)
    assert (u.data_ptr() % 16 == 0) == (shift == 0)
    d = wt.build_csr(g.n, u, v, w)
    try:
        check_structures(g, d)
        want = oracle.topk(g.n, g.u, g.v, g.w, 1.0, 100)
        tris, _ = d.topk(1.0, 100)
        assert np.array_equal(tris, want["tri"])
    finally:
        d.free()


@pytest.mark.parametrize("shift", [0, 1])
@pytest.mark.parametrize("where", ["first", "quad_end", "tail", "two"])
def test_first_bad_edge_on_both_paths(shift, where):
    g = synth.random_small_graph(80, 0.3, 9, 5)
    m = g.m - 4 - (g.m % 4) + 3  # a ragged tail of three
    u, v, w = g.u[:m].copy(), g.v[:m].copy(), g.w[:m].copy()
    idx = {"first": 0, "quad_end": 4 * (m // 8) + 3, "tail": m - 1, "two": 4 * (m // 8) + 1}[where]
    w[idx] = 0
    if where == "two":
        w[m - 2] = -5  # a later bad edge: the smaller index is the one reported
    du, dv, dw = _device((u, v, w), shift)
    with pytest.raises(wt.WtriError) as ei:
        wt.build_csr(g.n, du, dv, dw)
    assert ei.value.code == -1
    assert f"invalid edge {idx}:" in str(ei.value), str(ei.value)
