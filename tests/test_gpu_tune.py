"""Schedule tuning never changes results: extreme settings and the
autotuner's choice give the oracle's answer; the tuner picks a grid point
no slower than the defaults."""
import math

import pytest

import oracle
import synth
from wtri_testutil import PS, assert_topk_equal

pytestmark = pytest.mark.gpu

wt = pytest.importorskip("paper_1910_00692_gb300")


@pytest.mark.parametrize("which", ["tiny", "scaled"])
@pytest.mark.parametrize("tune", [(1, 2, 1), (3, 3, 2), (100000, 16, 1024)])
def test_extreme_settings_exact(which, tune):
    g = synth.tiny_graph(0) if which == "tiny" else synth.scaled_mid_graph(100000, 1000000, seed=12)
    d = wt.build_csr(g.n, g.u, g.v, g.w)
    try:
        d.set_tune(*tune)
        for p in PS:
            want = oracle.topk(g.n, g.u, g.v, g.w, p, 700)
            t, w = d.topk(p, 700)
            assert_topk_equal(t, w, want, p, f"{which} tune={tune} p={p}")
    finally:
        d.free()


def test_autotune_choice_exact():
    g = synth.scaled_mid_graph(100000, 1000000, seed=12)
    d = wt.build_csr(g.n, g.u, g.v, g.w)
    try:
        info = d.autotune(k=1000, reps=2)
        assert info["first_round"] in (32, 64, 256, 1024)
        assert info["growth"] in (4, 8, 16)
        assert info["t_short"] in (8, 16, 32, 64, 128)
        assert info["tuned_ms"] <= info["default_ms"] + 1e-9
        assert info["configs_tried"] == 60
        for p in PS:
            want = oracle.topk(g.n, g.u, g.v, g.w, p, 1000)
            t, w = d.topk(p, 1000)
            assert_topk_equal(t, w, want, p, f"tuned p={p}")
        res = wt.topk_batch([d, d], [1.0, -math.inf], [300, 300])
        for (t, w), p in zip(res, [1.0, -math.inf]):
            assert_topk_equal(t, w, oracle.topk(g.n, g.u, g.v, g.w, p, 300), p, "tuned batch")
    finally:
        d.free()


def test_tune_errors():
    g = synth.tiny_graph(0)
    d = wt.build_csr(g.n, g.u, g.v, g.w)
    try:
        with pytest.raises(wt.WtriError):
            d.set_tune(0, 8, 32)
        with pytest.raises(wt.WtriError):
            d.set_tune(64, 1, 32)
        with pytest.raises(wt.WtriError):
            d.autotune(k=0)
    finally:
        d.free()
