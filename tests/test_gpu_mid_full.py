"""GPU parity at the full mid workload size (Chung-Lu n=1e6, m=2e7, exponent
2.1, d_max 5e4, Zipf(2) weights capped at 1e6; k=1000 at every supported p), the
configuration of the mid bench workload: every output element against the oracle."""
import pytest

import oracle
import synth
from wtri_testutil import PS, assert_topk_equal, check_structures

pytestmark = pytest.mark.gpu

wt = pytest.importorskip("paper_1910_00692_gb300")


@pytest.fixture(scope="module")
def mid():
    g = synth.mid_graph(1)
    d = wt.build_csr(g.n, g.u, g.v, g.w)
    yield g, d
    d.free()


@pytest.mark.parametrize("p", PS)
def test_mid_full_k1000(mid, p):
    g, d = mid
    want = oracle.topk(g.n, g.u, g.v, g.w, p, 1000)
    tris, wts = d.topk(p, 1000)
    assert_topk_equal(tris, wts, want, p, f"mid p={p}")


def test_mid_structures_whole(mid):
    """Every device structure of the full mid build (2e7 edges, rows up to
    ~35,000 entries) against the oracle's construction, whole arrays."""
    g, d = mid
    check_structures(g, d)
