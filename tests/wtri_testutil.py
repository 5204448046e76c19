"""Helpers shared by the GPU parity tests: comparison against the oracle."""
import math

import numpy as np

PS = [-math.inf, 0.0, 1.0, 2.0, math.inf]

# fp64 weights: the same IEEE expression on both sides ((a+b+c)/3.0,
# sqrt(q/3.0), max, min) is expected bit-identical; the stated bound for
# p = 2 is 1e-12 relative, which is what the tests enforce.  p = 0 reports
# cbrt(a*b*c), and the host and device cube roots may differ in the last
# bit: 1e-12 relative as well.
REL_TOL = {1.0: 0.0, math.inf: 0.0, -math.inf: 0.0, 2.0: 1e-12, 0.0: 1e-12}

# p values outside {-inf, 0, 1, 2, +inf}: ranked by the fp64 mean itself.
GENERAL_PS = [-1.0, -2.0, 0.5, 3.0]
GEN_TOL = 1e-12


def assert_topk_close(got_tris, got_w, want_tris, want_w, ctx="", rel=GEN_TOL):
    """Comparison for fp64-keyed p: the same count; the value sequences equal
    within `rel` relative; every triangle in both answers with values equal
    within `rel`; a triangle in only one answer only if its value is within
    `rel` of the k-th value (where rounding may decide membership); and each
    answer ordered by value, except within `rel`."""
    got_tris = np.asarray(got_tris).reshape(-1, 3)
    want_tris = np.asarray(want_tris).reshape(-1, 3)
    got_w = np.asarray(got_w, dtype=np.float64)
    want_w = np.asarray(want_w, dtype=np.float64)
    assert got_tris.shape[0] == want_tris.shape[0], f"{ctx}: count {got_tris.shape[0]} != {want_tris.shape[0]}"
    n = got_tris.shape[0]
    if n == 0:
        return
    assert np.all(np.abs(got_w - want_w) <= rel * np.abs(want_w)), f"{ctx}: value sequences differ"
    for w_ in (got_w, want_w):
        assert np.all(w_[1:] <= w_[:-1] * (1 + rel)), f"{ctx}: not ordered by value"
    gd = {tuple(int(x) for x in t): v for t, v in zip(got_tris, got_w)}
    wd = {tuple(int(x) for x in t): v for t, v in zip(want_tris, want_w)}
    kth = want_w[-1]
    for t in set(gd) | set(wd):
        if t in gd and t in wd:
            assert abs(gd[t] - wd[t]) <= rel * abs(wd[t]), f"{ctx}: value of {t}"
        else:
            v = gd.get(t, wd.get(t))
            assert abs(v - kth) <= rel * abs(kth), f"{ctx}: {t} (value {v}) in one answer only, k-th {kth}"


def assert_topk_equal(got_tris, got_w, want, p, ctx=""):
    wt = want["tri"]
    assert got_tris.shape[0] == want["count"], f"{ctx}: count {got_tris.shape[0]} != {want['count']}"
    if want["count"] == 0:
        return
    mism = np.nonzero(np.any(got_tris != wt, axis=1))[0]
    assert mism.size == 0, (f"{ctx}: first triple mismatch at rank {mism[0]}: "
                            f"{got_tris[mism[0]].tolist()} vs {wt[mism[0]].tolist()}")
    tol = REL_TOL[p]
    if tol == 0.0:
        bad = np.nonzero(got_w != want["value"])[0]
    else:
        bad = np.nonzero(np.abs(got_w - want["value"]) > tol * np.abs(want["value"]))[0]
    assert bad.size == 0, f"{ctx}: weight mismatch at rank {bad[0]}: {got_w[bad[0]]!r} vs {want['value'][bad[0]]!r}"


def check_structures(g, d):
    """Every device structure of a built graph against the oracle's
    independent construction, whole arrays, element by element."""
    import oracle
    perm = oracle.edge_order(g.w)
    assert np.array_equal(d.array("order_w"), g.w[perm])
    ou, ov = d.array("order_u"), d.array("order_v")
    assert np.array_equal(ou, g.u[perm]) and np.array_equal(ov, g.v[perm])
    rank = np.empty(g.m, np.int64)
    rank[perm] = np.arange(g.m)
    wrp, wcol, wwt, wrk = oracle.weight_sorted_rows(g.n, g.u, g.v, g.w)
    assert np.array_equal(d.array("rowptr"), wrp)
    assert np.array_equal(d.array("degree"), np.diff(wrp).astype(np.int32))
    assert np.array_equal(d.array("wcol"), wcol)
    assert np.array_equal(d.array("wwt"), wwt)
    assert np.array_equal(d.array("wrank"), wrk)
    del wrp, wcol, wwt, wrk
    orow, ocol, owt, oeid = oracle.oriented_csr(g.n, g.u, g.v, g.w)
    assert np.array_equal(d.array("orowptr"), orow)
    assert np.array_equal(d.array("ocol"), ocol)
    assert np.array_equal(d.array("owt"), owt)
    assert np.array_equal(d.array("orank"), rank[oeid])
