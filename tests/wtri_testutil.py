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
