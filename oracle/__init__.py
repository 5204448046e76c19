"""CPU oracle for exact top-k weighted triangles (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never imports, links or executes anything here, and this
package never imports the product.

The C part (``wtri_oracle.c``) is plain brute force: NodeIterator++ with a
bounded heap, the paper's BF baseline (Sections 3 and 5.2), scoring each
triangle with the generalized p-mean of Eq. 1 through an exact integer key.
The numpy helpers below restate the intermediate structures the CUDA path
builds (edge order of Algorithm 2's first step, per-vertex weight-sorted
lists, the degree orientation) so that they can be compared one by one.

Parity pins (tests/test_oracle_*.py) check this oracle against closed forms,
an independent triangle count, hand-enumerated graphs in tests/golden/ and a
Python brute force on random small graphs.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wtri_oracle.c")
_SRC_DHL = os.path.join(_HERE, "wtri_dhl.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")

P_CODES = {-math.inf: 0, 1.0: 1, 2.0: 2, math.inf: 3, 0.0: 4}
P_GENERAL = 5  # any other finite p: fp64 key (the mean itself)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP) into oracle/_build/liboracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_DHL))):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", _SRC, _SRC_DHL, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(path)
        i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
        i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
        u64p = np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")
        f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
        I64P = ctypes.POINTER(ctypes.c_int64)
        L.or_validate.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i32p, i32p, I64P]
        L.or_sym_csr.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i32p, i32p,
                                 i64p, i32p, i32p, i64p]
        L.or_edge_order.argtypes = [ctypes.c_int64, i32p, i64p]
        L.or_oriented_csr.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i32p, i32p,
                                      i64p, i32p, i32p, i64p]
        L.or_score.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int32, ctypes.c_int32,
                               ctypes.c_int32, ctypes.POINTER(ctypes.c_uint64),
                               ctypes.POINTER(ctypes.c_double)]
        L.or_topk.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i32p, i32p, ctypes.c_int,
                              ctypes.c_double, ctypes.c_int64, ctypes.c_int, i32p, u64p, f64p, I64P,
                              I64P]
        L.or_count_triangles.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i32p, i32p, I64P]
        u64p_ = np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")
        u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
        L.or_philox4x64_10.argtypes = [u64p_, u64p_, u64p_]
        L.or_philox4x64_10.restype = None
        L.or_sample_edges.argtypes = [ctypes.c_int64, i32p, i64p, ctypes.c_int, ctypes.c_int64,
                                      ctypes.c_uint64, i64p]
        L.or_topk_of_sampled.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i32p, i32p, u8p,
                                         ctypes.c_int, ctypes.c_double, ctypes.c_int64, ctypes.c_int,
                                         i32p, u64p, f64p, I64P, I64P]
        L.or_topk_shard.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i32p, i32p, i64p, ctypes.c_int,
                                    ctypes.c_double, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                    ctypes.c_int, i32p, u64p, f64p, I64P, I64P]
        L.or_wedge_samples.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i32p, i32p, ctypes.c_int,
                                       ctypes.c_int64, ctypes.c_uint64, i32p, i32p, i32p, i32p]
        L.or_wedge_topk.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i32p, i32p, ctypes.c_int,
                                    ctypes.c_int64, ctypes.c_int64, ctypes.c_uint64, i32p, u64p, f64p,
                                    I64P, I64P]
        L.dhl_topk.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i32p, i32p, ctypes.c_int,
                               ctypes.c_int64, ctypes.c_double, i32p, u64p, f64p, I64P, i64p]
        L.dhl_alpha.argtypes = [ctypes.c_int, ctypes.c_double]
        L.dhl_alpha.restype = ctypes.c_double
        f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
        L.or_topk_real.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i32p, f32p, ctypes.c_int,
                                   ctypes.c_double, ctypes.c_int64, i32p, u64p, f64p, I64P, I64P]
        L.or_topk_real.restype = ctypes.c_int
        L.or_clique_topk.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i32p, i32p, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, i32p, u64p, f64p,
                                     I64P, I64P]
        for f in (L.dhl_topk, L.or_validate, L.or_sym_csr, L.or_edge_order, L.or_oriented_csr,
                  L.or_score, L.or_topk, L.or_count_triangles, L.or_sample_edges,
                  L.or_topk_of_sampled, L.or_topk_shard, L.or_wedge_samples, L.or_wedge_topk,
                  L.or_clique_topk):
            f.restype = ctypes.c_int
        _lib = L
    return _lib


class OracleError(ValueError):
    pass


def _arr(x):
    return np.ascontiguousarray(x, dtype=np.int32)


GEO_WMAX = (1 << 21) - 1  # p = 0 ranks by the product of the weights: exact below 2^63


def pcode(p: float) -> int:
    """p code of the C oracle: exact integer keys for -inf, 0, 1, 2, +inf;
    code 5 (an fp64 key) for any other finite p."""
    p = float(p)
    if math.isnan(p):
        raise OracleError("p is NaN")
    if p in P_CODES:
        return P_CODES[p]
    return P_GENERAL


def _check_geo(p, w):
    if p == 0.0 and w.shape[0] and int(w.max()) > GEO_WMAX:
        raise OracleError("p = 0 needs weights below 2^21 (exact product key)")


def validate(n, u, v, w):
    """Returns -1 if the edge list is a valid simple positive-weighted graph
    (apart from repeated pairs, which or_sym_csr detects), else the index of
    the first offending edge."""
    u, v, w = _arr(u), _arr(v), _arr(w)
    bad = ctypes.c_int64(0)
    lib().or_validate(n, u.shape[0], u, v, w, ctypes.byref(bad))
    return int(bad.value)


def sym_csr(n, u, v, w):
    """Symmetric CSR, rows ascending by id: (rowptr, col, wt, eid)."""
    u, v, w = _arr(u), _arr(v), _arr(w)
    m = u.shape[0]
    rowptr = np.zeros(n + 1, np.int64)
    col = np.zeros(2 * m, np.int32)
    wt = np.zeros(2 * m, np.int32)
    eid = np.zeros(2 * m, np.int64)
    rc = lib().or_sym_csr(n, m, u, v, w, rowptr, col, wt, eid)
    if rc != 0:
        raise OracleError(f"invalid graph (rc={rc})")
    return rowptr, col, wt, eid


def edge_order(w):
    """perm[r] = index of the r-th edge by (weight desc, index asc)."""
    w = _arr(w)
    perm = np.zeros(w.shape[0], np.int64)
    lib().or_edge_order(w.shape[0], w, perm)
    return perm


def oriented_csr(n, u, v, w):
    """Degree-oriented CSR (rank = (degree, id), low -> high), rows by id."""
    u, v, w = _arr(u), _arr(v), _arr(w)
    m = u.shape[0]
    orow = np.zeros(n + 1, np.int64)
    ocol = np.zeros(m, np.int32)
    owt = np.zeros(m, np.int32)
    oeid = np.zeros(m, np.int64)
    rc = lib().or_oriented_csr(n, m, u, v, w, orow, ocol, owt, oeid)
    if rc != 0:
        raise OracleError(f"invalid graph (rc={rc})")
    return orow, ocol, owt, oeid


def weight_sorted_rows(n, u, v, w):
    """Per-vertex neighbour lists ordered like the global edge order
    (weight desc, edge index asc).  Returns (rowptr, col, wt, rank) where
    rank is the position of the edge in edge_order()."""
    rowptr, col, wt, eid = sym_csr(n, u, v, w)
    perm = edge_order(w)
    rank = np.empty_like(perm)
    rank[perm] = np.arange(perm.shape[0], dtype=np.int64)
    r_ent = rank[eid]
    row_of = np.repeat(np.arange(n, dtype=np.int64), np.diff(rowptr))
    order = np.lexsort((r_ent, row_of))
    return rowptr, col[order], wt[order], r_ent[order]


def score(p, a, b, c):
    """(key, value) of one triangle with edge weights a, b, c (Eq. 1)."""
    key = ctypes.c_uint64(0)
    val = ctypes.c_double(0.0)
    rc = lib().or_score(pcode(p), float(p), int(a), int(b), int(c), ctypes.byref(key),
                        ctypes.byref(val))
    if rc != 0:
        raise OracleError("bad p")
    return int(key.value), float(val.value)


def topk(n, u, v, w, p, k, nthreads=0):
    """Exact top-k triangles.  Returns dict(tri [count,3] int32, key uint64,
    value float64, count, ntri)."""
    u, v, w = _arr(u), _arr(v), _arr(w)
    _check_geo(p, w)
    m = u.shape[0]
    k = int(k)
    tri = np.zeros(3 * max(k, 1), np.int32)
    key = np.zeros(max(k, 1), np.uint64)
    val = np.zeros(max(k, 1), np.float64)
    cnt = ctypes.c_int64(0)
    ntri = ctypes.c_int64(0)
    rc = lib().or_topk(n, m, u, v, w, pcode(p), float(p), k, int(nthreads), tri, key, val,
                       ctypes.byref(cnt), ctypes.byref(ntri))
    if rc != 0:
        raise OracleError(f"or_topk failed (rc={rc})")
    c = int(cnt.value)
    return {"tri": tri[: 3 * c].reshape(c, 3), "key": key[:c], "value": val[:c],
            "count": c, "ntri": int(ntri.value)}


def dhl_alpha(p, beta=2.0):
    """alpha_p = 2 - p / (p - 1 + beta) for power-law weights (Section 3.3)."""
    return float(lib().dhl_alpha(pcode(p), float(beta)))


def dhl_topk(n, u, v, w, p, k, alpha=None, beta=2.0):
    """The paper's dynamic heavy-light algorithm (Algorithm 2), single
    thread: exact top-k like topk().  alpha=None uses alpha_p for power-law
    weights of exponent beta; alpha <= 0 runs Auto-HL (Section 3.3).
    Adds 'stats': L->H moves, H->S moves, distinct triangles listed, edge
    probes, final h and l."""
    u, v, w = _arr(u), _arr(v), _arr(w)
    _check_geo(p, w)
    m = u.shape[0]
    k = int(k)
    if alpha is None:
        alpha = dhl_alpha(p, beta)
    tri = np.zeros(3 * max(k, 1), np.int32)
    key = np.zeros(max(k, 1), np.uint64)
    val = np.zeros(max(k, 1), np.float64)
    cnt = ctypes.c_int64(0)
    stats = np.zeros(6, np.int64)
    rc = lib().dhl_topk(n, m, u, v, w, pcode(p), k, float(alpha), tri, key, val, ctypes.byref(cnt), stats)
    if rc != 0:
        raise OracleError(f"dhl_topk failed (rc={rc})")
    c = int(cnt.value)
    names = ("light_to_heavy", "heavy_to_super", "listed", "probes", "h", "l")
    return {"tri": tri[: 3 * c].reshape(c, 3), "key": key[:c], "value": val[:c], "count": c,
            "stats": dict(zip(names, (int(x) for x in stats)))}


def philox4x64_10(counter, key):
    """One Philox4x64-10 block: counter (4 uint64), key (2 uint64) -> 4 uint64."""
    c = np.ascontiguousarray(np.array(counter, dtype=np.uint64).reshape(4))
    k = np.ascontiguousarray(np.array(key, dtype=np.uint64).reshape(2))
    out = np.zeros(4, np.uint64)
    lib().or_philox4x64_10(c, k, out)
    return out


def sample_edges(w, p, nsamples, seed):
    """Algorithm 3's edge draws (probability w^p / Z), p in {0, 1, 2} (p = 0:
    every edge equally likely).  Returns
    (perm, hits): hits[r] counts draws of the r-th edge of edge_order()."""
    w = _arr(w)
    perm = edge_order(w)
    hits = np.zeros(max(w.shape[0], 1), np.int64)
    rc = lib().or_sample_edges(w.shape[0], w, perm, pcode(p), int(nsamples),
                               ctypes.c_uint64(int(seed) & (2**64 - 1)), hits)
    if rc != 0:
        raise OracleError(f"or_sample_edges failed (rc={rc})")
    return perm, hits[: w.shape[0]]


def topk_of_marked(n, u, v, w, mark, p, k, nthreads=0):
    """Top-k of the triangles that have at least one marked edge (mark[i] != 0
    for input edge i): the triangle set T of Algorithm 3 for a given draw."""
    u, v, w = _arr(u), _arr(v), _arr(w)
    _check_geo(p, w)
    m = u.shape[0]
    mark = np.ascontiguousarray(mark, dtype=np.uint8)
    k = int(k)
    tri = np.zeros(3 * max(k, 1), np.int32)
    key = np.zeros(max(k, 1), np.uint64)
    val = np.zeros(max(k, 1), np.float64)
    cnt = ctypes.c_int64(0)
    ntri = ctypes.c_int64(0)
    rc = lib().or_topk_of_sampled(n, m, u, v, w, mark, pcode(p), float(p), k, int(nthreads), tri,
                                  key, val, ctypes.byref(cnt), ctypes.byref(ntri))
    if rc != 0:
        raise OracleError(f"or_topk_of_sampled failed (rc={rc})")
    c = int(cnt.value)
    return {"tri": tri[: 3 * c].reshape(c, 3), "key": key[:c], "value": val[:c], "count": c,
            "ntri": int(ntri.value)}


def sample_topk(n, u, v, w, p, k, nsamples, seed, nthreads=0):
    """Top-k of Algorithm 3's triangle set T (every triangle with at least one
    drawn edge).  Returns the topk() dict plus 'sampled_edges'."""
    u, v, w = _arr(u), _arr(v), _arr(w)
    m = u.shape[0]
    perm, hits = sample_edges(w, p, nsamples, seed)
    mark = np.zeros(max(m, 1), np.uint8)
    mark[perm[hits > 0]] = 1
    r = topk_of_marked(n, u, v, w, mark[:m], p, k, nthreads)
    r["sampled_edges"] = int((hits > 0).sum())
    return r


def topk_shard(n, u, v, w, p, k, shard, nshards, chunk_shift=10):
    """Top-k of the triangles whose first edge in the edge order falls in
    shard `shard` (edge positions dealt in chunks of 2^chunk_shift,
    round-robin over nshards)."""
    u, v, w = _arr(u), _arr(v), _arr(w)
    _check_geo(p, w)
    m = u.shape[0]
    perm = edge_order(w)
    rank = np.empty(max(m, 1), np.int64)
    rank[perm] = np.arange(m, dtype=np.int64)
    k = int(k)
    tri = np.zeros(3 * max(k, 1), np.int32)
    key = np.zeros(max(k, 1), np.uint64)
    val = np.zeros(max(k, 1), np.float64)
    cnt = ctypes.c_int64(0)
    ntri = ctypes.c_int64(0)
    rc = lib().or_topk_shard(n, m, u, v, w, rank, pcode(p), float(p), k, int(shard), int(nshards),
                             int(chunk_shift), tri, key, val, ctypes.byref(cnt), ctypes.byref(ntri))
    if rc != 0:
        raise OracleError(f"or_topk_shard failed (rc={rc})")
    c = int(cnt.value)
    return {"tri": tri[: 3 * c].reshape(c, 3), "key": key[:c], "value": val[:c], "count": c,
            "ntri": int(ntri.value)}


def count_triangles(n, u, v, w=None):
    u, v = _arr(u), _arr(v)
    if w is None:
        w = np.ones(u.shape[0], np.int32)
    w = _arr(w)
    out = ctypes.c_int64(0)
    rc = lib().or_count_triangles(n, u.shape[0], u, v, w, ctypes.byref(out))
    if rc != 0:
        raise OracleError(f"invalid graph (rc={rc})")
    return int(out.value)


if __name__ == "__main__":  # pragma: no cover
    build(force="--force" in sys.argv)
    print(_LIB_PATH)


def wedge_samples(n, u, v, w, p, nsamples, seed):
    """Algorithm 4's draws (Eqs. 6-8), p in {0, 1, 2}: per sample the center
    a, the positions jb, jc of b and c in a's weight-sorted row, and the
    sorted triangle (or -1s when the wedge does not close)."""
    u, v, w = _arr(u), _arr(v), _arr(w)
    ns = int(nsamples)
    center = np.zeros(max(ns, 1), np.int32)
    jb = np.zeros(max(ns, 1), np.int32)
    jc = np.zeros(max(ns, 1), np.int32)
    tri = np.zeros(3 * max(ns, 1), np.int32)
    rc = lib().or_wedge_samples(n, u.shape[0], u, v, w, pcode(p), ns,
                                ctypes.c_uint64(int(seed) & (2**64 - 1)), center, jb, jc, tri)
    if rc != 0:
        raise OracleError(f"or_wedge_samples failed (rc={rc})")
    return center[:ns], jb[:ns], jc[:ns], tri[: 3 * ns].reshape(ns, 3)


def wedge_topk(n, u, v, w, p, k, nsamples, seed):
    """Top-k of Algorithm 4's triangle set T (distinct closed wedges)."""
    u, v, w = _arr(u), _arr(v), _arr(w)
    k = int(k)
    tri = np.zeros(3 * max(k, 1), np.int32)
    key = np.zeros(max(k, 1), np.uint64)
    val = np.zeros(max(k, 1), np.float64)
    cnt = ctypes.c_int64(0)
    ntri = ctypes.c_int64(0)
    rc = lib().or_wedge_topk(n, u.shape[0], u, v, w, pcode(p), k, int(nsamples),
                             ctypes.c_uint64(int(seed) & (2**64 - 1)), tri, key, val, ctypes.byref(cnt),
                             ctypes.byref(ntri))
    if rc != 0:
        raise OracleError(f"or_wedge_topk failed (rc={rc})")
    c = int(cnt.value)
    return {"tri": tri[: 3 * c].reshape(c, 3), "key": key[:c], "value": val[:c], "count": c,
            "ntri": int(ntri.value)}


CLIQUE_P2_WMAX = 1 << 30  # p = 2 ranks cliques by the sum of ten squares: exact below 2^64


def clique_topk(n, u, v, w, q, p, k, edge_sampled=None):
    """Top-k q-cliques (q = 4, 5) by the p-mean of their edge weights (Section
    4.5, Appendix A), p in {-inf, 1, 2, +inf}.  edge_sampled (one flag per
    input edge, or None for every clique): only cliques with a flagged edge.
    Returns dict(ids (count x q), key, value, count, ncliques)."""
    u, v, w = _arr(u), _arr(v), _arr(w)
    pc = pcode(p)
    if pc > 3:
        raise OracleError("cliques rank at p in {-inf, 1, 2, +inf}")
    k = int(k)
    ids = np.zeros(max(k, 1) * q, np.int32)
    key = np.zeros(max(k, 1), np.uint64)
    val = np.zeros(max(k, 1), np.float64)
    cnt = ctypes.c_int64(0)
    ncl = ctypes.c_int64(0)
    flags = None
    if edge_sampled is not None:
        flags = np.ascontiguousarray(edge_sampled, dtype=np.uint8)
        if flags.shape[0] != u.shape[0]:
            raise OracleError("edge_sampled needs one flag per edge")
    rc = lib().or_clique_topk(n, u.shape[0], u, v, w, int(q), pc,
                              None if flags is None else flags.ctypes.data_as(ctypes.c_void_p),
                              k, ids, key, val, ctypes.byref(cnt), ctypes.byref(ncl))
    if rc != 0:
        raise OracleError(f"or_clique_topk failed (rc={rc})")
    c = cnt.value
    return {"ids": ids[:c * q].reshape(-1, q), "key": key[:c], "value": val[:c], "count": c,
            "ncliques": ncl.value}


def sampled_edge_flags(w, p, nsamples, seed):
    """One flag per input edge: drawn at least once by Algorithm 3's sampler."""
    perm, hits = sample_edges(w, p, nsamples, seed)
    flags = np.zeros(len(w), np.uint8)
    flags[perm[hits > 0]] = 1
    return flags


def topk_real(n, u, v, w, p, k):
    """Top-k triangles of a graph with positive finite fp32 weights (Eq. 1
    over reals), ranked by the fp64 mean.  Returns dict(tri, key, value,
    count, ntri) like topk()."""
    u, v = _arr(u), _arr(v)
    w = np.ascontiguousarray(w, dtype=np.float32)
    k = int(k)
    tri = np.zeros(max(k, 1) * 3, np.int32)
    key = np.zeros(max(k, 1), np.uint64)
    val = np.zeros(max(k, 1), np.float64)
    cnt = ctypes.c_int64(0)
    nt = ctypes.c_int64(0)
    rc = lib().or_topk_real(n, u.shape[0], u, v, w, pcode(p), float(p), k, tri, key, val,
                            ctypes.byref(cnt), ctypes.byref(nt))
    if rc != 0:
        raise OracleError(f"or_topk_real failed (rc={rc})")
    c = cnt.value
    return {"tri": tri[:3 * c].reshape(-1, 3), "key": key[:c], "value": val[:c], "count": c,
            "ntri": nt.value}
