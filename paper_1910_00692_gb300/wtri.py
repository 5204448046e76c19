"""ctypes binding of libwtri.so (argument marshalling only).

Names follow the C ABI: ``build_csr`` -> wtri_build_csr, ``topk`` ->
wtri_topk, ``topk_device`` -> wtri_topk_device, ``sample_topk`` ->
wtri_sample_topk.  Host inputs are numpy arrays; device inputs and outputs
are torch CUDA tensors (torch provides device memory and streams only).
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_lib", "libwtri.so")

WTRI_OK = 0
WTRI_PENDING = 1
CODES = {
    -1: "WTRI_EINVAL",
    -2: "WTRI_ENOMEM",
    -3: "WTRI_ECUDA",
    -4: "WTRI_ETIMEOUT",
    -5: "WTRI_EUNSUPPORTED",
    -6: "WTRI_ENOTFOUND",
}

ARRAYS = {
    "degree": (0, np.int32, "n"),
    "rowptr": (1, np.int64, "n+1"),
    "order_u": (2, np.int32, "m"),
    "order_v": (3, np.int32, "m"),
    "order_w": (4, np.int32, "m"),
    "wcol": (5, np.int32, "2m"),
    "wwt": (6, np.int32, "2m"),
    "wrank": (7, np.int32, "2m"),
    "orowptr": (11, np.int64, "n+1"),
    "ocol": (12, np.int32, "m"),
    "owt": (13, np.int32, "m"),
    "orank": (14, np.int32, "m"),
}


class WtriUnavailable(RuntimeError):
    """libwtri.so is missing or cannot be loaded: build it first
    (``python -c "import __graft_entry__ as g; g.build()"``)."""


class WtriError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{CODES.get(code, code)}: {msg}")
        self.code = code


class _Tri(ctypes.Structure):
    _fields_ = [("a", ctypes.c_int32), ("b", ctypes.c_int32), ("c", ctypes.c_int32)]


class _TuneInfo(ctypes.Structure):
    _fields_ = [("first_round", ctypes.c_int64), ("growth", ctypes.c_int32), ("t_short", ctypes.c_int32),
                ("default_ms", ctypes.c_double), ("tuned_ms", ctypes.c_double),
                ("configs_tried", ctypes.c_int32)]


class _Result(ctypes.Structure):
    _fields_ = [("tris", ctypes.c_void_p), ("weight", ctypes.c_void_p),
                ("capacity", ctypes.c_int32), ("count", ctypes.c_int32)]


_lib = None


def lib_path() -> str:
    return _LIB_PATH


def lib():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise WtriUnavailable(f"{_LIB_PATH} not built")
    try:
        L = ctypes.CDLL(_LIB_PATH)
    except OSError as e:  # pragma: no cover
        raise WtriUnavailable(str(e)) from e
    vp, i32, i64, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    L.wtri_build_csr.argtypes = [i32, i64, vp, vp, vp, ctypes.c_int, vp, ctypes.POINTER(vp)]
    L.wtri_build_csr_f32.argtypes = [i32, i64, vp, vp, vp, ctypes.c_int, vp, ctypes.POINTER(vp)]
    L.wtri_graph_free.argtypes = [vp]
    L.wtri_graph_free.restype = None
    L.wtri_graph_info.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i64), ctypes.POINTER(i32),
                                  ctypes.POINTER(i32), ctypes.POINTER(i64)]
    L.wtri_topk.argtypes = [vp, f64, i32, ctypes.POINTER(_Result)]
    L.wtri_topk_device.argtypes = [vp, f64, i32, vp, vp, vp, vp]
    L.wtri_topk_device_noalloc.argtypes = [vp, f64, i32, vp, vp, vp, vp]
    L.wtri_sample_topk.argtypes = [vp, f64, i32, i64, ctypes.c_uint64, ctypes.POINTER(_Result)]
    L.wtri_graph_copy_array.argtypes = [vp, ctypes.c_int, vp, i64, ctypes.POINTER(i64)]
    L.wtri_sample_edges.argtypes = [vp, f64, i64, ctypes.c_uint64, vp, i64]
    L.wtri_wedge_topk.argtypes = [vp, f64, i32, i64, ctypes.c_uint64, ctypes.POINTER(_Result)]
    L.wtri_sample_wedges.argtypes = [vp, f64, i64, ctypes.c_uint64, vp, vp, vp, vp]
    L.wtri_sample_cliques.argtypes = [vp, i32, f64, i32, i64, ctypes.c_uint64, vp, vp, vp,
                                      ctypes.POINTER(i32)]
    L.wtri_topk_batch.argtypes = [vp, vp, vp, i32, vp]
    L.wtri_topk_shard.argtypes = [vp, f64, i32, i32, i32, ctypes.POINTER(_Result), vp]
    L.wtri_autotune.argtypes = [vp, i32, i32, ctypes.POINTER(_TuneInfo)]
    L.wtri_set_tune.argtypes = [vp, i64, i32, i32]
    L.wtri_autotune_buckets.argtypes = [vp, i32, i32, i32, ctypes.POINTER(i32)]
    L.wtri_autotune_buckets.restype = ctypes.c_int
    L.wtri_merge_topk.argtypes = [i32, vp, vp, vp, vp, i32, ctypes.POINTER(_Result), vp]
    u64 = ctypes.c_uint64
    L.wtri_server_create.argtypes = [u64, i32, ctypes.POINTER(vp)]
    L.wtri_server_add_graph.argtypes = [vp, vp, ctypes.POINTER(i32)]
    L.wtri_submit.argtypes = [vp, i32, f64, i32, ctypes.POINTER(u64)]
    L.wtri_poll.argtypes = [vp, u64, ctypes.POINTER(_Result)]
    L.wtri_poll_timed.argtypes = [vp, u64, ctypes.POINTER(_Result), ctypes.POINTER(f64)]
    L.wtri_server_stats.argtypes = [vp, ctypes.POINTER(u64), ctypes.POINTER(u64), ctypes.POINTER(i32),
                                    ctypes.POINTER(i32), ctypes.POINTER(u64), ctypes.POINTER(u64)]
    L.wtri_debug_set_wait_limit.argtypes = [i64]
    L.wtri_debug_set_wait_limit.restype = ctypes.c_int
    L.wtri_server_set_option.argtypes = [vp, ctypes.c_int, i64]
    L.wtri_server_set_option.restype = ctypes.c_int
    L.wtri_server_free.argtypes = [vp]
    L.wtri_server_free.restype = None
    L.wtri_last_error.restype = ctypes.c_char_p
    L.wtri_last_error.argtypes = []
    L.wtri_version.restype = ctypes.c_char_p
    for f in (L.wtri_build_csr, L.wtri_build_csr_f32, L.wtri_graph_info, L.wtri_topk, L.wtri_topk_device,
              L.wtri_topk_device_noalloc,
              L.wtri_sample_topk, L.wtri_graph_copy_array, L.wtri_sample_edges,
              L.wtri_topk_batch, L.wtri_server_create, L.wtri_server_add_graph, L.wtri_submit,
              L.wtri_poll, L.wtri_poll_timed, L.wtri_server_stats, L.wtri_topk_shard,
              L.wtri_merge_topk, L.wtri_autotune, L.wtri_set_tune, L.wtri_wedge_topk,
              L.wtri_sample_cliques,
              L.wtri_sample_wedges):
        f.restype = ctypes.c_int
    _lib = L
    return L


def _check(rc: int):
    if rc != WTRI_OK:
        raise WtriError(rc, lib().wtri_last_error().decode())


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream


def _dev_ptr(t):
    return ctypes.c_void_p(int(t.data_ptr()))


class Graph:
    """A device-resident graph built by wtri_build_csr."""

    def __init__(self, handle: int):
        self._h = ctypes.c_void_p(handle)

    @property
    def handle(self):
        return self._h

    def free(self):
        if self._h:
            lib().wtri_graph_free(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):  # pragma: no cover
        try:
            self.free()
        except Exception:
            pass

    def info(self):
        n, m = ctypes.c_int32(), ctypes.c_int64()
        md, mw, nb = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
        _check(lib().wtri_graph_info(self._h, ctypes.byref(n), ctypes.byref(m), ctypes.byref(md),
                                     ctypes.byref(mw), ctypes.byref(nb)))
        return {"n": n.value, "m": m.value, "max_degree": md.value, "max_weight": mw.value,
                "device_bytes": nb.value}

    def array(self, name: str) -> np.ndarray:
        which, dt, _ = ARRAYS[name]
        nb = ctypes.c_int64()
        _check(lib().wtri_graph_copy_array(self._h, which, None, 0, ctypes.byref(nb)))
        out = np.empty(nb.value // np.dtype(dt).itemsize, dtype=dt)
        _check(lib().wtri_graph_copy_array(self._h, which, out.ctypes.data_as(ctypes.c_void_p),
                                           nb.value, ctypes.byref(nb)))
        return out

    def topk(self, p: float, k: int):
        return topk(self, p, k)

    def autotune(self, k: int = 1000, reps: int = 3) -> dict:
        """wtri_autotune: times the schedule grid on this graph and keeps the best."""
        info = _TuneInfo()
        _check(lib().wtri_autotune(self._h, int(k), int(reps), ctypes.byref(info)))
        return {"first_round": info.first_round, "growth": info.growth, "t_short": info.t_short,
                "default_ms": info.default_ms, "tuned_ms": info.tuned_ms,
                "configs_tried": info.configs_tried}

    def set_tune(self, first_round: int, growth: int, t_short: int):
        _check(lib().wtri_set_tune(self._h, int(first_round), int(growth), int(t_short)))

    def sample_topk(self, p: float, k: int, nsamples: int, seed: int):
        return sample_topk(self, p, k, nsamples, seed)


def build_csr(n: int, u, v, w, stream=None) -> Graph:
    """u, v: int32; w: int32 (wtri_build_csr) or float32 (wtri_build_csr_f32,
    real weights).  numpy arrays (host) or torch CUDA tensors (device)."""
    on_device = 0
    keep = []
    real = str(getattr(w, "dtype", "")) in ("float32", "torch.float32")
    if hasattr(u, "is_cuda") and u.is_cuda:
        for t, want in ((u, "torch.int32"), (v, "torch.int32"),
                        (w, "torch.float32" if real else "torch.int32")):
            if not (hasattr(t, "is_cuda") and t.is_cuda) or str(t.dtype) != want:
                raise TypeError("device inputs must be CUDA tensors: int32 ids, int32 or float32 weights")
            if not t.is_contiguous():
                raise TypeError("device inputs must be contiguous")
        ptrs = [_dev_ptr(t) for t in (u, v, w)]
        m = int(u.shape[0])
        on_device = 1
    else:
        arrs = [np.ascontiguousarray(u, dtype=np.int32), np.ascontiguousarray(v, dtype=np.int32),
                np.ascontiguousarray(w, dtype=np.float32 if real else np.int32)]
        keep = arrs
        ptrs = [a.ctypes.data_as(ctypes.c_void_p) for a in arrs]
        m = int(arrs[0].shape[0])
    h = ctypes.c_void_p()
    build = lib().wtri_build_csr_f32 if real else lib().wtri_build_csr
    rc = build(int(n), m, ptrs[0], ptrs[1], ptrs[2], on_device, _stream_ptr(stream), ctypes.byref(h))
    del keep
    _check(rc)
    return Graph(h.value)


def _host_query(fn, k):
    tris = np.zeros((max(k, 1), 3), dtype=np.int32)
    wts = np.zeros(max(k, 1), dtype=np.float64)
    res = _Result(tris.ctypes.data, wts.ctypes.data, max(k, 1), 0)
    _check(fn(ctypes.byref(res)))
    c = res.count
    return tris[:c].copy(), wts[:c].copy()


def topk(g: Graph, p: float, k: int):
    """Exact top-k: (tris int32 [count,3] ascending ids, weights float64)."""
    return _host_query(lambda r: lib().wtri_topk(g.handle, float(p), int(k), r), int(k))


def topk_device(g: Graph, p: float, k: int, out_tris, out_weight, out_count, stream=None):
    """Stream-ordered query into torch CUDA tensors: out_tris int32 [k,3],
    out_weight float64 [k], out_count int32 [1]."""
    _check(lib().wtri_topk_device(g.handle, float(p), int(k), _dev_ptr(out_tris),
                                  _dev_ptr(out_weight), _dev_ptr(out_count), _stream_ptr(stream)))


def topk_device_noalloc(g: Graph, p: float, k: int, out_tris, out_weight, out_count, stream=None):
    """wtri_topk_device_noalloc: the same query with scratch taken from the
    library's fixed device array instead of any allocation (k <= 16384)."""
    _check(lib().wtri_topk_device_noalloc(g.handle, float(p), int(k), _dev_ptr(out_tris),
                                          _dev_ptr(out_weight), _dev_ptr(out_count),
                                          _stream_ptr(stream)))


def sample_topk(g: Graph, p: float, k: int, nsamples: int, seed: int):
    return _host_query(lambda r: lib().wtri_sample_topk(g.handle, float(p), int(k), int(nsamples),
                                                         ctypes.c_uint64(seed & (2**64 - 1)), r),
                       int(k))


def wedge_topk(g: Graph, p: float, k: int, nsamples: int, seed: int):
    """wtri_wedge_topk: top-k of Algorithm 4's triangle set (host results)."""
    return _host_query(lambda r: lib().wtri_wedge_topk(g.handle, float(p), int(k), int(nsamples),
                                                        ctypes.c_uint64(seed & (2**64 - 1)), r),
                       int(k))


def sample_wedges(g: Graph, p: float, nsamples: int, seed: int):
    """wtri_sample_wedges: (center, jb, jc, tri) of each draw of Algorithm 4."""
    ns = int(nsamples)
    center = np.zeros(max(ns, 1), np.int32)
    jb = np.zeros(max(ns, 1), np.int32)
    jc = np.zeros(max(ns, 1), np.int32)
    tri = np.zeros(3 * max(ns, 1), np.int32)
    _check(lib().wtri_sample_wedges(g.handle, float(p), ns, ctypes.c_uint64(int(seed) & (2**64 - 1)),
                                    center.ctypes.data_as(ctypes.c_void_p), jb.ctypes.data_as(ctypes.c_void_p),
                                    jc.ctypes.data_as(ctypes.c_void_p), tri.ctypes.data_as(ctypes.c_void_p)))
    return center[:ns], jb[:ns], jc[:ns], tri[: 3 * ns].reshape(ns, 3)


def topk_shard(g: Graph, p: float, k: int, shard: int, nshards: int):
    """wtri_topk_shard: exact top-k of the triangles owned by one shard.
    Returns (tris, weights, keys)."""
    tris = np.zeros((max(k, 1), 3), dtype=np.int32)
    wts = np.zeros(max(k, 1), dtype=np.float64)
    keys = np.zeros(max(k, 1), dtype=np.uint64)
    res = _Result(tris.ctypes.data, wts.ctypes.data, max(k, 1), 0)
    _check(lib().wtri_topk_shard(g.handle, float(p), int(k), int(shard), int(nshards), ctypes.byref(res),
                                 keys.ctypes.data_as(ctypes.c_void_p)))
    c = res.count
    return tris[:c].copy(), wts[:c].copy(), keys[:c].copy()


def sample_cliques(g: Graph, q: int, p: float, k: int, nsamples: int, seed: int):
    """wtri_sample_cliques: top-k q-cliques (q = 4, 5) on the edges drawn by
    edge sampling (nsamples < 0: every edge, the exact top-k).  Returns
    (cliques (count x q), weights, keys)."""
    cl = np.zeros((max(k, 1), q), dtype=np.int32)
    wts = np.zeros(max(k, 1), dtype=np.float64)
    keys = np.zeros(max(k, 1), dtype=np.uint64)
    cnt = ctypes.c_int32(0)
    _check(lib().wtri_sample_cliques(g.handle, int(q), float(p), int(k), int(nsamples),
                                     ctypes.c_uint64(int(seed) & (2**64 - 1)), cl.ctypes.data_as(ctypes.c_void_p),
                                     wts.ctypes.data_as(ctypes.c_void_p), keys.ctypes.data_as(ctypes.c_void_p),
                                     ctypes.byref(cnt)))
    c = cnt.value
    return cl[:c].copy(), wts[:c].copy(), keys[:c].copy()


def merge_topk(parts, k: int):
    """wtri_merge_topk (host code, no device): parts = [(tris, weights,
    keys), ...] -> the k best (tris, weights, keys)."""
    n = len(parts)
    prepared = [(np.ascontiguousarray(t, dtype=np.int32).reshape(-1, 3),
                 np.ascontiguousarray(w, dtype=np.float64),
                 np.ascontiguousarray(kk, dtype=np.uint64)) for t, w, kk in parts]
    counts = np.array([p_[0].shape[0] for p_ in prepared], dtype=np.int32)
    tp = (ctypes.c_void_p * max(n, 1))(*[p_[0].ctypes.data for p_ in prepared])
    wp = (ctypes.c_void_p * max(n, 1))(*[p_[1].ctypes.data for p_ in prepared])
    kp = (ctypes.c_void_p * max(n, 1))(*[p_[2].ctypes.data for p_ in prepared])
    tris = np.zeros((max(k, 1), 3), dtype=np.int32)
    wts = np.zeros(max(k, 1), dtype=np.float64)
    keys = np.zeros(max(k, 1), dtype=np.uint64)
    res = _Result(tris.ctypes.data, wts.ctypes.data, max(k, 1), 0)
    _check(lib().wtri_merge_topk(n, counts.ctypes.data_as(ctypes.c_void_p), ctypes.cast(tp, ctypes.c_void_p),
                                 ctypes.cast(wp, ctypes.c_void_p), ctypes.cast(kp, ctypes.c_void_p), int(k),
                                 ctypes.byref(res), keys.ctypes.data_as(ctypes.c_void_p)))
    c = res.count
    return tris[:c].copy(), wts[:c].copy(), keys[:c].copy()


def autotune_buckets(graphs, k: int = 1000, reps: int = 2) -> int:
    """wtri_autotune_buckets: tunes the largest graph of each size group and
    applies its schedule to the group; returns the number of groups."""
    n = len(graphs)
    handles = (ctypes.c_void_p * max(n, 1))(*[g.handle.value for g in graphs])
    out = ctypes.c_int32()
    _check(lib().wtri_autotune_buckets(ctypes.cast(handles, ctypes.c_void_p), n, int(k), int(reps),
                                       ctypes.byref(out)))
    return out.value


_RESULT_DTYPE = np.dtype([("tris", "<u8"), ("weight", "<u8"), ("capacity", "<i4"), ("count", "<i4")])


def topk_batch(graphs, ps, ks):
    """wtri_topk_batch: one batched launch for query i = (graphs[i], ps[i],
    ks[i]).  Returns a list of (tris, weights) like topk() (views into one
    result buffer for the whole batch)."""
    nq = len(graphs)
    if nq == 0:
        return []
    assert ctypes.sizeof(_Result) == _RESULT_DTYPE.itemsize
    handles = np.array([g.handle.value for g in graphs], dtype=np.uint64)
    p_arr = np.ascontiguousarray(ps, dtype=np.float64)
    k_arr = np.ascontiguousarray(ks, dtype=np.int32)
    caps = np.maximum(k_arr.astype(np.int64), 1)
    offs = np.zeros(nq + 1, dtype=np.int64)
    np.cumsum(caps, out=offs[1:])
    tris_all = np.zeros((int(offs[-1]), 3), dtype=np.int32)
    wts_all = np.zeros(int(offs[-1]), dtype=np.float64)
    res = np.zeros(nq, dtype=_RESULT_DTYPE)
    res["tris"] = tris_all.ctypes.data + 12 * offs[:-1]
    res["weight"] = wts_all.ctypes.data + 8 * offs[:-1]
    res["capacity"] = caps
    _check(lib().wtri_topk_batch(handles.ctypes.data_as(ctypes.c_void_p),
                                 p_arr.ctypes.data_as(ctypes.c_void_p),
                                 k_arr.ctypes.data_as(ctypes.c_void_p), nq,
                                 res.ctypes.data_as(ctypes.c_void_p)))
    ends = (offs[:-1] + res["count"]).tolist()
    starts = offs[:-1].tolist()
    return [(tris_all[a:b], wts_all[a:b]) for a, b in zip(starts, ends)]


class Server:
    """wtri_server_*: continuous-batching server over resident graphs."""

    PENDING = WTRI_PENDING

    def __init__(self, hbm_budget_bytes: int, max_slots: int):
        h = ctypes.c_void_p()
        _check(lib().wtri_server_create(ctypes.c_uint64(int(hbm_budget_bytes)), int(max_slots),
                                        ctypes.byref(h)))
        self._h = h
        self._graphs = []

    def add_graph(self, g: Graph) -> int:
        gid = ctypes.c_int32()
        _check(lib().wtri_server_add_graph(self._h, g.handle, ctypes.byref(gid)))
        self._graphs.append(g)
        return gid.value

    def submit(self, graph_id: int, p: float, k: int) -> int:
        t = ctypes.c_uint64()
        _check(lib().wtri_submit(self._h, int(graph_id), float(p), int(k), ctypes.byref(t)))
        return t.value

    def poll(self, ticket: int, k: int):
        """None while pending, else (tris, weights, latency_s)."""
        tris = np.zeros((max(k, 1), 3), dtype=np.int32)
        wts = np.zeros(max(k, 1), dtype=np.float64)
        res = _Result(tris.ctypes.data, wts.ctypes.data, max(k, 1), 0)
        lat = ctypes.c_double()
        rc = lib().wtri_poll_timed(self._h, ctypes.c_uint64(ticket), ctypes.byref(res), ctypes.byref(lat))
        if rc == WTRI_PENDING:
            return None
        _check(rc)
        return tris[:res.count].copy(), wts[:res.count].copy(), lat.value

    def stats(self):
        b, a, sc, rt = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        wq, rn = ctypes.c_int32(), ctypes.c_int32()
        _check(lib().wtri_server_stats(self._h, ctypes.byref(b), ctypes.byref(a), ctypes.byref(wq),
                                       ctypes.byref(rn), ctypes.byref(sc), ctypes.byref(rt)))
        return {"batches": b.value, "admitted": a.value, "waiting": wq.value, "running": rn.value,
                "scratch_bytes": sc.value, "retries": rt.value}

    def set_coalesce(self, on: bool):
        """WTRI_SERVER_COALESCE: same-(graph, p) requests of a micro-batch share one query."""
        _check(lib().wtri_server_set_option(self._h, 1, 1 if on else 0))

    def free(self):
        if self._h:
            lib().wtri_server_free(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):  # pragma: no cover
        try:
            self.free()
        except Exception:
            pass


def sample_edges(g: Graph, p: float, nsamples: int, seed: int) -> np.ndarray:
    """wtri_sample_edges: boolean mask over edge-order positions of the edges
    drawn by Algorithm 3 (probability w^p / Z per draw)."""
    m = g.info()["m"]
    words = (m + 31) // 32
    out = np.zeros(max(words, 1), dtype=np.uint32)
    _check(lib().wtri_sample_edges(g.handle, float(p), int(nsamples),
                                   ctypes.c_uint64(int(seed) & (2**64 - 1)),
                                   out.ctypes.data_as(ctypes.c_void_p), words))
    bits = np.unpackbits(out.view(np.uint8), bitorder="little")
    return bits[:m].astype(bool)


def debug_set_wait_limit(polls: int):
    """wtri_debug_set_wait_limit: fault injection for tests (polls of the
    long-scan kernel's first bounded wait; 0: every staged wait times out;
    negative: the default)."""
    _check(lib().wtri_debug_set_wait_limit(int(polls)))


def p_values():
    return [-math.inf, 0.0, 1.0, 2.0, math.inf]
