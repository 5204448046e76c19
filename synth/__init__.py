"""Seeded synthetic weighted graphs shaped like the paper's workloads.

This module only draws inputs.  It holds none of the top-k method's
arithmetic (no triangle enumeration, no scoring, no ordering of edges by
weight), so both the CPU oracle and the CUDA path can consume its output
without sharing any code with each other.

Recipe (the paper's datasets, Table 1 of Section 5, are not available; these
graphs stand in for them):

* Structure: "erased" Chung-Lu power-law graphs.  Expected degrees
  ``theta_i = c * (i + i0) ** (-1 / (gamma - 1))`` with ``i0`` and ``c`` solved
  so that ``theta_0 = d_max`` and ``sum(theta) = 2 m``.  Endpoint pairs are drawn
  i.i.d. proportional to ``theta``; self-loops and repeated pairs are dropped
  and the draw is topped up until exactly ``m`` distinct edges remain.
* Weights: i.i.d. and independent of structure (the paper's model in the
  analysis of Section 3.3).  Truncated Zipf ``P(w) ~ w**-s`` on ``{1..cap}`` is
  sampled by inverse CDF over an fp64 table (not clamped).  The tiny workload
  uses ``1 + Geometric(0.3)`` (support starting at 1) with an independent 1 %
  of edges drawn from truncated Zipf(1.5, 1e4).
* Edge order is shuffled and each edge's endpoint order is a coin flip, so no
  consumer can rely on sorted input.

Every array is int32, as the C-ABI takes it.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Graph",
    "chung_lu",
    "zipf_weights",
    "tiny_weights",
    "tiny_graph",
    "mid_graph",
    "batch_graph",
    "batch_queries",
    "scaled_mid_graph",
    "random_small_graph",
]


@dataclasses.dataclass
class Graph:
    n: int
    u: np.ndarray  # int32 [m]
    v: np.ndarray  # int32 [m]
    w: np.ndarray  # int32 [m]
    name: str = ""

    @property
    def m(self) -> int:
        return int(self.u.shape[0])


def _rng(seed, *substream) -> np.random.Generator:
    # Philox keyed by (seed, substream...) so that sub-draws are independent
    # of one another and of how many values earlier draws consumed.
    key = [int(seed) & 0xFFFFFFFFFFFFFFFF]
    for s in substream:
        key.append(int(s) & 0xFFFFFFFFFFFFFFFF)
    ss = np.random.SeedSequence(key)
    return np.random.Generator(np.random.Philox(ss))


def _expected_degrees(n: int, m: int, gamma: float, d_max: float) -> np.ndarray:
    a = 1.0 / (gamma - 1.0)
    idx = np.arange(n, dtype=np.float64)

    def total(i0: float) -> float:
        c = d_max * i0 ** a
        return float(np.sum(c * (idx + i0) ** (-a)))

    target = 2.0 * m
    lo, hi = 1e-9, 1e12
    if total(hi) < target:
        # Even a flat sequence cannot reach 2m below d_max: use it.
        return np.full(n, target / n)
    for _ in range(200):
        mid = math.sqrt(lo * hi)
        if total(mid) < target:
            lo = mid
        else:
            hi = mid
        if hi / lo < 1 + 1e-12:
            break
    i0 = hi
    c = d_max * i0 ** a
    return c * (idx + i0) ** (-a)


def chung_lu(n: int, m: int, gamma: float, d_max: float, seed, substream=(0,)):
    """Erased Chung-Lu graph with exactly ``m`` distinct undirected edges.

    Returns ``(u, v)`` int32 arrays in shuffled order.
    """
    if m > n * (n - 1) // 2:
        raise ValueError("m exceeds the number of vertex pairs")
    rng = _rng(seed, 1, *substream)
    theta = _expected_degrees(n, m, gamma, d_max)
    cdf = np.cumsum(theta)
    cdf /= cdf[-1]
    keys = np.empty(0, dtype=np.int64)
    need = m
    rounds = 0
    while need > 0:
        draw = int(need * 1.15) + 1024
        a = np.searchsorted(cdf, rng.random(draw), side="right").astype(np.int64)
        b = np.searchsorted(cdf, rng.random(draw), side="right").astype(np.int64)
        np.minimum(a, n - 1, out=a)
        np.minimum(b, n - 1, out=b)
        ok = a != b
        a, b = a[ok], b[ok]
        lo_ = np.minimum(a, b)
        hi_ = np.maximum(a, b)
        new = lo_ * n + hi_
        keys = np.unique(np.concatenate([keys, new]))
        if keys.shape[0] >= m:
            # Keep a uniformly random subset of exactly m distinct pairs.
            pick = rng.permutation(keys.shape[0])[:m]
            keys = keys[np.sort(pick)]
        need = m - keys.shape[0]
        rounds += 1
        if rounds > 1000:
            raise RuntimeError("Chung-Lu top-up did not converge")
    keys = keys[rng.permutation(m)]
    u = (keys // n).astype(np.int32)
    v = (keys % n).astype(np.int32)
    flip = rng.random(m) < 0.5
    u2 = np.where(flip, v, u)
    v2 = np.where(flip, u, v)
    return u2.astype(np.int32), v2.astype(np.int32)


def _zipf_table(s: float, cap: int) -> np.ndarray:
    x = np.arange(1, cap + 1, dtype=np.float64)
    cdf = np.cumsum(x ** (-s))
    cdf /= cdf[-1]
    return cdf


def zipf_weights(m: int, s: float, cap: int, rng: np.random.Generator) -> np.ndarray:
    """Truncated Zipf on {1..cap} by inverse CDF over an fp64 table."""
    cdf = _zipf_table(s, cap)
    w = np.searchsorted(cdf, rng.random(m), side="right") + 1
    np.minimum(w, cap, out=w)
    return w.astype(np.int32)


def tiny_weights(m: int, rng: np.random.Generator) -> np.ndarray:
    """1 + Geometric(0.3) on {0,1,...}; an independent 1 % from Zipf(1.5, 1e4)."""
    w = rng.geometric(0.3, size=m).astype(np.int64)  # numpy's support starts at 1
    heavy = rng.random(m) < 0.01
    w[heavy] = zipf_weights(int(heavy.sum()), 1.5, 10_000, rng)
    return w.astype(np.int32)


def tiny_graph(seed: int = 0) -> Graph:
    """n=2,000, exponent 2.1, 20,000 edges, d_max = sqrt(2m)."""
    n, m = 2000, 20_000
    u, v = chung_lu(n, m, 2.1, math.sqrt(2 * m), seed)
    w = tiny_weights(m, _rng(seed, 2))
    return Graph(n, u, v, w, name="chung-lu n=2000 m=20000 g=2.1 geom(0.3)+1%zipf(1.5,1e4)")


def mid_graph(seed: int = 1) -> Graph:
    """n=1e6, m=2e7, exponent 2.1, d_max 5e4, Zipf(2) weights capped at 1e6."""
    return scaled_mid_graph(1_000_000, 20_000_000, seed=seed)


def scaled_mid_graph(n: int, m: int, seed: int = 1, gamma: float = 2.1,
                     d_max: float | None = None, s: float = 2.0, cap: int = 1_000_000) -> Graph:
    """The mid workload's recipe at another size (d_max scales with sqrt(m))."""
    if d_max is None:
        d_max = 50_000.0 * math.sqrt(m / 20_000_000)
        d_max = min(d_max, n - 1)
    u, v = chung_lu(n, m, gamma, d_max, seed)
    w = zipf_weights(m, s, cap, _rng(seed, 2))
    return Graph(n, u, v, w, name=f"chung-lu n={n} m={m} g={gamma} zipf({s},{cap})")


def clique_graph(n: int, m: int, seed: int = 4) -> Graph:
    """Stand-in for the small, dense clique datasets (Appendix A, Table 3:
    hundreds to a thousand vertices, thousands to tens of thousands of
    edges, heavy-tailed co-occurrence counts): Chung-Lu with exponent 2.1 and
    d_max = n / 2, Zipf(1.7) weights capped at 5e4."""
    u, v = chung_lu(n, m, 2.1, n / 2.0, seed, substream=(30,))
    w = zipf_weights(m, 1.7, 50_000, _rng(seed, 31))
    return Graph(n, u, v, w, name=f"clique chung-lu n={n} m={m} zipf(1.7,5e4)")


def batch_graph(g: int, seed: int = 3, n_hi: int = 200_000) -> Graph:
    """Graph ``g`` of the 4,096-graph batch: n log-uniform in [100, n_hi]
    (2e5 for the batch workload), m = 10 n, exponent 2.2, Zipf(2) weights
    capped at 1e6."""
    rng = _rng(seed, 10, g)
    n = int(round(math.exp(rng.uniform(math.log(100), math.log(n_hi)))))
    m = min(10 * n, n * (n - 1) // 2)
    d_max = min(n - 1, math.sqrt(2 * m))
    u, v = chung_lu(n, m, 2.2, d_max, seed, substream=(11, g))
    w = zipf_weights(m, 2.0, 1_000_000, _rng(seed, 12, g))
    return Graph(n, u, v, w, name=f"batch[{g}] n={n} m={m}")


def batch_queries(count: int, seed: int = 3):
    """Per-graph query parameters of the batch: k uniform in [10, 1000], p
    uniform over {-inf, 1, 2, +inf}."""
    rng = _rng(seed, 13)
    ks = rng.integers(10, 1001, size=count).astype(np.int32)
    ps = np.array([-math.inf, 1.0, 2.0, math.inf])[rng.integers(0, 4, size=count)]
    return ps, ks


def random_small_graph(n: int, p_edge: float, wmax: int, seed) -> Graph:
    """Erdos-Renyi G(n, p) with uniform integer weights in [1, wmax] (for
    property tests on tiny graphs, where ties are frequent)."""
    rng = _rng(seed, 20)
    iu, ju = np.triu_indices(n, 1)
    keep = rng.random(iu.shape[0]) < p_edge
    u = iu[keep].astype(np.int32)
    v = ju[keep].astype(np.int32)
    perm = rng.permutation(u.shape[0])
    u, v = u[perm], v[perm]
    flip = rng.random(u.shape[0]) < 0.5
    u2 = np.where(flip, v, u).astype(np.int32)
    v2 = np.where(flip, u, v).astype(np.int32)
    w = rng.integers(1, wmax + 1, size=u.shape[0]).astype(np.int32)
    return Graph(n, u2, v2, w, name=f"gnp n={n} p={p_edge} w<={wmax}")


# ---------------------------------------------------------------------------
# Device-side generation for sizes numpy cannot draw in reasonable time (the
# billion-edge workload).  Same recipe as chung_lu/zipf_weights (erased
# Chung-Lu with the same expected-degree profile, truncated Zipf weights),
# drawn with torch's seeded CUDA generator; torch serves only to draw the
# inputs.  Everything stays on the device.
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class DeviceGraph:
    n: int
    m: int
    u: "object"         # int32 [m], shuffled edge order, random endpoint order
    v: "object"         # int32 [m]
    w: "object"         # int32 [m], w[i] is the weight of edge (u[i], v[i])
    keys: "object"      # int64 [m], min*n+max of every edge, ascending
    w_by_key: "object"  # int32 [m], weight of the edge keys[j]
    name: str = ""


def _expected_degrees_torch(n, m, gamma, d_max, device):
    import torch
    a = 1.0 / (gamma - 1.0)
    idx = torch.arange(n, dtype=torch.float64, device=device)
    target = 2.0 * m

    def total(i0):
        return float(torch.sum(d_max * i0 ** a * (idx + i0) ** (-a)).item())

    lo, hi = 1e-9, 1e12
    if total(hi) < target:
        return torch.full((n,), target / n, dtype=torch.float64, device=device)
    for _ in range(200):
        mid = math.sqrt(lo * hi)
        if total(mid) < target:
            lo = mid
        else:
            hi = mid
        if hi / lo < 1 + 1e-12:
            break
    return d_max * hi ** a * (idx + hi) ** (-a)


def chung_lu_device(n: int, m: int, gamma: float, d_max: float, seed: int, device="cuda"):
    """Erased Chung-Lu graph drawn on the device.  Returns (u, v, keys, order):
    u, v int32 in shuffled order, keys the ascending edge keys min*n+max, and
    order (int64) with key(u[i], v[i]) == keys[order[i]]."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed) * 1_000_003 + 17)
    theta = _expected_degrees_torch(n, m, gamma, d_max, device)
    cdf = torch.cumsum(theta, 0)
    cdf /= cdf[-1].clone()
    del theta
    keys = torch.empty(0, dtype=torch.int64, device=device)
    rounds = 0
    while keys.numel() < m:
        need = m - keys.numel()
        draw = int(need * 1.15) + 1024
        parts = [keys]
        for start in range(0, draw, 1 << 28):
            cnt = min(1 << 28, draw - start)
            a = torch.searchsorted(cdf, torch.rand(cnt, dtype=torch.float64, device=device,
                                                   generator=gen), right=True).clamp_(max=n - 1)
            b = torch.searchsorted(cdf, torch.rand(cnt, dtype=torch.float64, device=device,
                                                   generator=gen), right=True).clamp_(max=n - 1)
            ok = a != b
            a, b = a[ok], b[ok]
            parts.append(torch.minimum(a, b) * n + torch.maximum(a, b))
            del a, b, ok
        keys = torch.unique(torch.cat(parts))
        del parts
        rounds += 1
        if rounds > 100:
            raise RuntimeError("Chung-Lu top-up did not converge")
    if keys.numel() > m:
        pick = torch.randperm(keys.numel(), device=device, generator=gen)[:m]
        keys = keys[torch.sort(pick).values]
        del pick
    del cdf
    order = torch.randperm(m, device=device, generator=gen)
    shuffled = keys[order]
    a = (shuffled // n).to(torch.int32)
    b = (shuffled % n).to(torch.int32)
    del shuffled
    flip = torch.rand(m, device=device, generator=gen) < 0.5
    u = torch.where(flip, b, a)
    v = torch.where(flip, a, b)
    del flip, a, b
    return u, v, keys, order


def zipf_weights_device(m: int, s: float, cap: int, seed: int, device="cuda"):
    """m i.i.d. weights P(w) proportional to w^-s on 1..cap (int32, device)."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed) * 1_000_003 + 29)
    x = torch.arange(1, cap + 1, dtype=torch.float64, device=device)
    cdf = torch.cumsum(x ** (-s), 0)
    cdf /= cdf[-1].clone()
    out = torch.empty(m, dtype=torch.int32, device=device)
    for start in range(0, m, 1 << 28):
        cnt = min(1 << 28, m - start)
        w = torch.searchsorted(cdf, torch.rand(cnt, dtype=torch.float64, device=device,
                                               generator=gen), right=True) + 1
        out[start:start + cnt] = w.clamp_(max=cap).to(torch.int32)
    return out


def large_graph_device(seed: int = 2, n: int = 50_000_000, m: int = 1_000_000_000,
                       device="cuda", gamma: float = 2.0, lookup: bool = True) -> DeviceGraph:
    """The billion-edge workload: Chung-Lu n=5e7, m=1e9, exponent 2.0,
    d_max 5e4, Zipf(2) int32 weights capped at 1e6, drawn on the device
    (about 36 GB of device memory for the result).  Smaller n, m (and
    another exponent) give the same recipe at another size; lookup=False
    drops the sorted edge keys and weights kept for edge lookups."""
    import torch
    u, v, keys, order = chung_lu_device(n, m, gamma, 50_000.0, seed, device)
    w = zipf_weights_device(m, 2.0, 1_000_000, seed, device)
    if lookup:
        w_by_key = torch.empty_like(w)
        w_by_key[order] = w
    else:
        keys = w_by_key = None
    del order
    torch.cuda.empty_cache()
    return DeviceGraph(n, m, u, v, w, keys, w_by_key,
                       f"chung-lu n={n} m={m} gamma={gamma} dmax=5e4 zipf(2,1e6) seed={seed} (device)")


def serve_pool_device(device="cuda"):
    """The serving pool's graphs, one at a time (a generator, so that each
    can be built and dropped before the next is drawn): the billion-edge
    graph (seed 2) and two Chung-Lu graphs of 2e8 edges, n = 1e7, exponent
    2.1, d_max 5e4, Zipf(2) weights (seeds 5 and 6)."""
    yield large_graph_device(2, device=device, lookup=False)
    for seed in (5, 6):
        yield large_graph_device(seed, n=10_000_000, m=200_000_000, device=device, gamma=2.1,
                                 lookup=False)


# ---------------------------------------------------------------------------
# The 4,096-graph batch drawn on the device in one pass.  Graph g has the
# size batch_graph(g) gives (n from the same seeded stream, m = 10 n,
# exponent 2.2, d_max = min(n - 1, sqrt(2 m))) and the same recipe (erased
# Chung-Lu, truncated Zipf(2) weights capped at 1e6); all graphs' endpoint
# draws, deduplication, top-ups and subset choice run as a few device-wide
# sorts instead of 4,096 numpy calls.
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class DeviceBatch:
    ns: np.ndarray    # int64 [G] vertices of each graph
    ms: np.ndarray    # int64 [G] edges of each graph
    offs: np.ndarray  # int64 [G] first edge of graph g in u/v/w (a multiple of 4)
    u: "object"       # int32 device [sum of padded m], local vertex ids
    v: "object"
    w: "object"
    name: str = ""

    @property
    def count(self) -> int:
        return int(self.ns.shape[0])

    def graph(self, g: int):
        """(n, u, v, w) of graph g: contiguous device slices, 16-byte aligned."""
        a, b = int(self.offs[g]), int(self.offs[g] + self.ms[g])
        return int(self.ns[g]), self.u[a:b], self.v[a:b], self.w[a:b]


def batch_sizes(count: int, seed: int = 3, n_hi: int = 200_000):
    """(n, m) of graphs 0..count-1 of the batch, as batch_graph draws them."""
    ns = np.empty(count, np.int64)
    for g in range(count):
        rng = _rng(seed, 10, g)
        ns[g] = int(round(math.exp(rng.uniform(math.log(100), math.log(n_hi)))))
    ms = np.minimum(10 * ns, ns * (ns - 1) // 2)
    return ns, ms


_PAIR_BITS = 36  # n <= 2e5 per graph, so min * n + max < 2**36


def batch_graphs_device(count: int = 4096, seed: int = 3, n_hi: int = 200_000,
                        device="cuda") -> DeviceBatch:
    """The batch workload drawn on the device: ``count`` Chung-Lu graphs,
    n log-uniform in [100, n_hi], m = 10 n, exponent 2.2, d_max = min(n - 1,
    sqrt(2 m)), Zipf(2) int32 weights capped at 1e6."""
    import torch
    ns, ms = batch_sizes(count, seed, n_hi)
    if int(ns.max()) ** 2 >= 2 ** _PAIR_BITS:
        raise ValueError("graph too large for the batch key packing")
    G = count
    gamma = 2.2
    a_exp = 1.0 / (gamma - 1.0)
    dmax = np.minimum(ns - 1, np.sqrt(2.0 * ms))
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed) * 1_000_003 + 41)

    # expected degrees of every graph, i0 solved by a vectorised bisection
    N = int(ns.sum())
    ns_t = torch.as_tensor(ns, device=device)
    vstart = torch.as_tensor(np.concatenate([[0], np.cumsum(ns)[:-1]]), device=device)
    gid = torch.repeat_interleave(torch.arange(G, device=device), ns_t)
    idx = torch.arange(N, dtype=torch.float64, device=device) - vstart[gid].double()
    dm = torch.as_tensor(dmax, dtype=torch.float64, device=device)
    target = torch.as_tensor(2.0 * ms, dtype=torch.float64, device=device)

    def theta_of(i0):
        i0v = i0[gid]
        return dm[gid] * i0v ** a_exp * (idx + i0v) ** (-a_exp)

    def total(i0):
        return torch.zeros(G, dtype=torch.float64, device=device).index_add_(0, gid, theta_of(i0))

    lo = torch.full((G,), 1e-9, dtype=torch.float64, device=device)
    hi = torch.full((G,), 1e12, dtype=torch.float64, device=device)
    flat = total(hi) < target
    for _ in range(64):
        mid = torch.sqrt(lo * hi)
        below = total(mid) < target
        lo = torch.where(below, mid, lo)
        hi = torch.where(below, hi, mid)
    theta = theta_of(hi)
    theta = torch.where(flat[gid], (target / ns_t.double())[gid], theta)
    del lo, hi, idx
    # per-graph cdf, offset by the graph index: draws for graph g are g + U
    cum = torch.cumsum(theta, 0)
    del theta
    seg_end = torch.as_tensor(np.cumsum(ns) - 1, device=device)
    before = torch.where(vstart > 0, cum[(vstart - 1).clamp(min=0)], torch.zeros_like(cum[:G]))
    tot = cum[seg_end] - before
    cdf = (cum - before[gid]) / tot[gid]
    cdf[seg_end] = 1.0
    cdf += gid.double()
    del cum, before, tot
    vend = vstart + ns_t

    ms_t = torch.as_tensor(ms, device=device)
    keys = torch.empty(0, dtype=torch.int64, device=device)
    have = torch.zeros(G, dtype=torch.int64, device=device)
    CH = 1 << 27
    for _round in range(100):
        need = (ms_t - have).clamp(min=0)
        if int(need.sum().item()) == 0:
            break
        draws = torch.where(need > 0, (need.double() * 1.15).long() + 64, torch.zeros_like(need)).cpu().numpy()
        parts = [keys]
        cdraw = np.cumsum(draws)
        g0 = 0
        while g0 < G:
            base = cdraw[g0 - 1] if g0 else 0
            g1 = int(np.searchsorted(cdraw, base + CH, side="right"))
            g1 = max(g1, g0 + 1)
            cnt_g = torch.as_tensor(draws[g0:g1], device=device)
            gs = torch.repeat_interleave(torch.arange(g0, g1, device=device), cnt_g)
            if gs.numel():
                x, y = [torch.searchsorted(cdf, gs.double() + torch.rand(gs.numel(), dtype=torch.float64,
                                                                        device=device, generator=gen),
                                           right=True) for _ in range(2)]
                last = vend[gs] - 1
                x = torch.minimum(x, last) - vstart[gs]
                y = torch.minimum(y, last) - vstart[gs]
                ok = x != y
                gs, x, y = gs[ok], x[ok], y[ok]
                parts.append((gs << _PAIR_BITS) + torch.minimum(x, y) * ns_t[gs] + torch.maximum(x, y))
                del x, y, ok, last
            del gs
            g0 = g1
        keys = torch.unique(torch.cat(parts))
        del parts
        have = torch.bincount(keys >> _PAIR_BITS, minlength=G)
    else:
        raise RuntimeError("batch Chung-Lu top-up did not converge")
    del cdf, gid, vstart, vend

    # exactly m of each graph's distinct pairs, uniformly, in random order:
    # sort by (graph, random priority) and keep each graph's first m
    gk = keys >> _PAIR_BITS
    prio = gk.double() + torch.rand(keys.numel(), dtype=torch.float64, device=device, generator=gen)
    order = torch.sort(prio, stable=True).indices
    del prio
    keys = keys[order]
    gk = gk[order]
    del order
    cstart = torch.cumsum(have, 0) - have
    rank = torch.arange(keys.numel(), device=device) - cstart[gk]
    keep = rank < ms_t[gk]
    keys, gk = keys[keep], gk[keep]
    del rank, keep

    # pad every graph to a multiple of 4 edges so slices stay 16-byte aligned
    pad = (ms + 3) // 4 * 4
    offs = np.concatenate([[0], np.cumsum(pad)[:-1]]).astype(np.int64)
    estart = torch.as_tensor(np.concatenate([[0], np.cumsum(ms)[:-1]]), device=device)
    dest = torch.as_tensor(offs, device=device)[gk] + (torch.arange(keys.numel(), device=device) - estart[gk])
    pair = keys & ((1 << _PAIR_BITS) - 1)
    ng = ns_t[gk]
    lo_, hi_ = (pair // ng).to(torch.int32), (pair % ng).to(torch.int32)
    del pair, ng, keys, gk
    flip = torch.rand(lo_.numel(), device=device, generator=gen) < 0.5
    total_pad = int(pad.sum())
    u = torch.zeros(total_pad, dtype=torch.int32, device=device)
    v = torch.zeros(total_pad, dtype=torch.int32, device=device)
    u[dest] = torch.where(flip, hi_, lo_)
    v[dest] = torch.where(flip, lo_, hi_)
    del flip, lo_, hi_
    w = torch.ones(total_pad, dtype=torch.int32, device=device)
    w[dest] = zipf_weights_device(int(ms.sum()), 2.0, 1_000_000, seed + 7919, device)
    del dest
    torch.cuda.empty_cache()
    return DeviceBatch(ns, ms, offs, u, v, w,
                       f"{count} chung-lu graphs, n log-uniform [100, {n_hi}], m=10n, gamma=2.2, "
                       f"zipf(2,1e6), seed={seed} (device)")
