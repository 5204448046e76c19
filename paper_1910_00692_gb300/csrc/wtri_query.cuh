// Shared device machinery of the top-k query, the edge sampler and the
// batched form (included by wtri_topk.cu and wtri_batch.cu).
//
// Exact top-k weighted triangles: heavy-first enumeration with a running
// threshold.
//
// Method (the exactness argument of Algorithm 2 and Section 3.2, re-derived
// for a parallel schedule):
//  * Edges are visited in the edge order (weight desc, input index asc); r is
//    an edge's position.  Each triangle is owned by its first edge in that
//    order, so edge r owns triangle {x, y, c} iff both (x,c) and (y,c) come
//    after r.  Every triangle is enumerated exactly once.
//  * Every triangle owned by r has all edge weights <= w_r, and m_p is
//    monotone in each argument with m_p <= max, so its key is at most
//    K(w_r, w_r, w_r).  Once that bound is below the threshold tau, no later
//    edge can contribute: the sweep stops.  This is the paper's heavy-first
//    threshold argument with one monotone cursor in place of two pointers.
//  * Per edge, the entries of x and y after r are suffixes of their
//    weight-sorted lists; their first entries bound the other two weights
//    (edge bound), and scanning x's suffix in weight order gives a wedge bound
//    K(w_r, w_xc, max_y) that only decreases, so the scan stops at the first
//    wedge below tau.  The closing edge (y, c) is found by binary search in
//    the oriented (degree-ordered) lists.
//  * tau is the key of the k-th best of k distinct triangles found so far, a
//    valid lower bound on the true k-th key; pruning is strict (< tau), so
//    triangles tied with the k-th key are still enumerated and the triple
//    tie-break decides them.
//
// Schedule: the edge order is processed in rounds of geometrically growing
// ranges [lo, hi).  Each round is three launches: k_round (thread per edge,
// short scans inline, long scans deferred), k_long (block per deferred scan,
// the closing-edge lookups go to the y row staged in shared memory by a bulk
// copy), and k_select (one block: radix select of the k-th candidate under
// the total order, in-place compaction, new tau).  Rounds after the stop
// return at once, so the launch sequence depends only on (m, k) and can be
// captured in a CUDA graph.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "wtri_internal.cuh"

namespace wtri {
namespace {

constexpr int RBLK = 256;          // k_round block
constexpr int LBLK = 256;          // k_long block
constexpr int SBLK = 1024;         // k_select block
constexpr int STAGE_MAX = 24576;   // ids of a y row staged in shared memory (96 KB)
constexpr int64_t FIRST_ROUND = 64;  // batch schedule (single queries use the graph's tune)
constexpr int ROUND_GROWTH = 8;
constexpr uint32_t WAIT_LIMIT = 1u << 24;  // bounded mbarrier polling
constexpr uint32_t STOP_NONE = 0x7fffffffu; // edge positions are below 2^31

struct QState {
    unsigned long long tau;   // keys below tau are pruned; 0 = no bound yet
    uint32_t stop_rev;        // STOP_NONE - (first edge whose bound fell below tau); 0 = none
    uint32_t err;             // DEV_ERR_* bits
    uint32_t count;           // candidates appended (may exceed capacity)
    uint32_t long_count;      // deferred scans
    uint32_t selected;        // count right after the last compaction
    uint32_t pad[3];
};

struct LongItem {
    int32_t r;      // owning edge (position in the edge order)
    int32_t x, y;   // scanned endpoint, probed endpoint
    int32_t w;      // w_r
    int32_t ymax;   // first weight of y's suffix
    int32_t pad;    // query index within a batch
    int64_t j0, j1; // remaining suffix of x's weight-sorted list
};

struct Query {
    QState* st;
    unsigned long long* ckey;
    int4* ctri;
    uint32_t cap;
    LongItem* longs;
    uint32_t long_cap;
    int32_t k;
    // Sampled mode (edge sampling): bitmap of drawn edges by edge-order
    // position, and the drawn positions in ascending order.
    const uint32_t* smark;
    const int32_t* slist;
    // Deferred-scan list counter (the query's own, or one shared by a batch)
    // and the query's index in a batch (stored in deferred items).
    uint32_t* long_count;
    int32_t qid;
    // Sharding (multi-GPU split of one query): this query owns the edges
    // whose chunk (position >> SHARD_SHIFT) is congruent to shard modulo
    // nshards; nshards <= 1 means every edge.
    int32_t shard;
    int32_t nshards;
    // Wedges an edge's thread scans before deferring the rest to a block (the
    // boundary between the short-list and long-list strategies).
    int32_t t_short;
    // Instrumented run: bytes of the adjacency loads are added here (null:
    // no counting).
    unsigned long long* qbytes;
    // The value of p for P_GEN queries.
    double gp;
    // Weights are positive fp32 bit patterns (a float-weight graph), not
    // integers: the means and reported values read them as floats.
    int32_t fw;
    // Polls of the first wait for a staged row (WAIT_LIMIT in production;
    // tests lower it to take the timeout path).
    uint32_t wait_first;
};

// Bytes of adjacency loads issued by one thread (instrumented runs only).
struct Tally {
    unsigned long long n = 0;
    bool on = false;
    __device__ __forceinline__ void add(uint32_t b) {
        if (on) n += b;
    }
};

// Adds every lane's tally to the query's counter (one atomic per warp).
__device__ __forceinline__ void flush_tally(const Query& q, const Tally& t) {
    if (!q.qbytes) return;
    unsigned long long v = t.n;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(q.qbytes, v);
}

constexpr int SHARD_SHIFT = 10;  // 1024-edge chunks of the edge order, dealt round-robin

__device__ __forceinline__ bool drawn(const Query& q, int32_t r) {
    return (__ldg(q.smark + (r >> 5)) >> (r & 31)) & 1u;
}

// Ownership.  Exact mode: a triangle belongs to its first edge in the edge
// order, so the edge at position r owns (x, y, c) iff both other edges come
// later.  Sampled mode (Algorithm 3's set T): a triangle belongs to its
// first DRAWN edge, so each triangle with a drawn edge is reported once.
template <bool SAMPLED>
__device__ __forceinline__ bool owns(const Query& q, int32_t r, int32_t rxc, int32_t ryc) {
    if (!SAMPLED) return rxc > r && ryc > r;
    return !(rxc < r && drawn(q, rxc)) && !(ryc < r && drawn(q, ryc));
}

// m_p of Eq. 1 in fp64 for a finite p outside {0, 1, 2}: the weights in
// ascending order (equal multisets give equal bits), scaled by the largest
// (p > 0) or the smallest (p < 0) so that no power overflows:
//   m_p = s * (((a/s)^p + (b/s)^p + (c/s)^p) / 3)^(1/p).
__device__ __forceinline__ double general_mean(double p, uint32_t a, uint32_t b, uint32_t c, bool fw = false) {
    uint32_t t;
    if (a > b) { t = a; a = b; b = t; }
    if (b > c) { t = b; b = c; c = t; }
    if (a > b) { t = a; a = b; b = t; }
    // positive fp32 bit patterns order like their values, so the sort holds
    const double x = fw ? (double)__uint_as_float(a) : (double)a;
    const double y = fw ? (double)__uint_as_float(b) : (double)b;
    const double z = fw ? (double)__uint_as_float(c) : (double)c;
    if (p == 0.0) return cbrt(x * y * z);  // the geometric mean (real weights only)
    const double s = p > 0 ? z : x;
    const double m = (pow(x / s, p) + pow(y / s, p) + pow(z / s, p)) / 3.0;
    return s * pow(m, 1.0 / p);
}

// Ranking key of a triangle with edge weights a, b, c: exact integers for
// p in {-inf, 0, 1, 2, +inf}; the mean's fp64 bit pattern for P_GEN.
template <int P>
__device__ __forceinline__ unsigned long long keyof(uint32_t a, uint32_t b, uint32_t c,
                                                    double gp = 0.0, bool fw = false) {
    if (P == P_ONE) return (unsigned long long)a + b + c;
    if (P == P_TWO)
        return (unsigned long long)a * a + (unsigned long long)b * b + (unsigned long long)c * c;
    if (P == P_MAX) return (unsigned long long)max(a, max(b, c));
    if (P == P_GEO) return (unsigned long long)a * b * c;  // weights < 2^21: below 2^63
    if (P == P_GEN) return (unsigned long long)__double_as_longlong(general_mean(gp, a, b, c, fw));
    return (unsigned long long)min(a, min(b, c));
}

// Upper bound used for pruning: the key itself for the exact keys; for
// P_GEN the mean raised by a relative 1e-12, far above fp64 rounding, so
// that a bound computed for larger weights is never below a key computed
// for smaller ones.
template <int P>
__device__ __forceinline__ unsigned long long boundof(uint32_t a, uint32_t b, uint32_t c,
                                                      double gp = 0.0, bool fw = false) {
    if (P == P_GEN)
        return (unsigned long long)__double_as_longlong(general_mean(gp, a, b, c, fw) * (1.0 + 1e-12));
    return keyof<P>(a, b, c);
}

__device__ __forceinline__ void sort3(int32_t& a, int32_t& b, int32_t& c) {
    int32_t t;
    if (a > b) { t = a; a = b; b = t; }
    if (b > c) { t = b; b = c; c = t; }
    if (a > b) { t = a; a = b; b = t; }
}

__device__ __forceinline__ unsigned long long ld_volatile_u64(const unsigned long long* p) {
    return *(volatile const unsigned long long*)p;
}

// Position just after edge r's own entry in x's weight-sorted list
// [lo, hi) (x's row).
__device__ __forceinline__ int64_t suffix_start(const DevGraph& G, int64_t lo, int64_t hi, int32_t r,
                                                uint32_t* err, Tally& tb) {
    const int64_t end = hi;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        tb.add(4);
        if (__ldg(G.wrk + mid) < r) lo = mid + 1;
        else hi = mid;
    }
    tb.add(4);
    if (lo >= end || __ldg(G.wrk + lo) != r) {
        atomicOr(err, DEV_ERR_INTERNAL);
        return end;
    }
    return lo + 1;
}

// Closing edge (y, c) in the oriented lists: stored once, at the endpoint of
// lower (degree, id) rank, rows ascending by id (row s at
// [orowptr[s], orowptr[s+1])).  y_owns: whether y is that endpoint.
__device__ __forceinline__ bool y_owns(const DevGraph& G, int32_t y, int64_t dy, int32_t c, Tally& tb) {
    const int64_t dc = __ldg(G.rowptr + c + 1) - __ldg(G.rowptr + c);
    tb.add(16);
    return dy < dc || (dy == dc && y < c);
}

// Searches oriented row s for t.
__device__ __forceinline__ bool search_oriented(const DevGraph& G, int32_t s, int32_t t, int32_t& wst,
                                                int32_t& rst, Tally& tb) {
    int64_t lo = __ldg(G.orowptr + s), hi = __ldg(G.orowptr + s + 1);
    const int64_t end = hi;
    tb.add(16);
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        tb.add(4);
        if (__ldg(G.ocol + mid) < t) lo = mid + 1;
        else hi = mid;
    }
    if (lo < end) tb.add(4);
    if (lo < end && __ldg(G.ocol + lo) == t) {
        wst = __ldg(G.owt + lo);
        rst = __ldg(G.ork + lo);
        tb.add(8);
        return true;
    }
    return false;
}

__device__ __forceinline__ bool probe_oriented(const DevGraph& G, int32_t y, int64_t dy, int32_t c,
                                               int32_t& wyc, int32_t& ryc, Tally& tb) {
    return y_owns(G, y, dy, c, tb) ? search_oriented(G, y, c, wyc, ryc, tb)
                                   : search_oriented(G, c, y, wyc, ryc, tb);
}

// Warp-aggregated append: the active lanes appending to the same query
// (a batched launch mixes queries within a warp) take one atomic together.
__device__ __forceinline__ void append(const Query& q, unsigned long long key, int32_t a, int32_t b,
                                       int32_t c) {
    const uint32_t active = __activemask();
    const uint32_t peers = __match_any_sync(active, (unsigned long long)(uintptr_t)q.st);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(peers) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(&q.st->count, (uint32_t)__popc(peers));
    base = __shfl_sync(peers, base, leader);
    const uint32_t idx = base + __popc(peers & ((1u << lane) - 1u));
    if (idx < q.cap) {
        q.ckey[idx] = key;
        q.ctri[idx] = make_int4(a, b, c, 0);
    } else {
        atomicOr(&q.st->err, DEV_ERR_OVERFLOW);
    }
}

// ---------------------------------------------------------------------------
// Round: threads stride over the edges of [lo, hi).
// ---------------------------------------------------------------------------
template <int P, bool SAMPLED>
__device__ __forceinline__ void scan_wedges(const DevGraph& G, const Query& q,
                                            unsigned long long tau, int32_t r, uint32_t w,
                                            int32_t x, int32_t y, int64_t dy, uint32_t ymax,
                                            int64_t& j, int64_t jstop, bool& done, Tally& tb) {
    for (; j < jstop; j++) {
        const uint32_t wxc = (uint32_t)__ldg(G.wwt + j);
        tb.add(4);
        if (boundof<P>(w, wxc, ymax, q.gp, q.fw != 0) < tau) {  // wedge bound, non-increasing along the list
            done = true;
            return;
        }
        const int32_t c = __ldg(G.wcol + j);
        tb.add(4);
        if (SAMPLED && c == y) continue;  // the edge itself (full rows in sampled mode)
        int32_t wyc, ryc;
        if (probe_oriented(G, y, dy, c, wyc, ryc, tb) &&
            (tb.add(4), owns<SAMPLED>(q, r, __ldg(G.wrk + j), ryc))) {
            const unsigned long long key = keyof<P>(w, wxc, (uint32_t)wyc, q.gp, q.fw != 0);
            if (key >= tau) {
                int32_t a = x, b = y, cc = c;
                sort3(a, b, cc);
                append(q, key, a, b, cc);
            }
        }
    }
}

// Returns false once this edge's bound is below tau (and so is every later
// edge's).
template <int P, bool SAMPLED>
__device__ __forceinline__ bool process_edge(const DevGraph& G, const Query& q,
                                             unsigned long long tau, int32_t idx, Tally& tb) {
    const int32_t r = SAMPLED ? __ldg(q.slist + idx) : idx;
    const uint32_t w = (uint32_t)__ldg(G.ord_w + r);
    tb.add(4);
    if (!SAMPLED && boundof<P>(w, w, w, q.gp, q.fw != 0) < tau) {
        // every later edge has a bound no larger: record the first such edge
        atomicMax(&q.st->stop_rev, STOP_NONE - (uint32_t)r);
        return false;
    }
    if (!SAMPLED && q.nshards > 1 &&
        (int32_t)(((uint32_t)r >> SHARD_SHIFT) % (uint32_t)q.nshards) != q.shard)
        return true;  // owned by another shard
    const int32_t u = __ldg(G.ord_u + r), v = __ldg(G.ord_v + r);
    const int64_t bu = __ldg(G.rowptr + u), eu = __ldg(G.rowptr + u + 1);
    const int64_t bv = __ldg(G.rowptr + v), ev = __ldg(G.rowptr + v + 1);
    tb.add(40);
    // Exact mode scans what comes after r in each list; sampled mode scans
    // whole lists (the other two edges may be heavier than a drawn edge).
    const int64_t su = SAMPLED ? bu : suffix_start(G, bu, eu, r, &q.st->err, tb);
    const int64_t sv = SAMPLED ? bv : suffix_start(G, bv, ev, r, &q.st->err, tb);
    if (su >= eu || sv >= ev) return true;  // no edge after r on one side: owns nothing
    const uint32_t umax = (uint32_t)__ldg(G.wwt + su), vmax = (uint32_t)__ldg(G.wwt + sv);
    tb.add(8);
    if (boundof<P>(w, umax, vmax, q.gp, q.fw != 0) < tau) return true;  // edge bound
    // Scan the shorter suffix; probe the other endpoint.
    const bool xu = (eu - su) <= (ev - sv);
    const int32_t x = xu ? u : v, y = xu ? v : u;
    const int64_t sx = xu ? su : sv, ex = xu ? eu : ev;
    const uint32_t ymax = xu ? vmax : umax;
    const int64_t dy = xu ? ev - bv : eu - bu;
    int64_t j = sx;
    bool done = false;
    scan_wedges<P, SAMPLED>(G, q, tau, r, w, x, y, dy, ymax, j, min(ex, sx + (int64_t)q.t_short),
                            done, tb);
    if (!done && j < ex) {
        const uint32_t slot = atomicAdd(q.long_count, 1u);
        if (slot < q.long_cap) {
            LongItem it;
            it.r = r;
            it.x = x;
            it.y = y;
            it.w = (int32_t)w;
            it.ymax = (int32_t)ymax;
            it.pad = q.qid;
            it.j0 = j;
            it.j1 = ex;
            q.longs[slot] = it;
        } else {
            // Deferred list full: finish the scan here.
            scan_wedges<P, SAMPLED>(G, q, tau, r, w, x, y, dy, ymax, j, ex, done, tb);
        }
    }
    return true;
}

template <int P, bool SAMPLED = false>
__global__ void __launch_bounds__(RBLK) k_round(DevGraph G, Query q, int64_t lo, int64_t hi) {
    // Blocks run in any order, so an edge is skipped only once an edge at or
    // before it has failed its bound (all later edges have no larger bound).
    const volatile uint32_t* stop_rev = &q.st->stop_rev;
    if (lo >= (int64_t)(STOP_NONE - *stop_rev)) return;
    if (*(volatile const uint32_t*)&q.st->err) return;  // the query has already failed
    const unsigned long long tau = ld_volatile_u64(&q.st->tau);
    const int64_t stride = (int64_t)gridDim.x * RBLK;
    Tally tb;
    tb.on = q.qbytes != nullptr;
    for (int64_t r64 = lo + (int64_t)blockIdx.x * RBLK + threadIdx.x; r64 < hi; r64 += stride) {
        if (r64 >= (int64_t)(STOP_NONE - *stop_rev)) break;
        if (!process_edge<P, SAMPLED>(G, q, tau, (int32_t)r64, tb)) break;
    }
    flush_tally(q, tb);
}

// Grid of a round: a few resident blocks per SM, striding over the range.
inline unsigned round_grid(int64_t edges) {
    const int64_t cap = (int64_t)sm_count() * 8;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(cap, (edges + RBLK - 1) / RBLK));
}

// ---------------------------------------------------------------------------
// Round at p = -inf by NodeIterator++ over the degree order (Section 5.2):
// one warp per edge r = {a, b}, a the endpoint of lower (degree, id) rank.
// A triangle a < b < c in that order is found exactly once, from its edge
// {a, b}, as c in N+(a) ∩ N+(b) (the oriented rows): the shorter row is
// scanned and each c binary-searched in the other.  Its key min(w_ab, w_ac,
// w_bc) is at most w_r, so the heavy-first stop of the sweep holds: once
// w_r < tau no later edge can close a triangle that enters the top-k, and
// entries lighter than tau are skipped before the search.  Every edge of a
// qualifying triangle is at least tau, which is why this replaces the
// weight-sorted scan (whose wedge bound prunes little at p = -inf) for the
// unsampled, unsharded query.
// ---------------------------------------------------------------------------
constexpr int MIN_WARPS = RBLK / 32;
#ifndef WTRI_MIN_STAGE
#define WTRI_MIN_STAGE 512
#endif
// Longest searched row staged in shared memory (per warp; 0: never staged).
constexpr int MIN_STAGE = WTRI_MIN_STAGE;

__global__ void __launch_bounds__(RBLK) k_round_min(DevGraph G, Query q, int64_t lo, int64_t hi) {
    const volatile uint32_t* stop_rev = &q.st->stop_rev;
    if (lo >= (int64_t)(STOP_NONE - *stop_rev)) return;
    if (*(volatile const uint32_t*)&q.st->err) return;  // the query has already failed
    const unsigned long long tau = ld_volatile_u64(&q.st->tau);
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * MIN_WARPS;
    __shared__ int32_t stage_all[MIN_WARPS][MIN_STAGE > 0 ? MIN_STAGE : 1];
    int32_t* srow = stage_all[threadIdx.x >> 5];
    Tally tb;
    tb.on = q.qbytes != nullptr;
    // The warp's next edge is fetched while this one is scanned: its weight
    // and endpoints at the top of the iteration, its degrees once this
    // edge's oriented-row bounds are issued.
    int64_t r = lo + (int64_t)blockIdx.x * MIN_WARPS + (threadIdx.x >> 5);
    uint32_t w_nx = 0;
    int32_t u_nx = 0, v_nx = 0;
    int64_t du_nx = 0, dv_nx = 0;
    if (r < hi) {
        w_nx = (uint32_t)__ldg(G.ord_w + r);
        u_nx = __ldg(G.ord_u + r);
        v_nx = __ldg(G.ord_v + r);
        du_nx = __ldg(G.rowptr + u_nx + 1) - __ldg(G.rowptr + u_nx);
        dv_nx = __ldg(G.rowptr + v_nx + 1) - __ldg(G.rowptr + v_nx);
    }
    for (; r < hi; r += nwarps) {
        const uint32_t w = w_nx;
        const int32_t u = u_nx, v = v_nx;
        const int64_t du = du_nx, dv = dv_nx;
        const int64_t rn = r + nwarps;
        const bool more = rn < hi;
        if (more) {
            w_nx = (uint32_t)__ldg(G.ord_w + rn);
            u_nx = __ldg(G.ord_u + rn);
            v_nx = __ldg(G.ord_v + rn);
        }
        if (r >= (int64_t)(STOP_NONE - *stop_rev)) break;
        if (w < tau) {
            // every later edge is lighter: record the first such edge
            if (lane == 0) atomicMax(&q.st->stop_rev, STOP_NONE - (uint32_t)r);
            break;
        }
        const bool ua = du < dv || (du == dv && u < v);
        const int32_t a = ua ? u : v, b = ua ? v : u;
        const int64_t ab = __ldg(G.orowptr + a), ae = __ldg(G.orowptr + a + 1);
        const int64_t bb = __ldg(G.orowptr + b), be = __ldg(G.orowptr + b + 1);
        if (more) {
            du_nx = __ldg(G.rowptr + u_nx + 1) - __ldg(G.rowptr + u_nx);
            dv_nx = __ldg(G.rowptr + v_nx + 1) - __ldg(G.rowptr + v_nx);
        }
        if (lane == 0) tb.add(12 + 32 + 32);
        const bool as = (ae - ab) <= (be - bb);
        const int64_t sb = as ? ab : bb, se = as ? ae : be;  // scanned row
        const int64_t lb = as ? bb : ab, le = as ? be : ae;  // searched row
        // The searched row goes to shared memory (coalesced, once per edge)
        // as soon as a chunk of the scanned row holds an entry >= tau: one
        // latency step instead of a global binary search per entry.
        const int64_t llen = le - lb;
        bool staged = false;
        for (int64_t base = sb; base < se; base += 32) {
            const int64_t j = base + lane;
            const uint32_t wsc = j < se ? (uint32_t)__ldg(G.owt + j) : 0u;
            if (j < se) tb.add(4);
            const bool heavy = j < se && wsc >= tau;
            if (__ballot_sync(0xffffffffu, heavy) == 0) continue;
            if (!staged && llen <= MIN_STAGE) {
                for (int t = lane; t < llen; t += 32) srow[t] = __ldg(G.ocol + lb + t);
                tb.add((uint32_t)(lane < llen ? 4 * ((llen - lane + 31) / 32) : 0));
                __syncwarp();
                staged = true;
            }
            if (!heavy) continue;
            const int32_t c = __ldg(G.ocol + j);
            tb.add(4);
            int64_t l0, found_at = -1;
            if (staged) {
                int s0 = 0, s1 = (int)llen;
                while (s0 < s1) {
                    const int mid = (s0 + s1) >> 1;
                    if (srow[mid] < c) s0 = mid + 1;
                    else s1 = mid;
                }
                if (s0 < llen && srow[s0] == c) found_at = lb + s0;
            } else {
                int64_t l1 = le;
                l0 = lb;
                while (l0 < l1) {
                    const int64_t mid = (l0 + l1) >> 1;
                    tb.add(4);
                    if (__ldg(G.ocol + mid) < c) l0 = mid + 1;
                    else l1 = mid;
                }
                if (l0 < le && (tb.add(4), __ldg(G.ocol + l0) == c)) found_at = l0;
            }
            if (found_at >= 0) {
                const uint32_t wlc = (uint32_t)__ldg(G.owt + found_at);
                tb.add(4);
                const unsigned long long key = keyof<P_MIN>(w, wsc, wlc);
                if (key >= tau) {
                    int32_t x = a, y = b, z = c;
                    sort3(x, y, z);
                    append(q, key, x, y, z);
                }
            }
        }
        __syncwarp();  // the staged row is reused by the warp's next edge
    }
    flush_tally(q, tb);
}

inline unsigned round_grid_warps(int64_t edges) {
    const int64_t cap = (int64_t)sm_count() * 8;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(cap, (edges + MIN_WARPS - 1) / MIN_WARPS));
}

// ---------------------------------------------------------------------------
// Round with one warp per edge, for the small early rounds (up to
// WTRI_WARP_ROUND_MAX edges), where a thread per edge leaves the GPU almost
// idle and each thread scans its entries one dependent search after another.
// Same sweep as k_round: the edge checks and the two suffix searches once
// per warp (lanes 0 and 1 search u's and v's lists at once), then the first
// t_short entries (rounded up to a multiple of 32) of the shorter suffix,
// one entry and one probe per lane; the rest is deferred to k_long.  The
// wedge bound does not increase along a list, so the lanes that pass it are
// exactly the entries a serial scan would reach.
// ---------------------------------------------------------------------------
#ifndef WTRI_WARP_ROUND_MAX
#define WTRI_WARP_ROUND_MAX 4096
#endif
constexpr int64_t WARP_ROUND_MAX = WTRI_WARP_ROUND_MAX;

// Scans [jb, je) of x's list, 32 entries per step; true once an entry fails
// the wedge bound (and so does every later one).  Warp-uniform result.
template <int P>
__device__ __forceinline__ bool scan_wedges_warp(const DevGraph& G, const Query& q, unsigned long long tau,
                                                 int32_t r, uint32_t w, int32_t x, int32_t y, int64_t dy,
                                                 uint32_t ymax, int64_t jb, int64_t je, Tally& tb) {
    const int lane = threadIdx.x & 31;
    for (int64_t base = jb; base < je; base += 32) {
        const int64_t j = base + lane;
        const bool live = j < je;
        uint32_t wxc = 0;
        if (live) {
            wxc = (uint32_t)__ldg(G.wwt + j);
            tb.add(4);
        }
        const bool fail = live && boundof<P>(w, wxc, ymax, q.gp, q.fw != 0) < tau;
        const bool stop = __any_sync(0xffffffffu, fail);
        if (live && !fail) {
            const int32_t c = __ldg(G.wcol + j);
            tb.add(4);
            int32_t wyc, ryc;
            if (probe_oriented(G, y, dy, c, wyc, ryc, tb) &&
                (tb.add(4), owns<false>(q, r, __ldg(G.wrk + j), ryc))) {
                const unsigned long long key = keyof<P>(w, wxc, (uint32_t)wyc, q.gp, q.fw != 0);
                if (key >= tau) {
                    int32_t a = x, b = y, cc = c;
                    sort3(a, b, cc);
                    append(q, key, a, b, cc);
                }
            }
        }
        if (stop) return true;
    }
    return false;
}

// process_edge with the warp: false once the edge's bound is below tau.
// tu counts the warp's shared loads once (lane 0).
template <int P>
__device__ __forceinline__ bool process_edge_warp(const DevGraph& G, const Query& q, unsigned long long tau,
                                                  int32_t r, Tally& tb, Tally& tu) {
    const int lane = threadIdx.x & 31;
    const uint32_t w = (uint32_t)__ldg(G.ord_w + r);
    tu.add(4);
    if (boundof<P>(w, w, w, q.gp, q.fw != 0) < tau) {
        if (lane == 0) atomicMax(&q.st->stop_rev, STOP_NONE - (uint32_t)r);
        return false;
    }
    if (q.nshards > 1 && (int32_t)(((uint32_t)r >> SHARD_SHIFT) % (uint32_t)q.nshards) != q.shard)
        return true;  // owned by another shard
    const int32_t u = __ldg(G.ord_u + r), v = __ldg(G.ord_v + r);
    const int64_t bu = __ldg(G.rowptr + u), eu = __ldg(G.rowptr + u + 1);
    const int64_t bv = __ldg(G.rowptr + v), ev = __ldg(G.rowptr + v + 1);
    tu.add(40);
    Tally ts;  // lanes 0 and 1 count their own search; the others repeat lane 0's
    ts.on = tb.on && lane < 2;
    const bool side_v = lane == 1;
    const int64_t s1 = suffix_start(G, side_v ? bv : bu, side_v ? ev : eu, r, &q.st->err, ts);
    tb.n += ts.n;
    const int64_t su = __shfl_sync(0xffffffffu, s1, 0), sv = __shfl_sync(0xffffffffu, s1, 1);
    if (su >= eu || sv >= ev) return true;  // no edge after r on one side: owns nothing
    const uint32_t umax = (uint32_t)__ldg(G.wwt + su), vmax = (uint32_t)__ldg(G.wwt + sv);
    tu.add(8);
    if (boundof<P>(w, umax, vmax, q.gp, q.fw != 0) < tau) return true;  // edge bound
    const bool xu = (eu - su) <= (ev - sv);
    const int32_t x = xu ? u : v, y = xu ? v : u;
    const int64_t sx = xu ? su : sv, ex = xu ? eu : ev;
    const uint32_t ymax = xu ? vmax : umax;
    const int64_t dy = xu ? ev - bv : eu - bu;
    const int64_t budget = q.t_short > 32 ? ((int64_t)q.t_short + 31) / 32 * 32 : 32;
    const int64_t jlim = ex < sx + budget ? ex : sx + budget;
    if (scan_wedges_warp<P>(G, q, tau, r, w, x, y, dy, ymax, sx, jlim, tb) || jlim >= ex) return true;
    uint32_t slot = 0;
    if (lane == 0) slot = atomicAdd(q.long_count, 1u);
    slot = __shfl_sync(0xffffffffu, slot, 0);
    if (slot < q.long_cap) {
        if (lane == 0) {
            LongItem it;
            it.r = r;
            it.x = x;
            it.y = y;
            it.w = (int32_t)w;
            it.ymax = (int32_t)ymax;
            it.pad = q.qid;
            it.j0 = jlim;
            it.j1 = ex;
            q.longs[slot] = it;
        }
    } else {
        // Deferred list full: finish the scan here.
        scan_wedges_warp<P>(G, q, tau, r, w, x, y, dy, ymax, jlim, ex, tb);
    }
    return true;
}

template <int P>
__global__ void __launch_bounds__(RBLK) k_round_warp(DevGraph G, Query q, int64_t lo, int64_t hi) {
    const volatile uint32_t* stop_rev = &q.st->stop_rev;
    if (lo >= (int64_t)(STOP_NONE - *stop_rev)) return;
    if (*(volatile const uint32_t*)&q.st->err) return;  // the query has already failed
    const unsigned long long tau = ld_volatile_u64(&q.st->tau);
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * MIN_WARPS;
    Tally tb, tu;
    tb.on = q.qbytes != nullptr;
    tu.on = tb.on && lane == 0;
    for (int64_t r = lo + (int64_t)blockIdx.x * MIN_WARPS + (threadIdx.x >> 5); r < hi; r += nwarps) {
        uint32_t sr = 0;
        if (lane == 0) sr = *stop_rev;
        sr = __shfl_sync(0xffffffffu, sr, 0);  // one reading for the whole warp
        if (r >= (int64_t)(STOP_NONE - sr)) break;
        if (!process_edge_warp<P>(G, q, tau, (int32_t)r, tb, tu)) break;
    }
    tb.n += tu.n;
    flush_tally(q, tb);
}

// ---------------------------------------------------------------------------
// Deferred long scans: one block per item.  y's oriented row (ids) is
// staged in shared memory with a bulk async copy completed on an mbarrier;
// closing edges that y owns are binary searches there, the others searches
// of the neighbour's oriented row in global memory.  Oriented rows longer
// than STAGE_MAX are searched in global memory too.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

// Stages y's oriented row (ids; beg = orowptr[y], len entries) in shared
// memory with one bulk copy (bounded wait: at most `limit` polls; a limit of
// 0 does not wait at all, which tests use to take the timeout path on
// purpose).  Returns false if the wait ran out (error recorded); the copy in
// flight is then drained with the full WAIT_LIMIT before the block goes on,
// so no copy outlives its block.
__device__ __forceinline__ bool stage_row(const DevGraph& G, int64_t beg, int32_t len, int32_t* srow,
                                          uint64_t* bar, uint32_t& phase, int32_t& off, uint32_t* err,
                                          int* timed_out, uint32_t limit) {
    // 16-byte aligned source: round the start down, the size up (the id
    // array has 16 bytes of slack after its end).
    const int64_t a0 = beg & ~int64_t(3);
    off = (int32_t)(beg - a0);
    const uint32_t bytes = (uint32_t)(((off + len) * 4 + 15) & ~15);
    if (threadIdx.x == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(bar, bytes);
        bulk_g2s(srow, G.ocol + a0, bytes, bar);
    }
    bool landed = false;
    for (uint32_t spins = 0; spins < limit; spins++) {
        if (mbar_try_wait(bar, phase)) {
            landed = true;
            break;
        }
    }
    if (!landed) {
        atomicOr(err, DEV_ERR_TIMEOUT);
        *timed_out = 1;
    }
    const uint32_t cur = phase;
    phase ^= 1u;
    __syncthreads();
    if (*timed_out) {
        uint32_t s2 = 0;
        while (!mbar_try_wait(bar, cur) && ++s2 < WAIT_LIMIT) {
        }
        return false;
    }
    return true;
}

// One deferred scan, all threads of the block.  Warps take 32-entry chunks
// in order; the wedge bound only decreases along the list, so a warp whose
// chunk fails entirely stops.
template <int P, bool SAMPLED>
__device__ __forceinline__ void long_scan(const DevGraph& G, const Query& q, unsigned long long tau,
                                          const LongItem& item, const int32_t* srow, int32_t off,
                                          int64_t obeg, int32_t ody, int64_t dy, bool staged, Tally& tb) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t w = (uint32_t)item.w, ymax = (uint32_t)item.ymax;
    const int32_t x = item.x, y = item.y, r = item.r;
    for (int64_t base = item.j0 + (int64_t)wid * 32; base < item.j1; base += LBLK) {
        const int64_t j = base + lane;
        bool live = false;
        uint32_t wxc = 0;
        if (j < item.j1) {
            wxc = (uint32_t)__ldg(G.wwt + j);
            tb.add(4);
            live = boundof<P>(w, wxc, ymax, q.gp, q.fw != 0) >= tau;
        }
        if (__ballot_sync(0xffffffffu, live) == 0) break;
        int32_t c = 0;
        if (live) {
            c = __ldg(G.wcol + j);
            tb.add(4);
            if (SAMPLED && c == y) live = false;  // the edge itself
        }
        if (live) {
            int32_t wyc = 0, ryc = -1;
            bool found = false;
            if (y_owns(G, y, dy, c, tb)) {
                if (staged) {
                    int lo = 0, hi = ody;
                    while (lo < hi) {
                        const int mid = (lo + hi) >> 1;
                        if (srow[off + mid] < c) lo = mid + 1;
                        else hi = mid;
                    }
                    if (lo < ody && srow[off + lo] == c) {
                        found = true;
                        wyc = __ldg(G.owt + obeg + lo);
                        ryc = __ldg(G.ork + obeg + lo);
                        tb.add(8);
                    }
                } else {
                    found = search_oriented(G, y, c, wyc, ryc, tb);
                }
            } else {
                found = search_oriented(G, c, y, wyc, ryc, tb);
            }
            if (found && (tb.add(4), owns<SAMPLED>(q, r, __ldg(G.wrk + j), ryc))) {
                const unsigned long long key = keyof<P>(w, wxc, (uint32_t)wyc, q.gp, q.fw != 0);
                if (key >= tau) {
                    int32_t a = x, b = y, cc = c;
                    sort3(a, b, cc);
                    append(q, key, a, b, cc);
                }
            }
        }
    }
}

// Deferred long scans: one block per item.  y's oriented row (ids) is
// staged in shared memory with a bulk async copy completed on an mbarrier;
// closing edges that y owns are binary searches there, the others searches
// of the neighbour's oriented row in global memory.  Oriented rows longer
// than STAGE_MAX are searched in global memory too.
template <int P, bool SAMPLED = false>
__global__ void __launch_bounds__(LBLK) k_long(DevGraph G, Query q);

// Dynamic shared memory of k_long: one staged row plus 16 bytes of rounding.
constexpr size_t LONG_SMEM = (size_t)STAGE_MAX * 4 + 16;

// Opts k_long<P, SAMPLED> in to LONG_SMEM bytes of dynamic shared memory on
// the current device (once per device).
template <int P, bool SAMPLED>
int long_optin() {
    static std::atomic<uint64_t> done{0};
    return smem_optin((const void*)k_long<P, SAMPLED>, (int)LONG_SMEM, done);
}

template <int P, bool SAMPLED>
__global__ void __launch_bounds__(LBLK) k_long(DevGraph G, Query q) {
    extern __shared__ __align__(128) unsigned char lsm[];
    int32_t* srow = reinterpret_cast<int32_t*>(lsm);
    __shared__ __align__(8) uint64_t bar;
    __shared__ int timed_out;
    const uint32_t n_items = min(*(volatile const uint32_t*)q.long_count, q.long_cap);
    if (blockIdx.x >= n_items) return;
    if (*(volatile const uint32_t*)&q.st->err) return;  // the query has already failed
    const unsigned long long tau = ld_volatile_u64(&q.st->tau);
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        timed_out = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    uint32_t phase = 0;
    Tally tb;
    tb.on = q.qbytes != nullptr;
    for (uint32_t it = blockIdx.x; it < n_items; it += gridDim.x) {
        const LongItem item = q.longs[it];
        const int64_t dy = __ldg(G.rowptr + item.y + 1) - __ldg(G.rowptr + item.y);
        const int64_t obeg = __ldg(G.orowptr + item.y);
        const int32_t ody = (int32_t)(__ldg(G.orowptr + item.y + 1) - obeg);
        const bool staged = ody > 0 && ody <= STAGE_MAX;
        int32_t off = 0;
        if (staged && !stage_row(G, obeg, ody, srow, &bar, phase, off, &q.st->err, &timed_out,
                                 q.wait_first))
            break;
        if (staged && threadIdx.x == 0) tb.add((uint32_t)ody * 4u + 32u);  // offsets, the staged row
        long_scan<P, SAMPLED>(G, q, tau, item, srow, off, obeg, ody, dy, staged, tb);
        __syncthreads();  // the staged row is reused by the next item
    }
    flush_tally(q, tb);
}

// ---------------------------------------------------------------------------
// Selection under the total order (key desc, a asc, b asc, c asc).
// Each candidate maps to a 5-word tuple where smaller is better:
//   (~key_hi, ~key_lo, a, b, c).  An MSB-first radix select over its 20
// bytes finds the prefix P such that exactly K candidates have tuple
// prefix <= P; those are kept (compacted in place).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t tuple_word(unsigned long long key, int4 t, int wi) {
    switch (wi) {
        case 0: return ~(uint32_t)(key >> 32);
        case 1: return ~(uint32_t)key;
        case 2: return (uint32_t)t.x;
        case 3: return (uint32_t)t.y;
        default: return (uint32_t)t.z;
    }
}

// Compare the first 'depth' bytes of a candidate's tuple with the prefix
// (pw = prefix words).  Returns <0, 0, >0.
__device__ __forceinline__ int cmp_prefix(unsigned long long key, int4 t, const uint32_t* pw,
                                          int depth) {
    const int full = depth >> 2, rem = depth & 3;
    for (int wi = 0; wi < full; wi++) {
        const uint32_t a = tuple_word(key, t, wi);
        if (a != pw[wi]) return a < pw[wi] ? -1 : 1;
    }
    if (rem) {
        const uint32_t mask = 0xffffffffu << (32 - 8 * rem);
        const uint32_t a = tuple_word(key, t, full) & mask;
        const uint32_t b = pw[full] & mask;
        if (a != b) return a < b ? -1 : 1;
    }
    return 0;
}

struct SelectSmem {
    unsigned long long prefix;   // key-only select: chosen high bytes
    unsigned long long maxkey;
    uint32_t need;               // key-only select: remaining rank
    uint32_t hist[256];
    uint32_t pw[5];
    uint32_t below;   // candidates strictly better than the prefix
    uint32_t eq;      // candidates equal to the prefix
    uint32_t done;
    uint32_t warp_cnt[SBLK / 32];
    uint32_t kept;
    unsigned long long minkey;
};

// Keeps exactly K = min(K_want, n) best candidates at the front; returns the
// kept count and sets *minkey_out to their smallest key.
__device__ uint32_t select_and_compact(unsigned long long* ckey, int4* ctri, uint32_t n,
                                       uint32_t K, SelectSmem& S,
                                       unsigned long long* minkey_out) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid < 5) S.pw[tid] = 0;
    if (tid == 0) {
        S.below = 0;
        S.eq = n;
        S.done = (n <= K) ? 1u : 0u;
        S.minkey = ~0ull;
    }
    __syncthreads();
    int depth = 0;  // bytes fixed in the prefix
    while (!S.done && depth < 20) {
        for (int i = tid; i < 256; i += SBLK) S.hist[i] = 0;
        __syncthreads();
        const int wi = depth >> 2, sh = 24 - 8 * (depth & 3);
        for (uint32_t base = 0; base < n; base += SBLK) {
            const uint32_t i = base + tid;
            uint32_t d = 256;
            if (i < n) {
                const unsigned long long kk = ckey[i];
                const int4 t = ctri[i];
                if (cmp_prefix(kk, t, S.pw, depth) == 0) d = (tuple_word(kk, t, wi) >> sh) & 255u;
            }
            const uint32_t peers = __match_any_sync(0xffffffffu, d);
            if (d < 256 && (__ffs(peers) - 1) == lane) atomicAdd(&S.hist[d], __popc(peers));
        }
        __syncthreads();
        if (tid == 0) {
            // Need the K-th overall: K - below among the prefix-equal ones.
            const uint32_t need = K - S.below;
            uint32_t acc = 0, dsel = 0;
            for (uint32_t d = 0; d < 256; d++) {
                const uint32_t h = S.hist[d];
                if (acc + h >= need) {
                    dsel = d;
                    break;
                }
                acc += h;
            }
            S.below += acc;
            S.eq = S.hist[dsel];
            S.pw[wi] |= dsel << sh;
            if (S.below + S.eq == K) S.done = 1;
        }
        __syncthreads();
        depth++;
    }
    const int final_depth = depth;
    // Compact in place: keep tuple prefix <= P (or everything if n <= K).
    const bool keep_all = (n <= K);
    uint32_t out = 0;
    unsigned long long mk = ~0ull;
    for (uint32_t base = 0; base < n; base += SBLK) {
        const uint32_t i = base + tid;
        bool keep = false;
        unsigned long long kk = 0;
        int4 t = make_int4(0, 0, 0, 0);
        if (i < n) {
            kk = ckey[i];
            t = ctri[i];
            keep = keep_all || cmp_prefix(kk, t, S.pw, final_depth) <= 0;
        }
        const uint32_t b = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) S.warp_cnt[wid] = __popc(b);
        __syncthreads();
        if (tid == 0) {
            uint32_t acc = 0;
            for (int wv = 0; wv < SBLK / 32; wv++) {
                const uint32_t c = S.warp_cnt[wv];
                S.warp_cnt[wv] = acc;
                acc += c;
            }
            S.kept = acc;
        }
        __syncthreads();
        if (keep) {
            const uint32_t p = out + S.warp_cnt[wid] + __popc(b & ((1u << lane) - 1u));
            ckey[p] = kk;  // p <= i: writes never overtake unread entries
            ctri[p] = t;
            mk = kk < mk ? kk : mk;
        }
        out += S.kept;
        __syncthreads();
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, mk, o);
        mk = y < mk ? y : mk;
    }
    if (lane == 0) atomicMin(&S.minkey, mk);
    __syncthreads();
    *minkey_out = S.minkey;
    return out;
}

// The K-th largest key among n candidates (one block, MSB-first over the
// significant bytes only).
__device__ unsigned long long kth_key(const unsigned long long* ckey, uint32_t n, uint32_t K,
                                      SelectSmem& S) {
    const int tid = threadIdx.x, lane = tid & 31;
    unsigned long long mx = 0;
    for (uint32_t i = tid; i < n; i += SBLK) mx = max(mx, ckey[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, mx, o);
        mx = y > mx ? y : mx;
    }
    if (tid == 0) {
        S.prefix = 0;
        S.maxkey = 0;
        S.need = K;
    }
    __syncthreads();
    if (lane == 0) atomicMax(&S.maxkey, mx);
    __syncthreads();
    int nbytes = 0;
    for (unsigned long long t = S.maxkey; t; t >>= 8) nbytes++;
    for (int byte = nbytes - 1; byte >= 0; byte--) {
        const int shift = 8 * byte;
        const unsigned long long hi_mask = (shift + 8 >= 64) ? 0ull : (~0ull << (shift + 8));
        for (int i = tid; i < 256; i += SBLK) S.hist[i] = 0;
        __syncthreads();
        const unsigned long long prefix = S.prefix;
        for (uint32_t base = 0; base < n; base += SBLK) {
            const uint32_t i = base + tid;
            uint32_t d = 256;
            if (i < n) {
                const unsigned long long kk = ckey[i];
                if ((kk & hi_mask) == (prefix & hi_mask)) d = (uint32_t)(kk >> shift) & 255u;
            }
            const uint32_t peers = __match_any_sync(0xffffffffu, d);
            if (d < 256 && (__ffs(peers) - 1) == lane) atomicAdd(&S.hist[d], __popc(peers));
        }
        __syncthreads();
        if (tid == 0) {
            const uint32_t need = S.need;
            uint32_t acc = 0;
            int dsel = 0;
            for (int d = 255; d >= 0; d--) {
                const uint32_t h = S.hist[d];
                if (acc + h >= need) {
                    dsel = d;
                    break;
                }
                acc += h;
            }
            S.need = need - acc;
            S.prefix = prefix | ((unsigned long long)dsel << shift);
        }
        __syncthreads();
    }
    const unsigned long long T = S.prefix;
    __syncthreads();
    return T;
}

// Keeps candidates with key >= T at the front (in place); returns how many.
__device__ uint32_t compact_ge(unsigned long long* ckey, int4* ctri, uint32_t n,
                               unsigned long long T, SelectSmem& S) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    uint32_t out = 0;
    for (uint32_t base = 0; base < n; base += SBLK) {
        const uint32_t i = base + tid;
        bool keep = false;
        unsigned long long kk = 0;
        int4 t = make_int4(0, 0, 0, 0);
        if (i < n) {
            kk = ckey[i];
            keep = kk >= T;
            if (keep) t = ctri[i];
        }
        const uint32_t b = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) S.warp_cnt[wid] = __popc(b);
        __syncthreads();
        if (tid == 0) {
            uint32_t acc = 0;
            for (int wv = 0; wv < SBLK / 32; wv++) {
                const uint32_t c = S.warp_cnt[wv];
                S.warp_cnt[wv] = acc;
                acc += c;
            }
            S.kept = acc;
        }
        __syncthreads();
        if (keep) {
            const uint32_t p = out + S.warp_cnt[wid] + __popc(b & ((1u << lane) - 1u));
            ckey[p] = kk;  // p <= i: writes never overtake unread entries
            ctri[p] = t;
        }
        out += S.kept;
        __syncthreads();
    }
    return out;
}

// After each round: tau = the k-th largest key among the candidates (a
// lower bound on the final k-th key, since they are k distinct triangles),
// and candidates below tau are dropped.  Ties with tau stay; the final step
// resolves them by the vertex triple.
__device__ void select_round(const Query& q, SelectSmem& S) {
    const uint32_t err = *(volatile uint32_t*)&q.st->err;
    if (err) return;
    const uint32_t n = min(*(volatile uint32_t*)&q.st->count, q.cap);
    if (n == q.st->selected || n < (uint32_t)q.k) {
        if (threadIdx.x == 0) *q.long_count = 0;
        return;
    }
    const unsigned long long T = kth_key(q.ckey, n, (uint32_t)q.k, S);
    const uint32_t kept = compact_ge(q.ckey, q.ctri, n, T, S);
    if (threadIdx.x == 0) {
        q.st->count = kept;
        q.st->selected = kept;
        *q.long_count = 0;
        if (T > q.st->tau) q.st->tau = T;
    }
}

__global__ void __launch_bounds__(SBLK) k_select(Query q) {
    __shared__ SelectSmem S;
    select_round(q, S);
}

// Final ranking: candidate i's rank is the number of kept candidates before
// it in the total order.
__device__ __forceinline__ bool before(unsigned long long ka, int4 a, unsigned long long kb, int4 b) {
    if (ka != kb) return ka > kb;
    if (a.x != b.x) return a.x < b.x;
    if (a.y != b.y) return a.y < b.y;
    return a.z < b.z;
}

// Candidate i's rank is the number of kept candidates before it in the
// total order; one warp per candidate.  Also writes the status word.
template <int P>
__device__ __forceinline__ void rank_one(const Query& q, uint32_t i, wtri_tri* out_tri,
                                         double* out_w, int32_t* out_count,
                                         unsigned long long* out_key = nullptr) {
    const uint32_t err = *(volatile uint32_t*)&q.st->err;
    const uint32_t n = min(*(volatile uint32_t*)&q.st->count, q.cap);
    const int lane = threadIdx.x & 31;
    if (i == 0 && lane == 0) {
        // a timeout first: it stops the per-round compaction, so a buffer
        // overflow that follows it is its consequence, not the cause
        int32_t status = (int32_t)n;
        if (err & DEV_ERR_TIMEOUT) status = WTRI_ETIMEOUT;
        else if (err & DEV_ERR_OVERFLOW) status = WTRI_ENOMEM;
        else if (err) status = WTRI_ECUDA;
        *out_count = status;
    }
    if (err || i >= n) return;
    const unsigned long long ki = q.ckey[i];
    const int4 ti = q.ctri[i];
    uint32_t rank = 0;
    for (uint32_t j = lane; j < n; j += 32) rank += before(q.ckey[j], q.ctri[j], ki, ti) ? 1u : 0u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rank += __shfl_xor_sync(0xffffffffu, rank, o);
    if (lane == 0) {
        out_tri[rank].a = ti.x;
        out_tri[rank].b = ti.y;
        out_tri[rank].c = ti.z;
        double val;
        if (P == P_ONE) val = (double)ki / 3.0;
        else if (P == P_TWO) val = sqrt((double)ki / 3.0);
        else if (P == P_GEO) val = cbrt((double)ki);
        else if (P == P_GEN) val = __longlong_as_double((long long)ki);
        else val = q.fw ? (double)__uint_as_float((uint32_t)ki) : (double)ki;  // min, max
        out_w[rank] = val;
        if (out_key) out_key[rank] = ki;
    }
}

template <int P>
__global__ void __launch_bounds__(256) k_rank_scatter(Query q, wtri_tri* out_tri, double* out_w,
                                                      int32_t* out_count,
                                                      unsigned long long* out_key) {
    const uint32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= (uint32_t)max(q.k, 1)) return;
    rank_one<P>(q, i, out_tri, out_w, out_count, out_key);
}

__device__ void final_select(const Query& q, SelectSmem& S) {
    const uint32_t err = *(volatile uint32_t*)&q.st->err;
    if (err) return;
    const uint32_t n = min(*(volatile uint32_t*)&q.st->count, q.cap);
    unsigned long long mk;
    const uint32_t kept = select_and_compact(q.ckey, q.ctri, n, (uint32_t)q.k, S, &mk);
    if (threadIdx.x == 0) q.st->count = kept;
}

__global__ void __launch_bounds__(SBLK) k_final_select(Query q) {
    __shared__ SelectSmem S;
    final_select(q, S);
}

}  // namespace
}  // namespace wtri
