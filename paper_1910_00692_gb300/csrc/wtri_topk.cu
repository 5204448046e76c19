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
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "wtri_internal.cuh"

namespace cg = cooperative_groups;

namespace wtri {
namespace {

constexpr int RBLK = 256;          // k_round block
constexpr int LBLK = 256;          // k_long block
constexpr int SBLK = 1024;         // k_select block
constexpr int T_SHORT = 32;        // wedges a thread scans before deferring
constexpr int STAGE_MAX = 24576;   // ids of a y row staged in shared memory (96 KB)
constexpr int64_t FIRST_ROUND = 64;
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
    int32_t pad;
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
};

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

template <int P>
__device__ __forceinline__ unsigned long long keyof(uint32_t a, uint32_t b, uint32_t c) {
    if (P == P_ONE) return (unsigned long long)a + b + c;
    if (P == P_TWO)
        return (unsigned long long)a * a + (unsigned long long)b * b + (unsigned long long)c * c;
    if (P == P_MAX) return (unsigned long long)max(a, max(b, c));
    return (unsigned long long)min(a, min(b, c));
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

// Position just after edge r's own entry in x's weight-sorted list.
__device__ __forceinline__ int64_t suffix_start(const DevGraph& G, int32_t x, int32_t r,
                                                uint32_t* err) {
    int64_t lo = G.rowptr[x], hi = G.rowptr[x + 1];
    const int64_t end = hi;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (__ldg(G.wrk + mid) < r) lo = mid + 1;
        else hi = mid;
    }
    if (lo >= end || __ldg(G.wrk + lo) != r) {
        atomicOr(err, DEV_ERR_INTERNAL);
        return end;
    }
    return lo + 1;
}

// Closing edge (y, c) in the oriented lists: stored once, at the endpoint of
// lower (degree, id) rank, rows ascending by id (row s starts at rowptr[s]
// and holds odeg[s] entries).
__device__ __forceinline__ bool probe_oriented(const DevGraph& G, int32_t y, int32_t dy, int32_t c,
                                               int32_t& wyc, int32_t& ryc) {
    const int32_t dc = __ldg(G.deg + c);
    const bool ylow = dy < dc || (dy == dc && y < c);
    const int32_t s = ylow ? y : c, t = ylow ? c : y;
    int64_t lo = __ldg(G.rowptr + s), hi = lo + __ldg(G.odeg + s);
    const int64_t end = hi;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (__ldg(G.ocol + mid) < t) lo = mid + 1;
        else hi = mid;
    }
    if (lo < end && __ldg(G.ocol + lo) == t) {
        wyc = __ldg(G.owt + lo);
        ryc = __ldg(G.ork + lo);
        return true;
    }
    return false;
}

__device__ __forceinline__ void append(const Query& q, unsigned long long key, int32_t a, int32_t b,
                                       int32_t c) {
    cg::coalesced_group g = cg::coalesced_threads();
    uint32_t base = 0;
    if (g.thread_rank() == 0) base = atomicAdd(&q.st->count, (uint32_t)g.size());
    base = g.shfl(base, 0);
    const uint32_t idx = base + g.thread_rank();
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
                                            int32_t x, int32_t y, int32_t dy, uint32_t ymax,
                                            int64_t& j, int64_t jstop, bool& done) {
    for (; j < jstop; j++) {
        const uint32_t wxc = (uint32_t)__ldg(G.wwt + j);
        if (keyof<P>(w, wxc, ymax) < tau) {  // wedge bound, non-increasing along the list
            done = true;
            return;
        }
        const int32_t c = __ldg(G.wcol + j);
        if (SAMPLED && c == y) continue;  // the edge itself (full rows in sampled mode)
        int32_t wyc, ryc;
        if (probe_oriented(G, y, dy, c, wyc, ryc) &&
            owns<SAMPLED>(q, r, __ldg(G.wrk + j), ryc)) {
            const unsigned long long key = keyof<P>(w, wxc, (uint32_t)wyc);
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
                                             unsigned long long tau, int32_t idx) {
    const int32_t r = SAMPLED ? __ldg(q.slist + idx) : idx;
    const uint32_t w = (uint32_t)__ldg(G.ord_w + r);
    if (!SAMPLED && keyof<P>(w, w, w) < tau) {
        // every later edge has a bound no larger: record the first such edge
        atomicMax(&q.st->stop_rev, STOP_NONE - (uint32_t)r);
        return false;
    }
    const int32_t u = __ldg(G.ord_u + r), v = __ldg(G.ord_v + r);
    // Exact mode scans what comes after r in each list; sampled mode scans
    // whole lists (the other two edges may be heavier than a drawn edge).
    const int64_t su = SAMPLED ? __ldg(G.rowptr + u) : suffix_start(G, u, r, &q.st->err);
    const int64_t sv = SAMPLED ? __ldg(G.rowptr + v) : suffix_start(G, v, r, &q.st->err);
    const int64_t eu = __ldg(G.rowptr + u + 1), ev = __ldg(G.rowptr + v + 1);
    if (su >= eu || sv >= ev) return true;  // no edge after r on one side: owns nothing
    const uint32_t umax = (uint32_t)__ldg(G.wwt + su), vmax = (uint32_t)__ldg(G.wwt + sv);
    if (keyof<P>(w, umax, vmax) < tau) return true;  // edge bound
    // Scan the shorter suffix; probe the other endpoint.
    const bool xu = (eu - su) <= (ev - sv);
    const int32_t x = xu ? u : v, y = xu ? v : u;
    const int64_t sx = xu ? su : sv, ex = xu ? eu : ev;
    const uint32_t ymax = xu ? vmax : umax;
    const int32_t dy = __ldg(G.deg + y);
    int64_t j = sx;
    bool done = false;
    scan_wedges<P, SAMPLED>(G, q, tau, r, w, x, y, dy, ymax, j, min(ex, sx + (int64_t)T_SHORT),
                            done);
    if (!done && j < ex) {
        const uint32_t slot = atomicAdd(&q.st->long_count, 1u);
        if (slot < q.long_cap) {
            LongItem it;
            it.r = r;
            it.x = x;
            it.y = y;
            it.w = (int32_t)w;
            it.ymax = (int32_t)ymax;
            it.pad = 0;
            it.j0 = j;
            it.j1 = ex;
            q.longs[slot] = it;
        } else {
            // Deferred list full: finish the scan here.
            scan_wedges<P, SAMPLED>(G, q, tau, r, w, x, y, dy, ymax, j, ex, done);
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
    const unsigned long long tau = ld_volatile_u64(&q.st->tau);
    const int64_t stride = (int64_t)gridDim.x * RBLK;
    for (int64_t r64 = lo + (int64_t)blockIdx.x * RBLK + threadIdx.x; r64 < hi; r64 += stride) {
        if (r64 >= (int64_t)(STOP_NONE - *stop_rev)) break;
        if (!process_edge<P, SAMPLED>(G, q, tau, (int32_t)r64)) break;
    }
}

// Grid of a round: a few resident blocks per SM, striding over the range.
inline unsigned round_grid(int64_t edges) {
    const int64_t cap = (int64_t)sm_count() * 8;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(cap, (edges + RBLK - 1) / RBLK));
}

// ---------------------------------------------------------------------------
// Deferred long scans: one block per item.  The y row (ids) is staged in
// shared memory with a bulk async copy completed on an mbarrier; lookups of
// the closing edge are binary searches there.  Rows longer than STAGE_MAX
// fall back to the oriented lists in global memory.
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

template <int P, bool SAMPLED = false>
__global__ void __launch_bounds__(LBLK) k_long(DevGraph G, Query q) {
    extern __shared__ __align__(128) unsigned char lsm[];
    int32_t* srow = reinterpret_cast<int32_t*>(lsm);
    __shared__ __align__(8) uint64_t bar;
    __shared__ int timed_out;
    const uint32_t n_items = min(*(volatile const uint32_t*)&q.st->long_count, q.long_cap);
    if (blockIdx.x >= n_items) return;
    const unsigned long long tau = ld_volatile_u64(&q.st->tau);
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        timed_out = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    uint32_t phase = 0;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (uint32_t it = blockIdx.x; it < n_items; it += gridDim.x) {
        const LongItem item = q.longs[it];
        const int64_t ybeg = __ldg(G.rowptr + item.y), yend = __ldg(G.rowptr + item.y + 1);
        const int32_t dy = (int32_t)(yend - ybeg);
        const bool staged = dy <= STAGE_MAX;
        int32_t off = 0;
        if (staged) {
            // 16-byte aligned source: round the start down, the size up (the
            // id array has 16 bytes of slack after its end).
            const int64_t a0 = ybeg & ~int64_t(3);
            off = (int32_t)(ybeg - a0);
            const uint32_t bytes = (uint32_t)(((off + dy) * 4 + 15) & ~15);
            if (threadIdx.x == 0) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_expect_tx(&bar, bytes);
                bulk_g2s(srow, G.scol + a0, bytes, &bar);
            }
            // Every thread waits (bounded).
            uint32_t spins = 0;
            while (!mbar_try_wait(&bar, phase)) {
                if (++spins >= WAIT_LIMIT) {
                    atomicOr(&q.st->err, DEV_ERR_TIMEOUT);
                    timed_out = 1;
                    break;
                }
            }
            phase ^= 1u;
            __syncthreads();
            if (timed_out) {
                // Give the copy a second bounded chance to land before exit.
                uint32_t s2 = 0;
                while (!mbar_try_wait(&bar, phase ^ 1u) && ++s2 < WAIT_LIMIT) {
                }
                return;
            }
        }
        const uint32_t w = (uint32_t)item.w, ymax = (uint32_t)item.ymax;
        const int32_t x = item.x, y = item.y, r = item.r;
        // Warps take 32-entry chunks in order; the wedge bound only decreases
        // along the list, so a warp whose chunk fails entirely stops.
        for (int64_t base = item.j0 + (int64_t)wid * 32; base < item.j1; base += LBLK) {
            const int64_t j = base + lane;
            bool live = false;
            uint32_t wxc = 0;
            if (j < item.j1) {
                wxc = (uint32_t)__ldg(G.wwt + j);
                live = keyof<P>(w, wxc, ymax) >= tau;
            }
            if (__ballot_sync(0xffffffffu, live) == 0) break;
            if (live) {
                const int32_t c = __ldg(G.wcol + j);
                if (SAMPLED && c == y) live = false;  // the edge itself
            }
            if (live) {
                const int32_t c = __ldg(G.wcol + j);
                int32_t wyc = 0, ryc = -1;
                bool found = false;
                if (staged) {
                    int lo = 0, hi = dy;
                    while (lo < hi) {
                        const int mid = (lo + hi) >> 1;
                        if (srow[off + mid] < c) lo = mid + 1;
                        else hi = mid;
                    }
                    if (lo < dy && srow[off + lo] == c) {
                        found = true;
                        wyc = __ldg(G.swt + ybeg + lo);
                        ryc = __ldg(G.srk + ybeg + lo);
                    }
                } else {
                    found = probe_oriented(G, y, dy, c, wyc, ryc);
                }
                if (found && owns<SAMPLED>(q, r, __ldg(G.wrk + j), ryc)) {
                    const unsigned long long key = keyof<P>(w, wxc, (uint32_t)wyc);
                    if (key >= tau) {
                        int32_t a = x, b = y, cc = c;
                        sort3(a, b, cc);
                        append(q, key, a, b, cc);
                    }
                }
            }
        }
        __syncthreads();  // the staged row is reused by the next item
    }
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
__global__ void __launch_bounds__(SBLK) k_select(Query q) {
    __shared__ SelectSmem S;
    const uint32_t err = *(volatile uint32_t*)&q.st->err;
    if (err) return;
    const uint32_t n = min(*(volatile uint32_t*)&q.st->count, q.cap);
    if (n == q.st->selected || n < (uint32_t)q.k) {
        if (threadIdx.x == 0) q.st->long_count = 0;
        return;
    }
    const unsigned long long T = kth_key(q.ckey, n, (uint32_t)q.k, S);
    const uint32_t kept = compact_ge(q.ckey, q.ctri, n, T, S);
    if (threadIdx.x == 0) {
        q.st->count = kept;
        q.st->selected = kept;
        q.st->long_count = 0;
        if (T > q.st->tau) q.st->tau = T;
    }
}

// Final ranking: candidate i's rank is the number of kept candidates before
// it in the total order.
__device__ __forceinline__ bool before(unsigned long long ka, int4 a, unsigned long long kb, int4 b) {
    if (ka != kb) return ka > kb;
    if (a.x != b.x) return a.x < b.x;
    if (a.y != b.y) return a.y < b.y;
    return a.z < b.z;
}

template <int P>
__global__ void __launch_bounds__(256) k_rank_scatter(Query q, wtri_tri* out_tri, double* out_w,
                                                      int32_t* out_count) {
    const uint32_t err = *(volatile uint32_t*)&q.st->err;
    const uint32_t n = min(*(volatile uint32_t*)&q.st->count, q.cap);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        int32_t status = (int32_t)n;
        if (err & DEV_ERR_OVERFLOW) status = WTRI_ENOMEM;
        else if (err & DEV_ERR_TIMEOUT) status = WTRI_ETIMEOUT;
        else if (err) status = WTRI_ECUDA;
        *out_count = status;
    }
    if (err) return;
    // One warp per kept candidate: its rank is the number of kept candidates
    // before it in the total order.
    const uint32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
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
        else val = (double)ki;
        out_w[rank] = val;
    }
}

__global__ void k_final_select(Query q) {
    __shared__ SelectSmem S;
    const uint32_t err = *(volatile uint32_t*)&q.st->err;
    if (err) return;
    const uint32_t n = min(*(volatile uint32_t*)&q.st->count, q.cap);
    unsigned long long mk;
    const uint32_t kept = select_and_compact(q.ckey, q.ctri, n, (uint32_t)q.k, S, &mk);
    if (threadIdx.x == 0) q.st->count = kept;
}

template <int P>
int run_query(const wtri_graph* g, int32_t k, wtri_tri* d_tris, double* d_weight, int32_t* d_count,
              cudaStream_t s, int scale) {
    const DevGraph& G = g->d;
    const int64_t m = G.m;
    const uint32_t cap = (uint32_t)std::min<int64_t>(
        (int64_t(1) << 20) * scale + 16 * (int64_t)k, (int64_t(1) << 31) - 1);
    const uint32_t long_cap = (uint32_t)((1u << 16) * scale);
    const size_t bytes = sizeof(QState) + 256 + (size_t)cap * (8 + 16) + 256 +
                         (size_t)long_cap * sizeof(LongItem) + 256;
    void* buf = nullptr;
    cudaError_t e = cudaMallocAsync(&buf, bytes, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(WTRI_ENOMEM, "query scratch allocation failed");
    }
    char* p = (char*)buf;
    Query q;
    q.st = (QState*)p;
    p += 256;
    q.ckey = (unsigned long long*)p;
    p += (size_t)cap * 8;
    q.ctri = (int4*)p;
    p += (size_t)cap * 16;
    p = (char*)(((uintptr_t)p + 255) & ~(uintptr_t)255);
    q.longs = (LongItem*)p;
    q.cap = cap;
    q.long_cap = long_cap;
    q.k = k;
    q.smark = nullptr;
    q.slist = nullptr;
    WTRI_CUDA(cudaMemsetAsync(q.st, 0, sizeof(QState), s));

    const size_t lsmem = (size_t)STAGE_MAX * 4 + 16;
    static bool attr_done[4] = {false, false, false, false};
    if (!attr_done[P]) {
        WTRI_CUDA(cudaFuncSetAttribute(k_long<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)lsmem));
        attr_done[P] = true;
    }
    const int long_grid = sm_count() * 2;
    static const char* qname[4] = {"query_p=-inf", "query_p=1", "query_p=2", "query_p=+inf"};
    ProfScope whole(qname[P], s, 0.0, 0);
    int64_t lo = 0, size = FIRST_ROUND;
    while (lo < m) {
        const int64_t hi = std::min(m, lo + size);
        {
            ProfScope ps("topk_round", s, 0.0, 1);
            k_round<P><<<round_grid(hi - lo), RBLK, 0, s>>>(G, q, lo, hi);
        }
        {
            ProfScope ps("topk_long", s, 0.0, 1);
            k_long<P><<<long_grid, LBLK, lsmem, s>>>(G, q);
        }
        {
            ProfScope ps("topk_select", s, 0.0, 1);
            k_select<<<1, SBLK, 0, s>>>(q);
        }
        lo = hi;
        size *= ROUND_GROWTH;
    }
    {
        ProfScope ps("topk_final", s, 0.0, 2);
        k_final_select<<<1, SBLK, 0, s>>>(q);
        k_rank_scatter<P><<<ceil_div_u(std::max(k, 1), 8), 256, 0, s>>>(q, d_tris, d_weight, d_count);
    }
    WTRI_CUDA(cudaGetLastError());
    WTRI_CUDA(cudaFreeAsync(buf, s));
    return WTRI_OK;
}

// ---------------------------------------------------------------------------
// Weighted edge sampling (Algorithm 3, Proposition 4.1, Section 4.1).
//
// Draw: with the edges in the edge order and C[r] = sum_{j<=r} w_j^p (exact
// integers), sample s takes x = word 0 of Philox4x64-10(counter (s,0,0,0),
// key (seed,0)), t = floor(x * Z / 2^64), and the edge is the first r with
// C[r] > t.  Equal weights are contiguous in the edge order (Section 4.1's
// weight classes), so the search runs over the class table (start, weight,
// cumulative mass) and the position inside the class is (t - C_prev) /
// w^p.  Drawn edges are marked in a bitmap; the marked positions, in
// ascending order, are then swept like the exact query (heaviest first) in
// sampled-ownership mode.
// ---------------------------------------------------------------------------
typedef unsigned __int128 u128;

// Philox4x64-10 (Salmon et al., SC'11), first output word only.
__device__ __forceinline__ uint64_t philox_word0(uint64_t c0, uint64_t k0) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
    uint64_t c1 = 0, c2 = 0, c3 = 0, k1 = 0;
#pragma unroll
    for (int i = 0; i < 10; i++) {
        const uint64_t hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
        const uint64_t hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
        const uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c1 = lo1;
        c3 = lo0;
        c0 = n0;
        c2 = n2;
        k0 += W0;
        k1 += W1;
    }
    return c0;
}

// Class starts: position r starts a class when its weight differs from r-1.
__global__ void k_class_flags(int64_t m, const int32_t* __restrict__ ow, int32_t* __restrict__ flag) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < m;
         r += (int64_t)gridDim.x * blockDim.x)
        flag[r] = (r == 0 || __ldg(ow + r) != __ldg(ow + r - 1)) ? 1 : 0;
}

__global__ void k_class_starts(int64_t m, const int32_t* __restrict__ flag,
                               const int64_t* __restrict__ cls, int64_t* __restrict__ cstart) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < m;
         r += (int64_t)gridDim.x * blockDim.x)
        if (flag[r]) cstart[cls[r]] = r;
    if (blockIdx.x == 0 && threadIdx.x == 0) cstart[cls[m]] = m;  // sentinel
}

// Inclusive prefix of class masses count * w^p, one block (classes are few:
// one per distinct weight).
template <int P>
__global__ void __launch_bounds__(1024) k_class_mass(const int64_t* __restrict__ cls_total,
                                                     const int64_t* __restrict__ cstart,
                                                     const int32_t* __restrict__ ow,
                                                     u128* __restrict__ cmass) {
    __shared__ u128 warp_sum[32];
    __shared__ u128 carry;
    const int64_t nc = *cls_total;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int64_t base = 0; base < nc; base += 1024) {
        const int64_t c = base + threadIdx.x;
        u128 x = 0;
        if (c < nc) {
            const u128 wv = (u128)(uint64_t)__ldg(ow + cstart[c]);
            x = (u128)(uint64_t)(cstart[c + 1] - cstart[c]) * (P == P_TWO ? wv * wv : wv);
        }
        u128 inc = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t lo = __shfl_up_sync(0xffffffffu, (uint64_t)inc, o);
            const uint64_t hi = __shfl_up_sync(0xffffffffu, (uint64_t)(inc >> 64), o);
            if (lane >= o) inc += ((u128)hi << 64) | lo;
        }
        if (lane == 31) warp_sum[wid] = inc;
        __syncthreads();
        if (threadIdx.x == 0) {
            u128 acc = carry;
            for (int k = 0; k < 32; k++) {
                const u128 t = warp_sum[k];
                warp_sum[k] = acc;
                acc += t;
            }
            carry = acc;
        }
        __syncthreads();
        if (c < nc) cmass[c] = warp_sum[wid] + inc;
        __syncthreads();
    }
}

template <int P>
__global__ void k_draw(int64_t nsamples, uint64_t seed, const int64_t* __restrict__ cls_total,
                       const int64_t* __restrict__ cstart, const int32_t* __restrict__ ow,
                       const u128* __restrict__ cmass, uint32_t* __restrict__ mark) {
    const int64_t nc = *cls_total;
    const u128 Z = cmass[nc - 1];
    const uint64_t zl = (uint64_t)Z, zh = (uint64_t)(Z >> 64);
    for (int64_t sidx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; sidx < nsamples;
         sidx += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t x = philox_word0((uint64_t)sidx, seed);
        const u128 t = (u128)x * zh + (u128)__umul64hi(x, zl);  // floor(x * Z / 2^64)
        int64_t lo = 0, hi = nc;                                   // first class with mass > t
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (cmass[mid] > t) hi = mid;
            else lo = mid + 1;
        }
        const u128 prev = lo > 0 ? cmass[lo - 1] : (u128)0;
        const u128 wv = (u128)(uint64_t)__ldg(ow + cstart[lo]);
        const u128 wp = P == P_TWO ? wv * wv : wv;
        const int64_t r = cstart[lo] + (int64_t)((t - prev) / wp);
        atomicOr(mark + (r >> 5), 1u << (r & 31));
    }
}

__global__ void k_mark_popc(int64_t words, const uint32_t* __restrict__ mark, int32_t* __restrict__ pc) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words;
         i += (int64_t)gridDim.x * blockDim.x)
        pc[i] = __popc(mark[i]);
}

__global__ void k_mark_list(int64_t words, const uint32_t* __restrict__ mark,
                            const int64_t* __restrict__ off, int32_t* __restrict__ list) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t b = mark[i];
        int64_t o = off[i];
        while (b) {
            const int bit = __ffs(b) - 1;
            list[o++] = (int32_t)(i * 32 + bit);
            b &= b - 1;
        }
    }
}

inline unsigned grid_of(int64_t work) {
    const int64_t cap = (int64_t)sm_count() * 16;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(cap, (work + 255) / 256));
}

// Draws the samples into a bitmap over edge-order positions (words =
// ceil(m/32), zeroed here).  Scratch: cls (m+1 int64), cstart (m+1 int64),
// cmass (m u128), flags (m int32).
template <int P>
int draw_samples(const wtri_graph* g, int64_t nsamples, uint64_t seed, uint32_t* mark,
                 cudaStream_t s) {
    const DevGraph& G = g->d;
    const int64_t m = G.m, words = (m + 31) / 32;
    const size_t bytes = 8 * (size_t)(m + 1) * 2 + 16 * (size_t)m + 4 * (size_t)m + 256;
    void* buf = nullptr;
    if (cudaMallocAsync(&buf, bytes, s) != cudaSuccess) {
        cudaGetLastError();
        return set_error(WTRI_ENOMEM, "sampling scratch allocation failed");
    }
    char* p = (char*)buf;
    int64_t* cls = (int64_t*)p;
    p += 8 * (size_t)(m + 1);
    int64_t* cstart = (int64_t*)p;
    p += 8 * (size_t)(m + 1);
    u128* cmass = (u128*)p;
    p += 16 * (size_t)m;
    int32_t* flag = (int32_t*)p;
    WTRI_CUDA(cudaMemsetAsync(mark, 0, 4 * (size_t)words, s));
    {
        ProfScope ps("sample_classes", s, 4.0 * m + 4.0 * m, 1);
        k_class_flags<<<grid_of(m), 256, 0, s>>>(m, G.ord_w, flag);
    }
    WTRI_TRY(exclusive_scan_i32_to_i64(flag, cls, m, s));  // cls[m] = number of classes
    {
        ProfScope ps("sample_class_table", s, 12.0 * m, 2);
        k_class_starts<<<grid_of(m), 256, 0, s>>>(m, flag, cls, cstart);
        k_class_mass<P><<<1, 1024, 0, s>>>(cls + m, cstart, G.ord_w, cmass);
    }
    {
        ProfScope ps("sample_draw", s, 0.0, 1);
        k_draw<P><<<grid_of(nsamples), 256, 0, s>>>(nsamples, seed, cls + m, cstart, G.ord_w, cmass,
                                                    mark);
    }
    WTRI_CUDA(cudaGetLastError());
    WTRI_CUDA(cudaFreeAsync(buf, s));
    return WTRI_OK;
}

template <int P>
int run_sample(const wtri_graph* g, int32_t k, int64_t nsamples, uint64_t seed, wtri_tri* d_tris,
               double* d_weight, int32_t* d_count, cudaStream_t s, int scale) {
    const DevGraph& G = g->d;
    const int64_t m = G.m, words = (m + 31) / 32;
    const uint32_t cap = (uint32_t)std::min<int64_t>(
        (int64_t(1) << 20) * scale + 16 * (int64_t)k, (int64_t(1) << 31) - 1);
    const uint32_t long_cap = (uint32_t)((1u << 16) * scale);
    const size_t qbytes = 256 + (size_t)cap * 24 + 256 + (size_t)long_cap * sizeof(LongItem) + 256;
    const size_t sbytes = 4 * (size_t)words + 8 * (size_t)(words + 1) + 4 * (size_t)words + 4 * (size_t)m + 256;
    void* buf = nullptr;
    if (cudaMallocAsync(&buf, qbytes + sbytes, s) != cudaSuccess) {
        cudaGetLastError();
        return set_error(WTRI_ENOMEM, "sampling query scratch allocation failed");
    }
    char* p = (char*)buf;
    Query q;
    q.st = (QState*)p;
    p += 256;
    q.ckey = (unsigned long long*)p;
    p += (size_t)cap * 8;
    q.ctri = (int4*)p;
    p += (size_t)cap * 16;
    p = (char*)(((uintptr_t)p + 255) & ~(uintptr_t)255);
    q.longs = (LongItem*)p;
    p += (size_t)long_cap * sizeof(LongItem);
    p = (char*)(((uintptr_t)p + 255) & ~(uintptr_t)255);
    uint32_t* mark = (uint32_t*)p;
    p += 4 * (size_t)words;
    p = (char*)(((uintptr_t)p + 7) & ~(uintptr_t)7);
    int64_t* off = (int64_t*)p;
    p += 8 * (size_t)(words + 1);
    int32_t* pc = (int32_t*)p;
    p += 4 * (size_t)words;
    int32_t* list = (int32_t*)p;
    q.cap = cap;
    q.long_cap = long_cap;
    q.k = k;
    q.smark = mark;
    q.slist = list;
    WTRI_CUDA(cudaMemsetAsync(q.st, 0, sizeof(QState), s));
    ProfScope whole(P == P_ONE ? "sample_p=1" : "sample_p=2", s, 0.0, 0);
    WTRI_TRY(draw_samples<P>(g, nsamples, seed, mark, s));
    {
        ProfScope ps("sample_compact", s, 8.0 * words, 2);
        k_mark_popc<<<grid_of(words), 256, 0, s>>>(words, mark, pc);
        WTRI_TRY(exclusive_scan_i32_to_i64(pc, off, words, s));
        k_mark_list<<<grid_of(words), 256, 0, s>>>(words, mark, off, list);
    }
    int64_t nlist = 0;
    WTRI_CUDA(cudaMemcpyAsync(&nlist, off + words, 8, cudaMemcpyDeviceToHost, s));
    WTRI_CUDA(cudaStreamSynchronize(s));
    const size_t lsmem = (size_t)STAGE_MAX * 4 + 16;
    static bool attr_done[4] = {false, false, false, false};
    if (!attr_done[P]) {
        WTRI_CUDA(cudaFuncSetAttribute(k_long<P, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)lsmem));
        attr_done[P] = true;
    }
    const int long_grid = sm_count() * 2;
    int64_t lo = 0, size = FIRST_ROUND;
    while (lo < nlist) {
        const int64_t hi = std::min(nlist, lo + size);
        {
            ProfScope ps("sample_round", s, 0.0, 1);
            k_round<P, true><<<round_grid(hi - lo), RBLK, 0, s>>>(G, q, lo, hi);
        }
        {
            ProfScope ps("sample_long", s, 0.0, 1);
            k_long<P, true><<<long_grid, LBLK, lsmem, s>>>(G, q);
        }
        {
            ProfScope ps("topk_select", s, 0.0, 1);
            k_select<<<1, SBLK, 0, s>>>(q);
        }
        lo = hi;
        size *= ROUND_GROWTH;
    }
    {
        ProfScope ps("topk_final", s, 0.0, 2);
        k_final_select<<<1, SBLK, 0, s>>>(q);
        k_rank_scatter<P><<<ceil_div_u(std::max(k, 1), 8), 256, 0, s>>>(q, d_tris, d_weight, d_count);
    }
    WTRI_CUDA(cudaGetLastError());
    WTRI_CUDA(cudaFreeAsync(buf, s));
    return WTRI_OK;
}

}  // namespace

int topk_device(const wtri_graph* g, int pcode, int32_t k, wtri_tri* d_tris, double* d_weight,
                int32_t* d_count, cudaStream_t stream, int retry_scale) {
    switch (pcode) {
        case P_MIN: return run_query<P_MIN>(g, k, d_tris, d_weight, d_count, stream, retry_scale);
        case P_ONE: return run_query<P_ONE>(g, k, d_tris, d_weight, d_count, stream, retry_scale);
        case P_TWO: return run_query<P_TWO>(g, k, d_tris, d_weight, d_count, stream, retry_scale);
        default: return run_query<P_MAX>(g, k, d_tris, d_weight, d_count, stream, retry_scale);
    }
}

}  // namespace wtri

// ---------------------------------------------------------------------------
// Query variant that allocates nothing.
//
// For callers that may not allocate device memory once they are running:
// for example a server whose device memory is all handed to its own caching
// allocator at start-up, or a latency-critical loop that must never wait on
// the allocator.  The query's scratch (status word, candidate buffer,
// deferred-scan list) lives in one fixed array compiled into the library.
// Every GPU that loads the library keeps this array (NOALLOC_BYTES, about
// 26 MB) until the process exits.  All calls share it: the status word is
// cleared at the start of each call, and calls that overlap on the GPU (on
// different streams, or from several host threads) race on it.
// ---------------------------------------------------------------------------
namespace wtri {
namespace {

constexpr uint32_t NOALLOC_CAP = 1u << 20;     // candidates
constexpr uint32_t NOALLOC_LONG = 1u << 16;    // deferred scans
constexpr int32_t NOALLOC_K_MAX = 16384;
constexpr size_t NOALLOC_CAND_OFF = 256;
constexpr size_t NOALLOC_TRI_OFF = NOALLOC_CAND_OFF + (size_t)NOALLOC_CAP * 8;
constexpr size_t NOALLOC_LONG_OFF = NOALLOC_TRI_OFF + (size_t)NOALLOC_CAP * 16;
constexpr size_t NOALLOC_BYTES = NOALLOC_LONG_OFF + (size_t)NOALLOC_LONG * sizeof(LongItem);
static_assert(sizeof(QState) <= NOALLOC_CAND_OFF, "status word fits its slot");
static_assert(NOALLOC_LONG_OFF % 256 == 0, "aligned deferred list");

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};

// Device address of the fixed array for the current device, looked up once
// per device (with that device current).
int noalloc_scratch(void** out) {
    int dev = 0;
    WTRI_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES)
        return set_error(WTRI_EUNSUPPORTED, "device index above 63");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return cuda_error(e == cudaSuccess ? cudaErrorInvalidSymbol : e,
                              "cudaGetSymbolAddress(static query scratch)", __FILE__, __LINE__);
        }
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return WTRI_OK;
}

template <int P>
int run_query_noalloc(const wtri_graph* g, int32_t k, wtri_tri* d_tris, double* d_weight,
                      int32_t* d_count, cudaStream_t s) {
    const DevGraph& G = g->d;
    const int64_t m = G.m;
    void* base = nullptr;
    WTRI_TRY(noalloc_scratch(&base));
    char* p = (char*)base;
    Query q;
    q.st = (QState*)p;
    q.ckey = (unsigned long long*)(p + NOALLOC_CAND_OFF);
    q.ctri = (int4*)(p + NOALLOC_TRI_OFF);
    q.longs = (LongItem*)(p + NOALLOC_LONG_OFF);
    q.cap = NOALLOC_CAP;
    q.long_cap = NOALLOC_LONG;
    q.k = k;
    q.smark = nullptr;
    q.slist = nullptr;
    // The array keeps the previous call's contents: reset the status word
    // (counters, threshold, stop flag, error bits).
    WTRI_CUDA(cudaMemsetAsync(q.st, 0, sizeof(QState), s));

    const size_t lsmem = (size_t)STAGE_MAX * 4 + 16;
    static bool attr_done[4] = {false, false, false, false};
    if (!attr_done[P]) {
        WTRI_CUDA(cudaFuncSetAttribute(k_long<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)lsmem));
        attr_done[P] = true;
    }
    const int long_grid = sm_count() * 2;
    int64_t lo = 0, size = FIRST_ROUND;
    while (lo < m) {
        const int64_t hi = std::min(m, lo + size);
        k_round<P><<<round_grid(hi - lo), RBLK, 0, s>>>(G, q, lo, hi);
        k_long<P><<<long_grid, LBLK, lsmem, s>>>(G, q);
        k_select<<<1, SBLK, 0, s>>>(q);
        count_launches(3);
        lo = hi;
        size *= ROUND_GROWTH;
    }
    k_final_select<<<1, SBLK, 0, s>>>(q);
    k_rank_scatter<P><<<ceil_div_u(std::max(k, 1), 8), 256, 0, s>>>(q, d_tris, d_weight, d_count);
    count_launches(2);
    WTRI_CUDA(cudaGetLastError());
    return WTRI_OK;
}

}  // namespace
int sample_topk_device(const wtri_graph* g, int pcode, int32_t k, int64_t nsamples, uint64_t seed,
                       wtri_tri* d_tris, double* d_weight, int32_t* d_count, cudaStream_t stream,
                       int retry_scale) {
    if (pcode == P_ONE)
        return run_sample<P_ONE>(g, k, nsamples, seed, d_tris, d_weight, d_count, stream, retry_scale);
    return run_sample<P_TWO>(g, k, nsamples, seed, d_tris, d_weight, d_count, stream, retry_scale);
}

int sample_edges_device(const wtri_graph* g, int pcode, int64_t nsamples, uint64_t seed,
                        uint32_t* d_mark, cudaStream_t stream) {
    if (pcode == P_ONE) return draw_samples<P_ONE>(g, nsamples, seed, d_mark, stream);
    return draw_samples<P_TWO>(g, nsamples, seed, d_mark, stream);
}

}  // namespace wtri

extern "C" WTRI_API int wtri_topk_device_noalloc(const wtri_graph* g, double p, int32_t k,
                                                 wtri_tri* d_tris, double* d_weight,
                                                 int32_t* d_count, void* stream) {
    using namespace wtri;
    if (!g) return set_error(WTRI_EINVAL, "graph is NULL");
    if (k <= 0) return set_error(WTRI_EINVAL, "k must be positive");
    if (k > NOALLOC_K_MAX)
        return set_error(WTRI_EINVAL, "k above 16384, the most the fixed query scratch supports");
    int code = 0;
    WTRI_TRY(p_to_code(p, &code));
    if (!d_tris || !d_weight || !d_count) return set_error(WTRI_EINVAL, "output pointers are NULL");
    cudaStream_t s = stream ? (cudaStream_t)stream : g->stream;
    if (g->d.m == 0) {
        WTRI_CUDA(cudaMemsetAsync(d_count, 0, sizeof(int32_t), s));
        return WTRI_OK;
    }
    switch (code) {
        case P_MIN: return run_query_noalloc<P_MIN>(g, k, d_tris, d_weight, d_count, s);
        case P_ONE: return run_query_noalloc<P_ONE>(g, k, d_tris, d_weight, d_count, s);
        case P_TWO: return run_query_noalloc<P_TWO>(g, k, d_tris, d_weight, d_count, s);
        default: return run_query_noalloc<P_MAX>(g, k, d_tris, d_weight, d_count, s);
    }
}

