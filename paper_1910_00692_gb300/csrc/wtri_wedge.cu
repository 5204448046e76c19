// Weighted wedge sampling (Algorithm 4, Eqs. 6-8, Proposition 4.2, Section
// 4.2) on the device: draws, the triangle set T of the closed wedges, and
// the top-k of T.
//
// Draw s (exact integer arithmetic, identical to the oracle's): with
// D(a) = sum over N(a) of w^p and the words (x0, x1, x2) of
// Philox4x64-10(counter (s, 0, 0, 0), key (seed, 1)):
//   a: the first vertex whose cumulative 2 d_v D(v) exceeds
//      floor(x0 * Z1 / 2^64), Z1 = sum_v 2 d_v D(v)               (Eq. 6);
//   b: entry j of a's weight-sorted row with weight d_a w_j^p + D(a): with
//      t = floor(x1 * 2 d_a D(a) / 2^64), t < d_a D(a) takes the entry whose
//      cumulative w^p first exceeds t / d_a, otherwise
//      j = (t - d_a D(a)) / D(a)                                   (Eq. 7);
//   c: entry j with weight w_j^p + w_ab^p: with
//      t = floor(x2 * (D(a) + d_a w_ab^p) / 2^64), t < D(a) takes the entry
//      whose cumulative w^p first exceeds t, otherwise
//      j = (t - D(a)) / w_ab^p                                     (Eq. 8).
// The wedge closes when c is not b and {b, c} is an edge (looked up in the
// oriented rows).  A closed triangle is identified by the two smallest edge
// ranks among its three edges (two edges fix the triangle), kept once in a
// hash set; the new ones are the candidates of the top-k select.
#include "wtri_query.cuh"

namespace wtri {
namespace {

typedef unsigned __int128 u128;

// Philox4x64-10 (Salmon et al., SC'11): the four output words.
__device__ __forceinline__ void philox4(uint64_t c0, uint64_t k0, uint64_t k1, uint64_t out[4]) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
    uint64_t c1 = 0, c2 = 0, c3 = 0;
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
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

// floor(x * Z / 2^64) for Z < 2^128.
__device__ __forceinline__ u128 mulhi_z(uint64_t x, u128 Z) {
    const uint64_t zl = (uint64_t)Z, zh = (uint64_t)(Z >> 64);
    return (u128)x * zh + (u128)__umul64hi(x, zl);
}

template <int P>
__device__ __forceinline__ uint64_t wpow(int32_t w) {
    const uint64_t x = (uint64_t)(uint32_t)w;
    return P == P_GEO ? 1ull : (P == P_ONE ? x : x * x);
}

constexpr int WBLK = 256;
constexpr unsigned long long HASH_EMPTY = ~0ull;

// Per-row cumulative w^p (u64, one warp per row, a warp scan per 32
// entries) and D(a); flags a row whose sum does not fit 64 bits.
template <int P>
__global__ void __launch_bounds__(WBLK) k_ws_rows(DevGraph G, uint64_t* __restrict__ cum,
                                                  uint64_t* __restrict__ D, uint32_t* err) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * WBLK) >> 5;
    for (int64_t x = ((int64_t)blockIdx.x * WBLK + threadIdx.x) >> 5; x < G.n; x += nwarps) {
        const int64_t b0 = __ldg(G.rowptr + x), e0 = __ldg(G.rowptr + x + 1);
        uint64_t carry = 0;
        bool over = false;
        for (int64_t base = b0; base < e0; base += 32) {
            const int64_t j = base + lane;
            uint64_t v = j < e0 ? wpow<P>(__ldg(G.wwt + j)) : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint64_t y = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) {
                    over |= v + y < v;
                    v += y;
                }
            }
            const uint64_t s = carry + v;
            over |= s < carry;
            if (j < e0) cum[j] = s;
            carry = __shfl_sync(0xffffffffu, s, 31);
        }
        if (__any_sync(0xffffffffu, over) && lane == 0) atomicOr(err, DEV_ERR_OVERFLOW);
        if (lane == 0) D[x] = carry;
    }
}

// Inclusive prefix over vertices of W1(v) = 2 d_v D(v) (u128): tile sums,
// one block scanning them, then each tile.
constexpr int CT = 1024;  // vertices per tile

__device__ __forceinline__ u128 w1_of(const DevGraph& G, const uint64_t* D, int64_t v) {
    const uint64_t d = (uint64_t)(__ldg(G.rowptr + v + 1) - __ldg(G.rowptr + v));
    return (u128)2 * (u128)d * (u128)D[v];
}

__device__ __forceinline__ u128 shfl_up_u128(u128 x, int o) {
    const uint64_t lo = __shfl_up_sync(0xffffffffu, (uint64_t)x, o);
    const uint64_t hi = __shfl_up_sync(0xffffffffu, (uint64_t)(x >> 64), o);
    return ((u128)hi << 64) | lo;
}

// Block-inclusive scan of u128 (1024 threads).
__device__ __forceinline__ u128 block_scan_u128(u128 x, u128* warp_sum) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const u128 y = shfl_up_u128(x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sum[wid] = x;
    __syncthreads();
    if (wid == 0) {
        u128 t = warp_sum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const u128 y = shfl_up_u128(t, o);
            if (lane >= o) t += y;
        }
        warp_sum[lane] = t;
    }
    __syncthreads();
    const u128 r = x + (wid > 0 ? warp_sum[wid - 1] : (u128)0);
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(CT) k_ws_tile_sums(DevGraph G, const uint64_t* __restrict__ D,
                                                     u128* __restrict__ tsum) {
    __shared__ u128 ws[32];
    const int64_t v = (int64_t)blockIdx.x * CT + threadIdx.x;
    const u128 x = v < G.n ? w1_of(G, D, v) : (u128)0;
    const u128 inc = block_scan_u128(x, ws);
    if (threadIdx.x == CT - 1) tsum[blockIdx.x] = inc;
}

__global__ void __launch_bounds__(CT) k_ws_scan_tiles(u128* __restrict__ tsum, int64_t tiles) {
    __shared__ u128 ws[32];
    __shared__ u128 carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t b = 0; b < tiles; b += CT) {
        const int64_t i = b + threadIdx.x;
        const u128 x = i < tiles ? tsum[i] : (u128)0;
        const u128 inc = block_scan_u128(x, ws);
        if (i < tiles) tsum[i] = carry + inc - x;  // exclusive
        __syncthreads();
        if (threadIdx.x == CT - 1) carry += inc;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(CT) k_ws_apply(DevGraph G, const uint64_t* __restrict__ D,
                                                 const u128* __restrict__ toff, u128* __restrict__ C1) {
    __shared__ u128 ws[32];
    const int64_t v = (int64_t)blockIdx.x * CT + threadIdx.x;
    const u128 x = v < G.n ? w1_of(G, D, v) : (u128)0;
    const u128 inc = block_scan_u128(x, ws);
    if (v < G.n) C1[v] = toff[blockIdx.x] + inc;
}

struct WsDraw {
    int32_t a;
    int64_t jb, jc;  // positions in a's weight-sorted row
};

// The draw of sample s (see the header).
template <int P>
__device__ __forceinline__ WsDraw ws_draw(const DevGraph& G, const uint64_t* __restrict__ cum,
                                          const uint64_t* __restrict__ D, const u128* __restrict__ C1,
                                          int64_t s, uint64_t seed) {
    uint64_t x[4];
    philox4((uint64_t)s, seed, 1ull, x);
    const u128 Z1 = C1[G.n - 1];
    const u128 t1 = mulhi_z(x[0], Z1);
    int64_t lo = 0, hi = G.n - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (C1[mid] > t1) hi = mid;
        else lo = mid + 1;
    }
    WsDraw r;
    r.a = (int32_t)lo;
    const int64_t b0 = __ldg(G.rowptr + lo);
    const uint64_t da = (uint64_t)(__ldg(G.rowptr + lo + 1) - b0);
    const u128 Da = D[lo];
    const u128 dD = (u128)da * Da;
    const u128 t2 = mulhi_z(x[1], 2 * dD);
    if (t2 < dD) {
        const uint64_t tp = (uint64_t)(t2 / da);
        int64_t l2 = 0, h2 = (int64_t)da - 1;
        while (l2 < h2) {
            const int64_t mid = (l2 + h2) >> 1;
            if (cum[b0 + mid] > tp) h2 = mid;
            else l2 = mid + 1;
        }
        r.jb = l2;
    } else {
        r.jb = (int64_t)((t2 - dD) / Da);
    }
    const u128 wab = wpow<P>(__ldg(G.wwt + b0 + r.jb));
    const u128 t3 = mulhi_z(x[2], Da + (u128)da * wab);
    if (t3 < Da) {
        const uint64_t tc = (uint64_t)t3;
        int64_t l2 = 0, h2 = (int64_t)da - 1;
        while (l2 < h2) {
            const int64_t mid = (l2 + h2) >> 1;
            if (cum[b0 + mid] > tc) h2 = mid;
            else l2 = mid + 1;
        }
        r.jc = l2;
    } else {
        r.jc = (int64_t)((t3 - Da) / wab);
    }
    return r;
}

// The draws alone (host checks against the oracle): center, jb, jc and the
// closed triangle (sorted) or -1s.
template <int P>
__global__ void k_ws_draws(DevGraph G, const uint64_t* __restrict__ cum, const uint64_t* __restrict__ D,
                           const u128* __restrict__ C1, int64_t nsamples, uint64_t seed, int32_t* center,
                           int32_t* jb, int32_t* jc, int32_t* tri) {
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < nsamples;
         s += (int64_t)gridDim.x * blockDim.x) {
        const WsDraw r = ws_draw<P>(G, cum, D, C1, s, seed);
        center[s] = r.a;
        jb[s] = (int32_t)r.jb;
        jc[s] = (int32_t)r.jc;
        int32_t t0 = -1, t1 = -1, t2 = -1;
        if (r.jb != r.jc) {
            const int64_t b0 = __ldg(G.rowptr + r.a);
            const int32_t b = __ldg(G.wcol + b0 + r.jb), c = __ldg(G.wcol + b0 + r.jc);
            int32_t wbc, rbc;
            Tally tb;
            const int64_t db = __ldg(G.rowptr + b + 1) - __ldg(G.rowptr + b);
            if (probe_oriented(G, b, db, c, wbc, rbc, tb)) {
                t0 = r.a;
                t1 = b;
                t2 = c;
                sort3(t0, t1, t2);
            }
        }
        tri[3 * s] = t0;
        tri[3 * s + 1] = t1;
        tri[3 * s + 2] = t2;
    }
}

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z ^= z >> 33;
    z *= 0xff51afd7ed558ccdull;
    z ^= z >> 33;
    z *= 0xc4ceb9fe1a85ec53ull;
    z ^= z >> 33;
    return z;
}

// Draws, closure checks, and the set T: each closed triangle goes into the
// hash set once (keyed by its two smallest edge ranks) and, when new, into
// the query's candidate buffer with its ranking key.
template <int P>
__global__ void __launch_bounds__(WBLK) k_ws_collect(DevGraph G, Query q, const uint64_t* __restrict__ cum,
                                                     const uint64_t* __restrict__ D,
                                                     const u128* __restrict__ C1, int64_t nsamples,
                                                     uint64_t seed, unsigned long long* __restrict__ table,
                                                     uint64_t tmask) {
    for (int64_t s = (int64_t)blockIdx.x * WBLK + threadIdx.x; s < nsamples;
         s += (int64_t)gridDim.x * WBLK) {
        const WsDraw r = ws_draw<P>(G, cum, D, C1, s, seed);
        if (r.jb == r.jc) continue;
        const int64_t b0 = __ldg(G.rowptr + r.a);
        const int32_t b = __ldg(G.wcol + b0 + r.jb), c = __ldg(G.wcol + b0 + r.jc);
        int32_t wbc, rbc;
        Tally tb;
        const int64_t db = __ldg(G.rowptr + b + 1) - __ldg(G.rowptr + b);
        if (!probe_oriented(G, b, db, c, wbc, rbc, tb)) continue;
        const int32_t wab = __ldg(G.wwt + b0 + r.jb), wac = __ldg(G.wwt + b0 + r.jc);
        int32_t r1 = __ldg(G.wrk + b0 + r.jb), r2 = __ldg(G.wrk + b0 + r.jc), r3 = rbc;
        sort3(r1, r2, r3);
        const unsigned long long hk = ((unsigned long long)(uint32_t)r1 << 32) | (uint32_t)r2;
        uint64_t h = mix64(hk) & tmask;
        bool fresh = false;
        for (;;) {  // at most nsamples keys in at least 2 nsamples slots: a free slot exists
            const unsigned long long old = atomicCAS(table + h, HASH_EMPTY, hk);
            if (old == HASH_EMPTY) {
                fresh = true;
                break;
            }
            if (old == hk) break;
            h = (h + 1) & tmask;
        }
        if (!fresh) continue;
        const unsigned long long key = keyof<P>((uint32_t)wab, (uint32_t)wac, (uint32_t)wbc);
        int32_t a = r.a, bb = b, cc = c;
        sort3(a, bb, cc);
        const uint32_t idx = atomicAdd(&q.st->count, 1u);
        if (idx < q.cap) {
            q.ckey[idx] = key;
            q.ctri[idx] = make_int4(a, bb, cc, 0);
        } else {
            atomicOr(&q.st->err, DEV_ERR_OVERFLOW);
        }
    }
}

// Scratch of one wedge-sampling call.
struct WsScratch {
    uint64_t* cum;   // 2m
    uint64_t* D;     // n
    u128* C1;        // n
    u128* tsum;      // tiles
    uint32_t* err;
};

template <int P>
int ws_prepare(const wtri_graph* g, const WsScratch& W, cudaStream_t s) {
    const DevGraph& G = g->d;
    const int64_t tiles = (G.n + CT - 1) / CT;
    ProfScope ps("wedge_tables", s, 0.0, 4, 8.0 * (double)G.m * 2 + 40.0 * (double)G.n);
    k_ws_rows<P><<<sm_count() * 16, WBLK, 0, s>>>(G, W.cum, W.D, W.err);
    k_ws_tile_sums<<<(unsigned)tiles, CT, 0, s>>>(G, W.D, W.tsum);
    k_ws_scan_tiles<<<1, CT, 0, s>>>(W.tsum, tiles);
    k_ws_apply<<<(unsigned)tiles, CT, 0, s>>>(G, W.D, W.tsum, W.C1);
    WTRI_CUDA(cudaGetLastError());
    return WTRI_OK;
}

size_t ws_bytes(const wtri_graph* g) {
    const int64_t n = g->d.n, m = g->d.m, tiles = (n + CT - 1) / CT;
    return 16 * (size_t)m + 8 * (size_t)n + 16 * (size_t)n + 16 * (size_t)tiles + 4 * 256;
}

WsScratch ws_carve(const wtri_graph* g, char* p) {
    const int64_t n = g->d.n, m = g->d.m, tiles = (n + CT - 1) / CT;
    WsScratch W;
    W.C1 = (u128*)p;  // 16-byte aligned first
    p += 16 * (size_t)n;
    W.tsum = (u128*)p;
    p += 16 * (size_t)tiles;
    W.cum = (uint64_t*)p;
    p += 16 * (size_t)m;
    W.D = (uint64_t*)p;
    p += 8 * (size_t)n;
    W.err = (uint32_t*)(((uintptr_t)p + 255) & ~(uintptr_t)255);
    return W;
}

template <int P>
int run_wedge_draws(const wtri_graph* g, int64_t nsamples, uint64_t seed, int32_t* hc, int32_t* hjb,
                    int32_t* hjc, int32_t* htri) {
    cudaStream_t s = g->stream;
    const size_t wsb = ws_bytes(g) + 512;
    const size_t ob = 24 * (size_t)nsamples + 64;
    void* buf = nullptr;
    if (cudaMallocAsync(&buf, wsb + ob, s) != cudaSuccess) {
        cudaGetLastError();
        return set_error(WTRI_ENOMEM, "wedge sampling scratch allocation failed");
    }
    WsScratch W = ws_carve(g, (char*)buf);
    WTRI_CUDA(cudaMemsetAsync(W.err, 0, 4, s));
    int32_t* dc = (int32_t*)((char*)buf + wsb);
    int32_t* djb = dc + nsamples;
    int32_t* djc = djb + nsamples;
    int32_t* dtri = djc + nsamples;
    int rc = ws_prepare<P>(g, W, s);
    if (rc == WTRI_OK) {
        k_ws_draws<P><<<sm_count() * 8, 256, 0, s>>>(g->d, W.cum, W.D, W.C1, nsamples, seed, dc, djb, djc,
                                                     dtri);
        count_launches(1);
        uint32_t herr = 0;
        cudaError_t e = cudaMemcpyAsync(&herr, W.err, 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hc, dc, 4 * (size_t)nsamples, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hjb, djb, 4 * (size_t)nsamples, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hjc, djc, 4 * (size_t)nsamples, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(htri, dtri, 12 * (size_t)nsamples, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = cuda_error(e, "wedge draws", __FILE__, __LINE__);
        else if (herr) rc = set_error(WTRI_EUNSUPPORTED, "a row's sum of w^p does not fit 64 bits");
    }
    cudaFreeAsync(buf, s);
    return rc;
}

template <int P>
int run_wedge_topk(const wtri_graph* g, int32_t k, int64_t nsamples, uint64_t seed, wtri_tri* d_tris,
                   double* d_weight, int32_t* d_count, cudaStream_t s) {
    const DevGraph& G = g->d;
    uint64_t tcap = 1024;
    while (tcap < 2 * (uint64_t)nsamples) tcap <<= 1;
    const uint32_t cap = (uint32_t)std::min<int64_t>(std::max<int64_t>(nsamples, k), (int64_t(1) << 31) - 1);
    const size_t wsb = ws_bytes(g) + 512;
    const size_t qb = 256 + (size_t)cap * 24 + 256 + 16 * sizeof(LongItem);
    const size_t hb = 8 * (size_t)tcap;
    void* buf = nullptr;
    if (cudaMallocAsync(&buf, wsb + qb + hb, s) != cudaSuccess) {
        cudaGetLastError();
        return set_error(WTRI_ENOMEM, "wedge sampling scratch allocation failed");
    }
    char* p = (char*)buf;
    WsScratch W = ws_carve(g, p);
    p += wsb;
    Query q;
    q.st = (QState*)p;
    p += 256;
    q.ckey = (unsigned long long*)p;
    p += (size_t)cap * 8;
    q.ctri = (int4*)p;
    p += (size_t)cap * 16;
    p = (char*)(((uintptr_t)p + 255) & ~(uintptr_t)255);
    q.longs = (LongItem*)p;
    p += 16 * sizeof(LongItem);
    unsigned long long* table = (unsigned long long*)p;
    q.cap = cap;
    q.long_cap = 16;
    q.k = k;
    q.smark = nullptr;
    q.slist = nullptr;
    q.long_count = &q.st->long_count;
    q.qid = 0;
    q.shard = 0;
    q.nshards = 1;
    q.t_short = g->tune.t_short;
    q.qbytes = nullptr;
    q.gp = 0.0;
    q.fw = 0;
    q.wait_first = WAIT_LIMIT;
    WTRI_CUDA(cudaMemsetAsync(q.st, 0, sizeof(QState), s));
    WTRI_CUDA(cudaMemsetAsync(W.err, 0, 4, s));
    WTRI_CUDA(cudaMemsetAsync(table, 0xff, hb, s));
    ProfScope whole(P == P_ONE ? "wedge_p=1" : (P == P_TWO ? "wedge_p=2" : "wedge_p=0"), s, 0.0, 0);
    {
        const int rc = ws_prepare<P>(g, W, s);
        if (rc != WTRI_OK) {
            cudaFreeAsync(buf, s);
            return rc;
        }
    }
    {
        ProfScope ps("wedge_collect", s, 0.0, 1);
        k_ws_collect<P><<<sm_count() * 8, WBLK, 0, s>>>(G, q, W.cum, W.D, W.C1, nsamples, seed, table,
                                                       tcap - 1);
    }
    {
        ProfScope ps("topk_final", s, 0.0, 3);
        k_select<<<1, SBLK, 0, s>>>(q);
        k_final_select<<<1, SBLK, 0, s>>>(q);
        k_rank_scatter<P><<<ceil_div_u(std::max(k, 1), 8), 256, 0, s>>>(q, d_tris, d_weight, d_count,
                                                                        nullptr);
    }
    WTRI_CUDA(cudaGetLastError());
    // a row sum above 64 bits: report it through the status word
    uint32_t herr = 0;
    WTRI_CUDA(cudaMemcpyAsync(&herr, W.err, 4, cudaMemcpyDeviceToHost, s));
    WTRI_CUDA(cudaStreamSynchronize(s));
    cudaFreeAsync(buf, s);
    if (herr) return set_error(WTRI_EUNSUPPORTED, "a row's sum of w^p does not fit 64 bits");
    return WTRI_OK;
}

}  // namespace

int wedge_topk_device(const wtri_graph* g, int pcode, int32_t k, int64_t nsamples, uint64_t seed,
                      wtri_tri* d_tris, double* d_weight, int32_t* d_count, cudaStream_t s) {
    if (pcode == P_ONE) return run_wedge_topk<P_ONE>(g, k, nsamples, seed, d_tris, d_weight, d_count, s);
    if (pcode == P_GEO) return run_wedge_topk<P_GEO>(g, k, nsamples, seed, d_tris, d_weight, d_count, s);
    return run_wedge_topk<P_TWO>(g, k, nsamples, seed, d_tris, d_weight, d_count, s);
}

int wedge_draws_host(const wtri_graph* g, int pcode, int64_t nsamples, uint64_t seed, int32_t* center,
                     int32_t* jb, int32_t* jc, int32_t* tri) {
    if (pcode == P_ONE) return run_wedge_draws<P_ONE>(g, nsamples, seed, center, jb, jc, tri);
    if (pcode == P_GEO) return run_wedge_draws<P_GEO>(g, nsamples, seed, center, jb, jc, tri);
    return run_wedge_draws<P_TWO>(g, nsamples, seed, center, jb, jc, tri);
}

}  // namespace wtri
