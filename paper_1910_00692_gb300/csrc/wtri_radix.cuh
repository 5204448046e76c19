// Stable LSD radix sort passes (reduce-then-scan), 8-bit digits.
//
// One pass orders N records by digit (key >> shift) & mask, stably, where a
// record is a 32-bit key plus NV 32-bit values.  Records come from a Loader
// and go to a Storer, so a pass can read a virtual stream (e.g. two
// adjacency entries per edge) and write final arrays without staging copies.
//
//   Loader: __device__ uint32_t key(int64_t i) const;
//           __device__ uint32_t val(int q, int64_t i) const;   // q < NV
//   Storer: __device__ void key(int64_t pos, uint32_t k) const;
//           __device__ void val(int q, int64_t pos, uint32_t x) const;
//
// Three kernels per pass: per-chunk digit histograms (upsweep), a per-digit
// scan over chunks, and the scatter (downsweep).  Within a tile the scatter
// ranks records with warp match + per-warp counters (stable), stages them in
// shared memory in digit order, and writes each digit's run contiguously.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>

#include "wtri_internal.cuh"

namespace wtri {
namespace radix {

constexpr int BITS = 8;
constexpr int RADIX = 1 << BITS;
constexpr int THREADS = 256;
constexpr int WARPS = THREADS / 32;
constexpr int ITEMS = 12;
constexpr int TILE = THREADS * ITEMS;
static_assert(THREADS == RADIX, "one thread per digit in the tile scan");

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Exclusive scan of one value per thread over a 256-thread block.
__device__ __forceinline__ uint32_t block_exclusive_scan_256(uint32_t x, uint32_t* warp_tot,
                                                             uint32_t* total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_tot[w] = inc;
    __syncthreads();
    if (w == 0) {
        uint32_t t = lane < WARPS ? warp_tot[lane] : 0;
        uint32_t ti = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, ti, o);
            if (lane >= o) ti += y;
        }
        if (lane < WARPS) warp_tot[lane] = ti - t;
        if (lane == WARPS - 1) *total = ti;
    }
    __syncthreads();
    uint32_t r = warp_tot[w] + inc - x;
    __syncthreads();
    return r;
}

// Exclusive scan of one value per thread over an NT-thread block (NT <= 1024).
template <int NT>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t x, uint32_t* warp_tot,
                                                         uint32_t* total) {
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_tot[w] = inc;
    __syncthreads();
    if (w == 0) {
        uint32_t t = lane < NW ? warp_tot[lane] : 0;
        uint32_t ti = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, ti, o);
            if (lane >= o) ti += y;
        }
        if (lane < NW) warp_tot[lane] = ti - t;
        if (lane == NW - 1) *total = ti;
    }
    __syncthreads();
    uint32_t r = warp_tot[w] + inc - x;
    __syncthreads();
    return r;
}

struct PassGeom {
    int64_t n;        // records
    int64_t chunk;    // records per chunk (multiple of TILE)
    int chunks;       // G
    int shift;
    uint32_t mask;
};

// Digit histogram of each chunk.  UP_SPLIT blocks share a chunk (each a
// slice of it) and add their counts into the zeroed per-chunk histogram.
constexpr int UP_SPLIT = 8;

template <class Loader>
__global__ void __launch_bounds__(THREADS) k_upsweep(Loader ld, PassGeom g, uint32_t* counts) {
    __shared__ uint32_t hist[WARPS][RADIX];
    const int w = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < WARPS * RADIX; i += THREADS) (&hist[0][0])[i] = 0;
    __syncthreads();
    const int chunk = blockIdx.x / UP_SPLIT, part = blockIdx.x % UP_SPLIT;
    const int64_t cbeg = (int64_t)chunk * g.chunk;
    const int64_t cend = min(g.n, cbeg + g.chunk);
    const int64_t slice = (g.chunk + UP_SPLIT - 1) / UP_SPLIT;
    const int64_t beg = cbeg + part * slice;
    const int64_t end = min(cend, beg + slice);
    for (int64_t i = beg + threadIdx.x; i < end; i += THREADS) {
        uint32_t d = (ld.key(i) >> g.shift) & g.mask;
        atomicAdd(&hist[w][d], 1u);
    }
    __syncthreads();
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < WARPS; k++) s += hist[k][threadIdx.x];
    if (s) atomicAdd(&counts[(int64_t)threadIdx.x * g.chunks + chunk], s);
}

// Block d: exclusive scan of counts[d][0..G) in place; totals[d] = sum.
__global__ void __launch_bounds__(THREADS) k_digit_scan(uint32_t* counts, int chunks,
                                                        uint32_t* totals) {
    __shared__ uint32_t warp_tot[WARPS];
    __shared__ uint32_t tot;
    uint32_t* c = counts + (int64_t)blockIdx.x * chunks;
    uint32_t carry = 0;
    for (int base = 0; base < chunks; base += THREADS) {
        int i = base + threadIdx.x;
        uint32_t x = i < chunks ? c[i] : 0;
        uint32_t ex = block_exclusive_scan_256(x, warp_tot, &tot);
        if (i < chunks) c[i] = carry + ex;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) totals[blockIdx.x] = carry;
}

template <int NV>
struct TileSmem {
    uint32_t cnt[WARPS][RADIX];
    uint32_t stage[NV + 1][TILE];  // key, then values, in tile-sorted order
    uint32_t run[RADIX];           // global position of this chunk's next record per digit
    uint32_t tile_start[RADIX];    // tile-local start of each digit
    uint32_t tile_total[RADIX];
    uint32_t warp_tot[WARPS];
    uint32_t total;
};

template <int NV, class Loader, class Storer, bool STORE_KEY>
__global__ void __launch_bounds__(THREADS) k_downsweep(Loader ld, Storer st, PassGeom g,
                                                       const uint32_t* counts,
                                                       const uint32_t* totals) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TileSmem<NV>& S = *reinterpret_cast<TileSmem<NV>*>(smem_raw);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;

    {   // global base of each digit = exclusive scan of digit totals
        uint32_t t = totals[threadIdx.x];
        uint32_t base = block_exclusive_scan_256(t, S.warp_tot, &S.total);
        S.run[threadIdx.x] = base + counts[(int64_t)threadIdx.x * g.chunks + blockIdx.x];
    }
    __syncthreads();

    const int64_t beg = (int64_t)blockIdx.x * g.chunk;
    const int64_t end = min(g.n, beg + g.chunk);
    const uint32_t lt = lanemask_lt();

    for (int64_t tbase = beg; tbase < end; tbase += TILE) {
        const int tcount = (int)min((int64_t)TILE, end - tbase);
        for (int i = threadIdx.x; i < WARPS * RADIX; i += THREADS) (&S.cnt[0][0])[i] = 0;

        // Every load of the tile is issued before any use (one round trip).
        uint32_t key[ITEMS];
        uint32_t val[NV > 0 ? NV : 1][ITEMS];
        uint32_t rank[ITEMS];
#pragma unroll
        for (int j = 0; j < ITEMS; j++) {
            const int li = w * 32 * ITEMS + j * 32 + lane;
            const bool valid = li < tcount;
            key[j] = valid ? ld.key(tbase + li) : 0u;
#pragma unroll
            for (int q = 0; q < NV; q++) val[q][j] = valid ? ld.val(q, tbase + li) : 0u;
        }
        __syncthreads();  // counters cleared
#pragma unroll
        for (int j = 0; j < ITEMS; j++) {
            const int li = w * 32 * ITEMS + j * 32 + lane;
            const bool valid = li < tcount;
            const uint32_t d = valid ? ((key[j] >> g.shift) & g.mask) : (uint32_t)RADIX;
            const uint32_t peers = __match_any_sync(0xffffffffu, d);
            uint32_t base = valid ? S.cnt[w][d] : 0u;
            rank[j] = base + __popc(peers & lt);
            __syncwarp();
            if (valid && (__ffs(peers) - 1) == lane) S.cnt[w][d] = base + __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        {   // per digit: warp offsets, tile totals, tile starts
            const int d = threadIdx.x;
            uint32_t s = 0;
#pragma unroll
            for (int k = 0; k < WARPS; k++) {
                uint32_t c = S.cnt[k][d];
                S.cnt[k][d] = s;
                s += c;
            }
            S.tile_total[d] = s;
            uint32_t st0 = block_exclusive_scan_256(s, S.warp_tot, &S.total);
            S.tile_start[d] = st0;
#pragma unroll
            for (int k = 0; k < WARPS; k++) S.cnt[k][d] += st0;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < ITEMS; j++) {
            const int li = w * 32 * ITEMS + j * 32 + lane;
            if (li < tcount) {
                const uint32_t d = (key[j] >> g.shift) & g.mask;
                const uint32_t pos = rank[j] + S.cnt[w][d];
                S.stage[0][pos] = key[j];
#pragma unroll
                for (int q = 0; q < NV; q++) S.stage[q + 1][pos] = val[q][j];
            }
        }
        __syncthreads();
        // Consecutive threads write consecutive positions of one digit's run.
#pragma unroll
        for (int i = 0; i < ITEMS; i++) {
            const int p = i * THREADS + threadIdx.x;
            if (p < tcount) {
                const uint32_t k = S.stage[0][p];
                const uint32_t d = (k >> g.shift) & g.mask;
                const int64_t gp = (int64_t)S.run[d] + (p - (int64_t)S.tile_start[d]);
                if (STORE_KEY) st.key(gp, k);
#pragma unroll
                for (int q = 0; q < NV; q++) st.val(q, gp, S.stage[q + 1][p]);
            }
        }
        __syncthreads();
        S.run[threadIdx.x] += S.tile_total[threadIdx.x];
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// TMA-fed scatter.  One CTA per SM streams its chunk tile by tile; while a
// tile is ranked and scattered, the next tile's source arrays arrive in the
// other half of a double buffer by bulk async copies (cp.async.bulk) that
// complete on one mbarrier per buffer.  Waits are bounded: on timeout the
// pass records DEV_ERR_TIMEOUT and the CTA returns.  Only whole tiles go
// through TMA; a chunk's last partial tile is loaded with plain loads.
// ---------------------------------------------------------------------------
constexpr int TMA_ARRS = 4;                 // source arrays per loader, at most
constexpr uint32_t TMA_WAIT_LIMIT = 1u << 24;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void tma_bar_init(uint64_t* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void tma_expect(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ bool tma_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// One CTA per SM with full 3,072-record tiles: on the mid build this beat
// half tiles at two CTAs per SM (3.40 vs 4.16 ms) and 512-thread CTAs (3.57
// ms), longer per-digit write runs mattering more than overlap.
constexpr int TMA_THREADS = 256;
constexpr int TMA_WARPS = TMA_THREADS / 32;
constexpr int TMA_ITEMS = 12;
constexpr int TT = TMA_THREADS * TMA_ITEMS;  // records per TMA tile
constexpr int TMA_CTAS_PER_SM = 1;
static_assert(TILE % TT == 0, "chunks of whole plain tiles are whole TMA tiles");

constexpr int RANK_GROUPS = 1;  // counter sets per warp (4 independent groups measured slower: 3.61 vs 3.29 ms)

template <int NV>
struct TmaSmem {
    uint32_t in[2][TMA_ARRS][TT];  // source arrays of the current / next tile
    uint4 stage4[TT];              // (key, values) of each record in digit order
    uint32_t cnt[TMA_WARPS][RANK_GROUPS][RADIX];
    uint32_t run[RADIX];
    uint32_t tile_start[RADIX];
    uint32_t tile_total[RADIX];
    uint32_t warp_tot[32];
    uint32_t total;
    int timed_out;
    uint64_t bar[2];
};

// Records of the current tile from the TMA buffer.
template <class Loader>
struct SmemSrc {
    const Loader& ld;
    const uint32_t* in;  // in[b][0]; array a at in + a * TILE
    int64_t tbase;
    __device__ __forceinline__ uint32_t key(int li) const { return ld.skey(in, li, tbase); }
    __device__ __forceinline__ uint32_t val(int q, int li) const { return ld.sval(in, q, li, tbase); }
};

// Records of a tile straight from global memory.
template <class Loader>
struct GlobalSrc {
    const Loader& ld;
    int64_t tbase;
    __device__ __forceinline__ uint32_t key(int li) const { return ld.key(tbase + li); }
    __device__ __forceinline__ uint32_t val(int q, int li) const { return ld.val(q, tbase + li); }
};

// Rank, stage and scatter one tile of tcount <= TL records (all NT threads).
// A warp's items are ranked in RANK_GROUPS groups of consecutive item
// indices, each with its own digit counters, so the groups' match/count
// chains are independent; the per-digit scan over (warp, group) in order
// keeps the ranking stable.
template <int NT, int TL, int NV, bool STORE_KEY, class Src, class Storer, class Smem>
__device__ __forceinline__ void scatter_tile(const Src& src, const Storer& st, const PassGeom& g,
                                             int tcount, Smem& S) {
    constexpr int NW = NT / 32, IT = TL / NT, NG = RANK_GROUPS, PER = IT / NG;
    static_assert(PER * NG == IT, "items split evenly into groups");
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t lt = lanemask_lt();
    for (int i = threadIdx.x; i < NW * NG * RADIX; i += NT) (&S.cnt[0][0][0])[i] = 0;
    __syncthreads();
    uint32_t key[IT];
    uint32_t rank[IT];
#pragma unroll
    for (int j = 0; j < IT; j++) {
        const int li = w * 32 * IT + j * 32 + lane;
        key[j] = li < tcount ? src.key(li) : 0u;
    }
#pragma unroll
    for (int t = 0; t < PER; t++) {
        uint32_t dd[NG], pp[NG], bb[NG];
#pragma unroll
        for (int gi = 0; gi < NG; gi++) {
            const int j = gi * PER + t;
            const int li = w * 32 * IT + j * 32 + lane;
            const bool valid = li < tcount;
            dd[gi] = valid ? ((key[j] >> g.shift) & g.mask) : (uint32_t)RADIX;
            pp[gi] = __match_any_sync(0xffffffffu, dd[gi]);
            bb[gi] = valid ? S.cnt[w][gi][dd[gi]] : 0u;
            rank[j] = bb[gi] + __popc(pp[gi] & lt);
        }
        __syncwarp();
#pragma unroll
        for (int gi = 0; gi < NG; gi++)
            if (dd[gi] < (uint32_t)RADIX && (__ffs(pp[gi]) - 1) == lane)
                S.cnt[w][gi][dd[gi]] = bb[gi] + __popc(pp[gi]);
        __syncwarp();
    }
    __syncthreads();
    {   // per digit (first RADIX threads): offsets of (warp, group), tile totals and starts
        const int d = threadIdx.x;
        uint32_t s = 0;
        if (d < RADIX) {
#pragma unroll
            for (int k = 0; k < NW; k++)
#pragma unroll
                for (int gi = 0; gi < NG; gi++) {
                    uint32_t c = S.cnt[k][gi][d];
                    S.cnt[k][gi][d] = s;
                    s += c;
                }
            S.tile_total[d] = s;
        }
        const uint32_t st0 = block_exclusive_scan<NT>(d < RADIX ? s : 0u, S.warp_tot, &S.total);
        if (d < RADIX) {
            S.tile_start[d] = st0;
#pragma unroll
            for (int k = 0; k < NW; k++)
#pragma unroll
                for (int gi = 0; gi < NG; gi++) S.cnt[k][gi][d] += st0;
        }
    }
    __syncthreads();
    static_assert(NV <= 3, "a record (key + values) is staged as one 16-byte word");
#pragma unroll
    for (int j = 0; j < IT; j++) {
        const int li = w * 32 * IT + j * 32 + lane;
        if (li < tcount) {
            const uint32_t d = (key[j] >> g.shift) & g.mask;
            const uint32_t pos = rank[j] + S.cnt[w][j / PER][d];
            uint4 rec;
            rec.x = key[j];
            rec.y = NV > 0 ? src.val(0, li) : 0u;
            rec.z = NV > 1 ? src.val(1, li) : 0u;
            rec.w = NV > 2 ? src.val(2, li) : 0u;
            S.stage4[pos] = rec;  // one 16-byte store per record
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < IT; i++) {
        const int p = i * NT + threadIdx.x;
        if (p < tcount) {
            const uint4 rec = S.stage4[p];
            const uint32_t d = (rec.x >> g.shift) & g.mask;
            const int64_t gp = (int64_t)S.run[d] + (p - (int64_t)S.tile_start[d]);
            if (STORE_KEY) st.key(gp, rec.x);
            if (NV > 0) st.val(0, gp, rec.y);
            if (NV > 1) st.val(1, gp, rec.z);
            if (NV > 2) st.val(2, gp, rec.w);
        }
    }
    __syncthreads();
    if (threadIdx.x < RADIX) S.run[threadIdx.x] += S.tile_total[threadIdx.x];
    __syncthreads();
}

template <int NV, class Loader, class Storer, bool STORE_KEY>
__global__ void __launch_bounds__(TMA_THREADS, TMA_CTAS_PER_SM) k_downsweep_tma(Loader ld, Storer st, PassGeom g,
                                                               const uint32_t* counts,
                                                               const uint32_t* totals, uint32_t* err) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    TmaSmem<NV>& S = *reinterpret_cast<TmaSmem<NV>*>(smem_raw);
    {
        const int d = threadIdx.x;
        const uint32_t t = d < RADIX ? totals[d] : 0u;
        const uint32_t base = block_exclusive_scan<TMA_THREADS>(t, S.warp_tot, &S.total);
        if (d < RADIX) S.run[d] = base + counts[(int64_t)d * g.chunks + blockIdx.x];
    }
    const int64_t beg = (int64_t)blockIdx.x * g.chunk;
    const int64_t end = min(g.n, beg + g.chunk);
    const int64_t nfull = end > beg ? (end - beg) / TT : 0;
    const uint32_t arr_bytes = Loader::TILE_ELEMS * 4u;
    if (threadIdx.x == 0) {
        tma_bar_init(&S.bar[0]);
        tma_bar_init(&S.bar[1]);
        S.timed_out = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    auto issue = [&](int64_t t, int b) {
        const int64_t tbase = beg + t * TT;
        tma_expect(&S.bar[b], arr_bytes * Loader::NARR);
#pragma unroll
        for (int a = 0; a < Loader::NARR; a++)
            tma_load_1d(&S.in[b][a][0], ld.tile_src(a, tbase), arr_bytes, &S.bar[b]);
    };
    if (threadIdx.x == 0 && nfull > 0) issue(0, 0);
    for (int64_t t = 0; t < nfull; t++) {
        const int b = (int)(t & 1);
        if (threadIdx.x == 0 && t + 1 < nfull) {
            // the other buffer was last read by tile t-1, finished at its
            // closing barrier; order those reads before the async writes
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(t + 1, b ^ 1);
        }
        const uint32_t parity = (uint32_t)((t >> 1) & 1);
        uint32_t spins = 0;
        while (!tma_try_wait(&S.bar[b], parity)) {
            if (++spins >= TMA_WAIT_LIMIT) {
                S.timed_out = 1;
                break;
            }
        }
        __syncthreads();
        if (S.timed_out) {
            if (threadIdx.x == 0) atomicOr(err, DEV_ERR_TIMEOUT);
            // give copies still in flight a bounded chance to land
            for (int bb = 0; bb < 2; bb++) {
                uint32_t s2 = 0;
                while (!tma_try_wait(&S.bar[bb], parity) && ++s2 < TMA_WAIT_LIMIT) {
                }
            }
            return;
        }
        SmemSrc<Loader> src{ld, &S.in[b][0][0], beg + t * TT};
        scatter_tile<TMA_THREADS, TT, NV, STORE_KEY>(src, st, g, TT, S);
    }
    const int64_t tail = beg + nfull * TT;
    if (tail < end) {
        GlobalSrc<Loader> src{ld, tail};
        scatter_tile<TMA_THREADS, TT, NV, STORE_KEY>(src, st, g, (int)(end - tail), S);
    }
}

// Record arrays (ping-pong buffers between passes).
template <int NV>
struct ArrLoader {
    static constexpr double KEY_BYTES = 4.0;
    static constexpr double REC_BYTES = 4.0 * (1 + NV);
    static constexpr int NARR = 1 + NV;
    static constexpr uint32_t TILE_ELEMS = TT;
    const uint32_t* k;
    const uint32_t* v[NV > 0 ? NV : 1];
    __device__ __forceinline__ uint32_t key(int64_t i) const { return __ldg(k + i); }
    __device__ __forceinline__ uint32_t val(int q, int64_t i) const { return __ldg(v[q] + i); }
    __device__ __forceinline__ const void* tile_src(int a, int64_t tbase) const {
        return (a == 0 ? k : v[a - 1]) + tbase;
    }
    __device__ __forceinline__ uint32_t skey(const uint32_t* in, int li, int64_t) const { return in[li]; }
    __device__ __forceinline__ uint32_t sval(const uint32_t* in, int q, int li, int64_t) const {
        return in[(q + 1) * TT + li];
    }
    bool tma_ok() const {
        bool ok = ((uintptr_t)k & 15) == 0;
        for (int q = 0; q < NV; q++) ok = ok && ((uintptr_t)v[q] & 15) == 0;
        return ok;
    }
};

template <int NV>
struct ArrStorer {
    __host__ __device__ double rec_bytes() const { return 4.0 * (1 + NV); }
    uint32_t* k;
    uint32_t* v[NV > 0 ? NV : 1];
    __device__ __forceinline__ void key(int64_t p, uint32_t x) const { k[p] = x; }
    __device__ __forceinline__ void val(int q, int64_t p, uint32_t x) const { v[q][p] = x; }
};

// Chunks per SM.  Each chunk keeps one partially written line per digit and
// output array in L2 while it streams, so the chunk count is kept small
// enough that those write fronts fit in L2 (WTRI_RADIX_CHUNKS_PER_SM
// overrides the default of 2 for tuning).
inline int chunks_per_sm() {
    static int v = 0;
    if (v == 0) {
        const char* e = getenv("WTRI_RADIX_CHUNKS_PER_SM");
        int x = e ? atoi(e) : 0;
        v = (x >= 1 && x <= 64) ? x : 2;
    }
    return v;
}

// Chunking: enough chunks to fill the GPU, each a whole number of tiles.
inline PassGeom make_geom(int64_t n, int shift, int bits, int per_sm = 0) {
    PassGeom g;
    g.n = n;
    const int64_t tiles = (n + TILE - 1) / TILE;
    int64_t want = (int64_t)sm_count() * (per_sm > 0 ? per_sm : chunks_per_sm());
    if (want > tiles) want = tiles;
    if (want < 1) want = 1;
    const int64_t tiles_per = (tiles + want - 1) / want;
    g.chunk = tiles_per * TILE;
    g.chunks = (int)((n + g.chunk - 1) / g.chunk);
    if (g.chunks < 1) g.chunks = 1;
    g.shift = shift;
    g.mask = (bits >= 32) ? 0xffffffffu : ((1u << bits) - 1u);
    return g;
}

template <int NV>
inline size_t downsweep_smem() {
    return sizeof(TileSmem<NV>);
}

// Scratch for counts: RADIX * chunks + RADIX totals (uint32).
inline size_t scratch_words(int64_t n) {
    PassGeom g = make_geom(n, 0, BITS);
    return (size_t)RADIX * g.chunks + RADIX;
}

// One pass.  'scratch' holds scratch_words(n) uint32 (device).
// Whether the TMA-fed scatter is used (WTRI_RADIX_TMA=0 turns it off).
inline bool tma_enabled() {
    static int v = -1;
    if (v < 0) {
        const char* e = getenv("WTRI_RADIX_TMA");
        v = (e && e[0] == '0') ? 0 : 1;
    }
    return v == 1;
}

template <int NV, bool STORE_KEY, class Loader, class Storer>
int run_pass(const Loader& ld, const Storer& st, int64_t n, int shift, int bits,
             uint32_t* scratch, cudaStream_t s, uint32_t* err) {
    if (n <= 0) return WTRI_OK;
    const bool use_tma = tma_enabled() && err != nullptr && ld.tma_ok();
    PassGeom g = make_geom(n, shift, bits, use_tma ? TMA_CTAS_PER_SM : 0);
    uint32_t* counts = scratch;
    uint32_t* totals = scratch + (size_t)RADIX * g.chunks;
    {
        ProfScope ps("radix_upsweep", s, (double)n * Loader::KEY_BYTES + 4.0 * RADIX * g.chunks, 1);
        WTRI_CUDA(cudaMemsetAsync(counts, 0, sizeof(uint32_t) * RADIX * (size_t)g.chunks, s));
        k_upsweep<Loader><<<g.chunks * UP_SPLIT, THREADS, 0, s>>>(ld, g, counts);
    }
    {
        ProfScope ps("radix_digit_scan", s, 8.0 * RADIX * g.chunks, 1);
        k_digit_scan<<<RADIX, THREADS, 0, s>>>(counts, g.chunks, totals);
    }
    if (use_tma) {
        const size_t smem = sizeof(TmaSmem<NV>);
        static bool attr_tma = false;  // per instantiation; idempotent
        if (!attr_tma) {
            WTRI_CUDA(cudaFuncSetAttribute(k_downsweep_tma<NV, Loader, Storer, STORE_KEY>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            attr_tma = true;
        }
        ProfScope ps("radix_downsweep", s, (double)n * (Loader::REC_BYTES + st.rec_bytes()), 1);
        k_downsweep_tma<NV, Loader, Storer, STORE_KEY><<<g.chunks, TMA_THREADS, smem, s>>>(
            ld, st, g, counts, totals, err);
    } else {
        const size_t smem = downsweep_smem<NV>();
        static bool attr_set = false;  // per instantiation; idempotent
        if (!attr_set) {
            WTRI_CUDA(cudaFuncSetAttribute(k_downsweep<NV, Loader, Storer, STORE_KEY>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            attr_set = true;
        }
        ProfScope ps("radix_downsweep", s, (double)n * (Loader::REC_BYTES + st.rec_bytes()), 1);
        k_downsweep<NV, Loader, Storer, STORE_KEY><<<g.chunks, THREADS, smem, s>>>(ld, st, g, counts,
                                                                                  totals);
    }
    WTRI_CUDA(cudaGetLastError());
    return WTRI_OK;
}

inline int bit_length(uint64_t x) {
    int b = 0;
    while (x) {
        b++;
        x >>= 1;
    }
    return b;
}

}  // namespace radix
}  // namespace wtri
