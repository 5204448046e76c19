// Stable LSD radix sort passes (reduce-then-scan) over 16-byte records.
//
// A record is (key, v0, v1, v2), four 32-bit words.  One pass orders N
// records by the digit (key >> shift) & mask, stably, with digits of up to
// MAX_BITS bits.  The first pass of a sort reads its records through a
// Loader (a view of the source arrays, possibly a virtual stream such as
// "two adjacency entries per edge"); the last writes them through a Storer
// (the final arrays).  Passes in between read and write whole 16-byte
// records (one vector access each) and, beside every record, the next
// pass's digit as a 16-bit word, so the next histogram reads 2 bytes per
// record instead of the record.
//
//   Loader: static NARR, TILE_WORDS     source arrays copied per tile, words each
//           static REC_BYTES            bytes read per record
//           const void* tile_src(int a, int64_t tbase)
//           uint4 srec(const uint32_t* in, int li, int64_t tbase)   from a copied tile
//           uint4 grec(int64_t i)       from global memory
//           uint32_t key(int64_t i)     (first-pass histogram)
//           bool tma_ok()               sources 16-byte aligned
//   Storer: void store(int64_t p, const uint4& rec); double rec_bytes();
//           void prepare()          once per CTA before the first store
//
// Gating: every kernel of a pass first reads the device status word and
// returns at once if an earlier step reported an error, so a build needs no
// host round trip between its steps.  A pass may also be conditional on the
// largest key: with g.glo > 0 it runs only if some key has a bit at or above
// g.glo (bit length of *g.gwmax), which lets a sort over keys whose width is
// only known on the device launch the widest plan and skip the passes it
// does not need.
//
// Three kernels per pass: per-chunk digit histograms (upsweep), a per-digit
// scan over chunks, and the scatter.  The scatter streams its chunk tile by
// tile; the next tile's sources arrive by bulk asynchronous copies
// (cp.async.bulk, one mbarrier per half of a double buffer) while the
// current one is ranked (per-warp peer masks built by shared-memory
// atomicOr, per-warp counters; stable), staged in
// digit order in the same shared-memory buffer it was read from, and written
// out so that consecutive threads store consecutive positions of one
// digit's run.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>

#include "wtri_internal.cuh"

namespace wtri {
namespace radix {

constexpr int MAX_BITS = 10;               // widest digit of a pass
constexpr int MAX_BINS = 1 << MAX_BITS;
#ifndef WTRI_RADIX_NT
#define WTRI_RADIX_NT 256
#endif
constexpr int NT = WTRI_RADIX_NT;          // threads of the histogram and scatter CTAs
constexpr int NW = NT / 32;
// Ranking within a warp: peer masks built by shared-memory atomicOr, one
// word per (warp, digit) (1), or ballots over the digit's bits (0).
#ifndef WTRI_RANK_SMEM
#define WTRI_RANK_SMEM 1
#endif
#ifndef WTRI_RADIX_IT
#if WTRI_RANK_SMEM
#define WTRI_RADIX_IT (WTRI_RADIX_NT == 512 ? 9 : 21)  // tiles, counters, masks and staging fit 227 KB
#else
#define WTRI_RADIX_IT (WTRI_RADIX_NT == 512 ? 11 : 24)  // the tiles, counters and staging fit 227 KB
#endif
#endif
#ifndef WTRI_RADIX_CTAS
#define WTRI_RADIX_CTAS 1
#endif
constexpr int IT = WTRI_RADIX_IT;          // records per thread per tile
constexpr int TT = NT * IT;                // records per tile
constexpr int CTAS_PER_SM = WTRI_RADIX_CTAS;
constexpr int DPT = MAX_BINS / NT;         // digits owned by a thread in the tile scan
constexpr int UP_SPLIT = 8;                // histogram blocks per chunk
constexpr int UNT = 256;                   // threads of a histogram block
constexpr int UNW = UNT / 32;
constexpr uint32_t WAIT_LIMIT = 1u << 24;  // bounded mbarrier polling
static_assert(TT % 16 == 0, "tiles are whole 16-byte lines of every source array");
static_assert(DPT == 2 || DPT == 4, "a thread's digits are one 4- or 8-byte word of each warp's counters");

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Exclusive scan of one value per thread over an NTH-thread block (NTH <= 1024).
template <int NTH>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t x, uint32_t* warp_tot,
                                                         uint32_t* total) {
    constexpr int NWW = NTH / 32;
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
        uint32_t t = lane < NWW ? warp_tot[lane] : 0;
        uint32_t ti = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, ti, o);
            if (lane >= o) ti += y;
        }
        if (lane < NWW) warp_tot[lane] = ti - t;
        if (lane == NWW - 1) *total = ti;
    }
    __syncthreads();
    uint32_t r = warp_tot[w] + inc - x;
    __syncthreads();
    return r;
}

struct PassGeom {
    int64_t n;        // records
    int64_t chunk;    // records per chunk (whole tiles)
    int chunks;       // G
    int shift;
    int bins;         // 1 << digit bits
    int bits;
    uint32_t mask;
    const uint32_t* gerr;   // status word: nonzero -> skip (may be null)
    const int32_t* gwmax;   // largest key value (conditional passes; may be null)
    int glo;                // conditional pass: runs iff bit_length(*gwmax) > glo
};

__device__ __forceinline__ bool pass_closed(const PassGeom& g) {
    if (g.gerr && *(volatile const uint32_t*)g.gerr) return true;
    if (g.glo > 0 && g.gwmax) {
        const int32_t wm = *(volatile const int32_t*)g.gwmax;
        const int B = wm > 0 ? 32 - __clz(wm) : 0;
        if (g.glo >= B) return true;
    }
    return false;
}

// ---- histogram sources ------------------------------------------------------
template <class Loader>
struct KeyDigits {  // first pass: the loader's keys
    static constexpr bool PACKED = false;
    Loader ld;
    int shift;
    uint32_t mask;
    __device__ __forceinline__ uint32_t digit(int64_t i) const { return (ld.key(i) >> shift) & mask; }
};
struct StoredDigits {  // later passes: 16-bit digits written by the previous scatter
    static constexpr bool PACKED = true;
    const uint16_t* d;
    __device__ __forceinline__ uint32_t digit(int64_t i) const { return __ldg(d + i); }
};

// Digit histogram of each chunk.  UP_SPLIT blocks share a chunk (each a
// slice of it, a multiple of 8 records) and add their counts into the
// zeroed per-chunk histogram; each warp counts into its own shared copy.
// Stored digits are read eight at a time (one 16-byte load).
template <class Dig>
__global__ void __launch_bounds__(UNT) k_upsweep(Dig dg, PassGeom g, uint32_t* counts) {
    if (pass_closed(g)) return;
    __shared__ uint32_t hist[UNW][MAX_BINS];
    const int w = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < UNW * MAX_BINS; i += UNT) (&hist[0][0])[i] = 0;
    __syncthreads();
    uint32_t* h = hist[w];
    const int chunk = blockIdx.x / UP_SPLIT, part = blockIdx.x % UP_SPLIT;
    const int64_t cbeg = (int64_t)chunk * g.chunk;
    const int64_t cend = min(g.n, cbeg + g.chunk);
    const int64_t slice = ((g.chunk + UP_SPLIT - 1) / UP_SPLIT + 7) & ~int64_t(7);
    const int64_t beg = min(cend, cbeg + part * slice);
    const int64_t end = min(cend, beg + slice);
    int64_t i0 = beg;
    if constexpr (Dig::PACKED) {
        const int64_t nv = (end - beg) >> 3;  // whole groups of 8 (beg is a multiple of 8)
        const uint4* v = reinterpret_cast<const uint4*>(dg.d + beg);
        for (int64_t q = threadIdx.x; q < nv; q += UNT) {
            const uint4 x = __ldg(v + q);
            atomicAdd(&h[x.x & 0xffffu], 1u);
            atomicAdd(&h[x.x >> 16], 1u);
            atomicAdd(&h[x.y & 0xffffu], 1u);
            atomicAdd(&h[x.y >> 16], 1u);
            atomicAdd(&h[x.z & 0xffffu], 1u);
            atomicAdd(&h[x.z >> 16], 1u);
            atomicAdd(&h[x.w & 0xffffu], 1u);
            atomicAdd(&h[x.w >> 16], 1u);
        }
        i0 = beg + (nv << 3);
    } else {
        constexpr int U = 4;
        for (; i0 + (int64_t)U * UNT <= end; i0 += (int64_t)U * UNT) {
            uint32_t d[U];
#pragma unroll
            for (int u = 0; u < U; u++) d[u] = dg.digit(i0 + (int64_t)u * UNT + threadIdx.x);
#pragma unroll
            for (int u = 0; u < U; u++) atomicAdd(&h[d[u]], 1u);
        }
    }
    for (int64_t i = i0 + threadIdx.x; i < end; i += UNT) atomicAdd(&h[dg.digit(i)], 1u);
    __syncthreads();
    for (int d = threadIdx.x; d < g.bins; d += UNT) {
        uint32_t s = 0;
#pragma unroll
        for (int k = 0; k < UNW; k++) s += hist[k][d];
        if (s) atomicAdd(&counts[(int64_t)d * g.chunks + chunk], s);
    }
}

// Block d: exclusive scan of counts[d][0..G) in place; totals[d] = sum.
__global__ void __launch_bounds__(NT) k_digit_scan(uint32_t* counts, int chunks, uint32_t* totals,
                                                   PassGeom g) {
    if (pass_closed(g)) return;
    __shared__ uint32_t warp_tot[NW];
    __shared__ uint32_t tot;
    uint32_t* c = counts + (int64_t)blockIdx.x * chunks;
    uint32_t carry = 0;
    for (int base = 0; base < chunks; base += NT) {
        int i = base + threadIdx.x;
        uint32_t x = i < chunks ? c[i] : 0;
        uint32_t ex = block_exclusive_scan<NT>(x, warp_tot, &tot);
        if (i < chunks) c[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) totals[blockIdx.x] = carry;
}

// ---- scatter -----------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void bar_init(uint64_t* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void bar_expect(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}
#ifndef WTRI_RADIX_LOAD_HINT
#define WTRI_RADIX_LOAD_HINT 1
#endif
// Tile sources are read once: an evict-first L2 policy keeps them from
// displacing the partially written lines of the digit runs.
__device__ __forceinline__ uint64_t evict_first_policy() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                          uint64_t policy) {
#if WTRI_RADIX_LOAD_HINT
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(policy)
        : "memory");
#else
    (void)policy;
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
#endif
}
__device__ __forceinline__ bool bar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

struct ScatterSmem {
    uint4 buf[2][TT];              // a tile's sources, then its records in digit order
    uint16_t cnt[NW][MAX_BINS];    // per (warp, digit): count, then staging offset
#if WTRI_RANK_SMEM
    uint32_t match[NW][MAX_BINS];  // per (warp, digit): lanes of the current strip; zero between strips
#endif
    uint32_t delta[MAX_BINS];      // output position of a staged record = delta[d] + index
    uint32_t warp_tot[32];
    uint32_t total;
    int timed_out;
    uint64_t bar[2];
};

__device__ __forceinline__ uint32_t lo16(uint32_t x) { return x & 0xffffu; }

#ifndef WTRI_RANK_BALLOT
#define WTRI_RANK_BALLOT 1
#endif
#ifndef WTRI_PEERS_ALL_BITS
#define WTRI_PEERS_ALL_BITS 0
#endif
#ifndef WTRI_FULL_TILES
#define WTRI_FULL_TILES 0
#endif
// Lanes of the warp holding the same digit as this lane (digits of 'bits'
// bits; lanes with valid == false group only among themselves): one ballot
// per digit bit.
template <bool FULL>
__device__ __forceinline__ uint32_t digit_peers(uint32_t d, int bits, bool valid) {
#if WTRI_RANK_BALLOT
    uint32_t p = 0xffffffffu;  // a full tile: every lane holds a record
    if (!FULL) {
        const uint32_t vb = __ballot_sync(0xffffffffu, valid);
        p = valid ? vb : ~vb;
    }
#if WTRI_PEERS_ALL_BITS
    // digits are below 1 << bits, so the ballots of the bits above are all
    // zero and leave p unchanged: no per-bit test
    (void)bits;
#pragma unroll
    for (int k = 0; k < MAX_BITS; k++) {
        const bool bit = (d >> k) & 1u;
        const uint32_t b = __ballot_sync(0xffffffffu, bit);
        p &= bit ? b : ~b;
    }
#else
#pragma unroll
    for (int k = 0; k < MAX_BITS; k++) {
        if (k < bits) {
            const bool bit = (d >> k) & 1u;
            const uint32_t b = __ballot_sync(0xffffffffu, bit);
            p &= bit ? b : ~b;
        }
    }
#endif
    return p;
#else
    return __match_any_sync(0xffffffffu, valid ? d : 0xffffffffu);
#endif
}
__device__ __forceinline__ uint32_t hi16(uint32_t x) { return x >> 16; }

// A thread's DPT consecutive 16-bit counters as one 4- or 8-byte word.
__device__ __forceinline__ void load_counts(const uint16_t* p, uint32_t (&c)[DPT]) {
    if constexpr (DPT == 4) {
        const uint2 r = *reinterpret_cast<const uint2*>(p);
        c[0] = lo16(r.x);
        c[1] = hi16(r.x);
        c[2] = lo16(r.y);
        c[3] = hi16(r.y);
    } else {
        const uint32_t r = *reinterpret_cast<const uint32_t*>(p);
        c[0] = lo16(r);
        c[1] = hi16(r);
    }
}
__device__ __forceinline__ void store_counts(uint16_t* p, const uint32_t (&s)[DPT]) {
    if constexpr (DPT == 4) {
        *reinterpret_cast<uint2*>(p) = make_uint2(s[0] | (s[1] << 16), s[2] | (s[3] << 16));
    } else {
        *reinterpret_cast<uint32_t*>(p) = s[0] | (s[1] << 16);
    }
}

// Rank, stage and write one tile of tcount <= TT records held in registers.
// Item j of warp w, lane l is record w * 32 * IT + j * 32 + l of the tile;
// ranking strips in order and warps in order keeps equal digits stable.
// run[] holds this thread's digits' next output positions (digits
// threadIdx.x * DPT + i).
template <bool FULL, class Storer>
__device__ __forceinline__ void scatter_tile(const uint4 (&rec)[IT], int tcount, uint4* stage,
                                             const Storer& st, const PassGeom& g,
                                             uint32_t (&run)[DPT], ScatterSmem& S) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t lt = lanemask_lt();
    // 1. zero the counters of the used digits (16-byte words, 8 digits each)
    const int zw = (g.bins + 7) >> 3;  // at least one word, so digits 0..3 always start at zero
    for (int q = threadIdx.x; q < zw; q += NT) {
#pragma unroll
        for (int k = 0; k < NW; k++) reinterpret_cast<uint4*>(&S.cnt[k][0])[q] = make_uint4(0, 0, 0, 0);
    }
    __syncthreads();
    uint32_t rank[IT];
#if WTRI_RANK_SMEM
    // 2. rank within the warp, strip by strip: each lane sets its bit in its
    //    digit's mask word, reads the word back (its peers), and the lowest
    //    peer advances the digit's counter and clears the word
    uint32_t* mm = S.match[w];
#pragma unroll
    for (int j = 0; j < IT; j++) {
        const int li = w * 32 * IT + j * 32 + lane;
        const bool valid = FULL || li < tcount;
        const uint32_t d = (rec[j].x >> g.shift) & g.mask;
        if (valid) atomicOr(&mm[d], 1u << lane);
        __syncwarp();
        const uint32_t peers = valid ? mm[d] : 0u;
        const uint32_t b = valid ? (uint32_t)S.cnt[w][d] : 0u;
        rank[j] = b + __popc(peers & lt);
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) {
            S.cnt[w][d] = (uint16_t)(b + __popc(peers));
            mm[d] = 0u;
        }
        __syncwarp();
    }
#else
    // 2. rank within the warp: first every item's peers (ballots, independent
    //    across strips), then the running per-warp counters strip by strip
#pragma unroll
    for (int j = 0; j < IT; j++) {
        const int li = w * 32 * IT + j * 32 + lane;
        rank[j] = digit_peers<FULL>((rec[j].x >> g.shift) & g.mask, g.bits, FULL || li < tcount);
    }
#pragma unroll
    for (int j = 0; j < IT; j++) {
        const int li = w * 32 * IT + j * 32 + lane;
        const bool valid = FULL || li < tcount;
        const uint32_t d = (rec[j].x >> g.shift) & g.mask;
        const uint32_t peers = rank[j];
        const uint32_t b = valid ? (uint32_t)S.cnt[w][d] : 0u;
        rank[j] = b + __popc(peers & lt);
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) S.cnt[w][d] = (uint16_t)(b + __popc(peers));
        __syncwarp();
    }
#endif
    __syncthreads();
    // 3. per digit: offsets of each warp, tile start, output delta.  Thread t
    //    owns digits DPT t .. DPT t + DPT - 1: one word of each warp's counters.
    {
        const int d0 = threadIdx.x * DPT;
        const bool mine = d0 < g.bins;
        uint32_t tot[DPT];
#pragma unroll
        for (int i = 0; i < DPT; i++) tot[i] = 0;
        if (mine) {
#pragma unroll
            for (int k = 0; k < NW; k++) {
                uint32_t c[DPT];
                load_counts(&S.cnt[k][d0], c);
#pragma unroll
                for (int i = 0; i < DPT; i++) tot[i] += c[i];
            }
        }
        uint32_t sum = 0;
#pragma unroll
        for (int i = 0; i < DPT; i++) sum += tot[i];
        const uint32_t start = block_exclusive_scan<NT>(sum, S.warp_tot, &S.total);
        if (mine) {
            uint32_t s[DPT];
            s[0] = start;
#pragma unroll
            for (int i = 1; i < DPT; i++) s[i] = s[i - 1] + tot[i - 1];
#pragma unroll
            for (int i = 0; i < DPT; i++) {
                S.delta[d0 + i] = run[i] - s[i];
                run[i] += tot[i];
            }
#pragma unroll
            for (int k = 0; k < NW; k++) {
                uint32_t c[DPT];
                load_counts(&S.cnt[k][d0], c);
                store_counts(&S.cnt[k][d0], s);
#pragma unroll
                for (int i = 0; i < DPT; i++) s[i] += c[i];
            }
        }
    }
    __syncthreads();
    // 4. stage in digit order (the tile's sources were read by every thread
    //    before the barriers above)
#pragma unroll
    for (int j = 0; j < IT; j++) {
        const int li = w * 32 * IT + j * 32 + lane;
        if (FULL || li < tcount) {
            const uint32_t d = (rec[j].x >> g.shift) & g.mask;
            stage[rank[j] + S.cnt[w][d]] = rec[j];
        }
    }
    __syncthreads();
    // 5. write: consecutive threads, consecutive positions of one digit's run
#pragma unroll
    for (int i = 0; i < IT; i++) {
        const int p = i * NT + threadIdx.x;
        if (FULL || p < tcount) {
            const uint4 r = stage[p];
            const uint32_t d = (r.x >> g.shift) & g.mask;
            st.store((int64_t)S.delta[d] + p, r);
        }
    }
    // generic accesses to the buffer are ordered before the next bulk copy into it
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
}

// One CTA per chunk; whole tiles arrive by bulk copies when USE_BULK (sources
// 16-byte aligned), the last partial tile (and every tile otherwise) by plain
// loads.  Waits are bounded: on timeout the pass sets DEV_ERR_TIMEOUT, gives
// copies in flight a bounded chance to land and the CTA returns.
template <class Loader, class Storer, bool USE_BULK>
__global__ void __launch_bounds__(NT, CTAS_PER_SM) k_scatter(Loader ld, Storer st_in, PassGeom g,
                                                           const uint32_t* counts,
                                                           const uint32_t* totals, uint32_t* err) {
    if (pass_closed(g)) return;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    ScatterSmem& S = *reinterpret_cast<ScatterSmem*>(smem_raw);
    Storer st = st_in;
    st.prepare();
    uint32_t run[DPT];
    {   // global start of this chunk's records of each digit
        uint32_t t[DPT], sum = 0;
#pragma unroll
        for (int i = 0; i < DPT; i++) {
            const int d = threadIdx.x * DPT + i;
            t[i] = d < g.bins ? totals[d] : 0u;
            sum += t[i];
        }
        uint32_t base = block_exclusive_scan<NT>(sum, S.warp_tot, &S.total);
#pragma unroll
        for (int i = 0; i < DPT; i++) {
            const int d = threadIdx.x * DPT + i;
            run[i] = d < g.bins ? base + counts[(int64_t)d * g.chunks + blockIdx.x] : 0u;
            base += t[i];
        }
    }
    const int64_t beg = (int64_t)blockIdx.x * g.chunk;
    const int64_t end = min(g.n, beg + g.chunk);
    const int64_t nfull = USE_BULK && end > beg ? (end - beg) / TT : 0;
    constexpr uint32_t ARR_BYTES = Loader::TILE_WORDS * 4u;
    static_assert(Loader::NARR * Loader::TILE_WORDS <= 4 * TT, "a tile's sources fit one buffer");
#if WTRI_RANK_SMEM
    for (int t = threadIdx.x; t < NW * MAX_BINS; t += NT) (&S.match[0][0])[t] = 0u;
#endif
    if (threadIdx.x == 0) {
        bar_init(&S.bar[0]);
        bar_init(&S.bar[1]);
        S.timed_out = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const uint64_t policy = evict_first_policy();
    auto issue = [&](int64_t t, int b) {
        const int64_t tbase = beg + t * TT;
        bar_expect(&S.bar[b], ARR_BYTES * Loader::NARR);
        uint32_t* dst = reinterpret_cast<uint32_t*>(&S.buf[b][0]);
#pragma unroll
        for (int a = 0; a < Loader::NARR; a++)
            bulk_load(dst + (size_t)a * TT, ld.tile_src(a, tbase), ARR_BYTES, &S.bar[b], policy);
    };
    if (threadIdx.x == 0 && nfull > 0) issue(0, 0);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int64_t t = 0; t < nfull; t++) {
        const int b = (int)(t & 1);
        // the other buffer was last used by tile t-1, released at its closing barrier
        if (threadIdx.x == 0 && t + 1 < nfull) issue(t + 1, b ^ 1);
        const uint32_t parity = (uint32_t)((t >> 1) & 1);
        uint32_t spins = 0;
        while (!bar_try_wait(&S.bar[b], parity)) {
            if (++spins >= WAIT_LIMIT) {
                S.timed_out = 1;
                break;
            }
        }
        __syncthreads();
        if (S.timed_out) {
            if (threadIdx.x == 0) atomicOr(err, DEV_ERR_TIMEOUT);
            for (int bb = 0; bb < 2; bb++) {
                uint32_t s2 = 0;
                while (!bar_try_wait(&S.bar[bb], parity) && ++s2 < WAIT_LIMIT) {
                }
            }
            return;
        }
        const int64_t tbase = beg + t * TT;
        const uint32_t* in = reinterpret_cast<const uint32_t*>(&S.buf[b][0]);
        uint4 rec[IT];
#pragma unroll
        for (int j = 0; j < IT; j++) rec[j] = ld.srec(in, w * 32 * IT + j * 32 + lane, tbase);
        scatter_tile<WTRI_FULL_TILES != 0>(rec, TT, &S.buf[b][0], st, g, run, S);
    }
    for (int64_t tbase = beg + nfull * TT; tbase < end; tbase += TT) {
        const int tcount = (int)min((int64_t)TT, end - tbase);
        uint4 rec[IT];
#pragma unroll
        for (int j = 0; j < IT; j++) {
            const int li = w * 32 * IT + j * 32 + lane;
            rec[j] = li < tcount ? ld.grec(tbase + li) : make_uint4(0, 0, 0, 0);
        }
        scatter_tile<false>(rec, tcount, &S.buf[0][0], st, g, run, S);
    }
}

// ---- intermediate records -----------------------------------------------------
struct AosLoader {
    static constexpr double REC_BYTES = 16.0;
    static constexpr int NARR = 1;
    static constexpr uint32_t TILE_WORDS = 4 * TT;
    const uint4* r;
    __device__ __forceinline__ uint32_t key(int64_t i) const { return __ldg(&r[i].x); }
    __device__ __forceinline__ const void* tile_src(int, int64_t tbase) const { return r + tbase; }
    __device__ __forceinline__ uint4 srec(const uint32_t* in, int li, int64_t) const {
        return reinterpret_cast<const uint4*>(in)[li];
    }
    __device__ __forceinline__ uint4 grec(int64_t i) const { return __ldg(r + i); }
    bool tma_ok() const { return ((uintptr_t)r & 15) == 0; }
};

struct AosStorer {
    uint4* r;
    uint16_t* dig;  // next pass's digit of each record
    int next_shift;
    uint32_t next_mask;
    __host__ __device__ double rec_bytes() const { return 18.0; }
    __device__ __forceinline__ void prepare() {}
    __device__ __forceinline__ void store(int64_t p, const uint4& x) const {
        r[p] = x;
        dig[p] = (uint16_t)((x.x >> next_shift) & next_mask);
    }
};

// A pass whose output is either the final arrays or the next pass's records:
// final iff the following pass is skipped (see PassGeom::glo), decided once
// per CTA from the device-side key width.
template <class Final>
struct SwitchStorer {
    Final fin;
    AosStorer mid;
    const int32_t* gwmax;
    int next_lo;   // lowest key bit of the following pass
    bool is_final;
    __host__ __device__ double rec_bytes() const { return mid.rec_bytes(); }
    __device__ __forceinline__ void prepare() {
        const int32_t wm = *(volatile const int32_t*)gwmax;
        const int B = wm > 0 ? 32 - __clz(wm) : 0;
        is_final = next_lo >= B;
    }
    __device__ __forceinline__ void store(int64_t p, const uint4& x) const {
        if (is_final) fin.store(p, x);
        else mid.store(p, x);
    }
};

// ---- host side ------------------------------------------------------------------
// Chunking: CTAS_PER_SM chunks per SM at most, each a whole number of tiles.
inline PassGeom make_geom(int64_t n, int shift, int bits) {
    PassGeom g;
    g.n = n;
    const int64_t tiles = (n + TT - 1) / TT;
    int64_t want = (int64_t)sm_count() * CTAS_PER_SM;
    if (want > tiles) want = tiles;
    if (want < 1) want = 1;
    const int64_t tiles_per = (tiles + want - 1) / want;
    g.chunk = tiles_per * TT;
    g.chunks = (int)((n + g.chunk - 1) / g.chunk);
    if (g.chunks < 1) g.chunks = 1;
    g.shift = shift;
    g.bins = 1 << bits;
    g.bits = bits;
    g.mask = (uint32_t)g.bins - 1u;
    g.gerr = nullptr;
    g.gwmax = nullptr;
    g.glo = 0;
    return g;
}

// Scratch for counts: MAX_BINS * chunks + MAX_BINS (uint32).
inline size_t scratch_words(int64_t n) {
    PassGeom g = make_geom(n, 0, MAX_BITS);
    return (size_t)MAX_BINS * g.chunks + MAX_BINS;
}

// Whether whole tiles use bulk copies (WTRI_RADIX_TMA=0 turns them off).
inline bool bulk_enabled() {
    static int v = -1;
    if (v < 0) {
        const char* e = getenv("WTRI_RADIX_TMA");
        v = (e && e[0] == '0') ? 0 : 1;
    }
    return v == 1;
}

// Digit widths of a sort over 'bits' key bits: as few passes as MAX_BITS
// allows, bits spread evenly (e.g. 26 -> 9, 9, 8; 20 -> 10, 10).
inline int pass_count(int bits) { return (bits + MAX_BITS - 1) / MAX_BITS; }
inline int pass_bits(int bits, int p) {
    const int passes = pass_count(bits);
    return bits / passes + (p < bits % passes ? 1 : 0);
}
inline int pass_shift(int bits, int p) {
    int s = 0;
    for (int q = 0; q < p; q++) s += pass_bits(bits, q);
    return s;
}

// alg_bytes: this pass's share of the sort's algorithmic bytes (the
// scatter's phase timer; histograms and scans declare none).  expected:
// whether the pass is expected to run (a conditional pass that the widest
// expected keys skip declares no moved bytes either).
template <class Dig, class Loader, class Storer>
int run_pass(const Dig& dg, const Loader& ld, const Storer& st, const PassGeom& g, uint32_t* scratch,
             cudaStream_t s, uint32_t* err, double hist_bytes, double alg_bytes, bool expected = true) {
    const double mv = expected ? 1.0 : 0.0;
    if (g.n <= 0) return WTRI_OK;
    uint32_t* counts = scratch;
    uint32_t* totals = scratch + (size_t)MAX_BINS * g.chunks;
    {
        ProfScope ps("radix_upsweep", s, 0.0, 1, mv * (hist_bytes * (double)g.n + 4.0 * g.bins * g.chunks));
        WTRI_CUDA(cudaMemsetAsync(counts, 0, sizeof(uint32_t) * (size_t)g.bins * g.chunks, s));
        k_upsweep<Dig><<<g.chunks * UP_SPLIT, UNT, 0, s>>>(dg, g, counts);
    }
    {
        ProfScope ps("radix_digit_scan", s, 0.0, 1, mv * 8.0 * g.bins * g.chunks);
        k_digit_scan<<<g.bins, NT, 0, s>>>(counts, g.chunks, totals, g);
    }
    const size_t smem = sizeof(ScatterSmem);
    ProfScope ps("radix_downsweep", s, alg_bytes, 1, mv * (double)g.n * (Loader::REC_BYTES + st.rec_bytes()));
    if (bulk_enabled() && ld.tma_ok()) {
        static std::atomic<uint64_t> done{0};  // per instantiation and device
        WTRI_TRY(smem_optin((const void*)k_scatter<Loader, Storer, true>, (int)smem, done));
        k_scatter<Loader, Storer, true><<<g.chunks, NT, smem, s>>>(ld, st, g, counts, totals, err);
    } else {
        static std::atomic<uint64_t> done{0};
        WTRI_TRY(smem_optin((const void*)k_scatter<Loader, Storer, false>, (int)smem, done));
        k_scatter<Loader, Storer, false><<<g.chunks, NT, smem, s>>>(ld, st, g, counts, totals, err);
    }
    WTRI_CUDA(cudaGetLastError());
    return WTRI_OK;
}

// Full stable LSD sort of n records over 'bits' key bits: first pass from
// 'first', middle passes through the 16-byte record buffers rec_a / rec_b
// (n records each) with digits in 'dig' (n 16-bit words), last pass into
// 'last'.  alg_total: the sort's algorithmic bytes (one read and one write
// of its payload), spread evenly over its passes' scatters.  Every kernel
// returns at once while *err is nonzero.
template <class First, class Last>
int lsd_sort(const First& first, const Last& last, int64_t n, int bits, uint4* rec_a, uint4* rec_b,
             uint16_t* dig, uint32_t* scratch, cudaStream_t s, uint32_t* err, double alg_total) {
    const int passes = pass_count(bits);
    if (passes == 0) return set_error(WTRI_EINVAL, "internal: zero-pass sort");
    const double alg = alg_total / passes;
    uint4* cur = rec_a;
    uint4* nxt = rec_b;
    for (int p = 0; p < passes; p++) {
        PassGeom g = make_geom(n, pass_shift(bits, p), pass_bits(bits, p));
        g.gerr = err;
        AosStorer as{nxt, dig, 0, 0u};
        if (p + 1 < passes) {
            as.next_shift = pass_shift(bits, p + 1);
            as.next_mask = (1u << pass_bits(bits, p + 1)) - 1u;
        }
        AosLoader al{cur};
        StoredDigits sd{dig};
        if (p == 0) {
            KeyDigits<First> kd{first, g.shift, g.mask};
            if (passes == 1) {
                WTRI_TRY(run_pass(kd, first, last, g, scratch, s, err, 4.0, alg));
            } else {
                WTRI_TRY(run_pass(kd, first, as, g, scratch, s, err, 4.0, alg));
            }
        } else if (p == passes - 1) {
            WTRI_TRY(run_pass(sd, al, last, g, scratch, s, err, 2.0, alg));
        } else {
            WTRI_TRY(run_pass(sd, al, as, g, scratch, s, err, 2.0, alg));
        }
        if (p + 1 < passes) std::swap(cur, nxt);
    }
    return WTRI_OK;
}

// The same sort for keys whose width is known only on the device: the key's
// largest value is *wmax (written by an earlier kernel on the stream).  The
// plan covers max_bits in digits of MAX_BITS (pass p: bits [10p, 10p+10));
// pass p > 0 runs only if a key has a bit at or above 10p, and each pass
// writes the final arrays when the next one will not run.  alg_total is
// spread over the passes the widest keys need (the phase timers see what
// runs).
template <class First, class Last>
int lsd_sort_device_width(const First& first, const Last& last, int64_t n, int max_bits,
                          const int32_t* wmax, uint4* rec_a, uint4* rec_b, uint16_t* dig,
                          uint32_t* scratch, cudaStream_t s, uint32_t* err, double alg_total,
                          int expected_passes) {
    const int passes = (max_bits + MAX_BITS - 1) / MAX_BITS;
    const double alg = alg_total / std::max(1, expected_passes);
    uint4* cur = rec_a;
    uint4* nxt = rec_b;
    for (int p = 0; p < passes; p++) {
        const int shift = p * MAX_BITS;
        const int bits = std::min(MAX_BITS, max_bits - shift);
        PassGeom g = make_geom(n, shift, bits);
        g.gerr = err;
        g.gwmax = wmax;
        g.glo = shift;  // pass 0 always runs (glo = 0)
        AosStorer as{nxt, dig, 0, 0u};
        if (p + 1 < passes) {
            as.next_shift = shift + MAX_BITS;
            as.next_mask = (1u << std::min(MAX_BITS, max_bits - shift - MAX_BITS)) - 1u;
        }
        SwitchStorer<Last> sw{last, as, wmax, shift + MAX_BITS, false};
        AosLoader al{cur};
        StoredDigits sd{dig};
        const bool ex = p < expected_passes;
        const double a = ex ? alg : 0.0;
        if (p == 0) {
            KeyDigits<First> kd{first, g.shift, g.mask};
            if (passes == 1) {
                WTRI_TRY(run_pass(kd, first, last, g, scratch, s, err, 4.0, a, ex));
            } else {
                WTRI_TRY(run_pass(kd, first, sw, g, scratch, s, err, 4.0, a, ex));
            }
        } else if (p == passes - 1) {
            WTRI_TRY(run_pass(sd, al, last, g, scratch, s, err, 2.0, a, ex));
        } else {
            WTRI_TRY(run_pass(sd, al, sw, g, scratch, s, err, 2.0, a, ex));
        }
        std::swap(cur, nxt);
    }
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
