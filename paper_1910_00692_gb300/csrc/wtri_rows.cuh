// The oriented rows of NodeIterator++ (Section 5.2), derived from the
// weight-sorted rows by a per-row segmented sort.
//
// Input: the weight-sorted rows (row x holds its neighbours in edge order at
// [rowptr[x], rowptr[x+1]) of wcol / wwt / wrk) and the row of each entry
// (wrow, build scratch).  Output, for every row x: the neighbours c of
// higher (degree, id) rank than x, ascending by id, at [orowptr[x],
// orowptr[x+1]) of ocol / owt / ork -- every edge once, under its
// lower-ranked endpoint, the lists the closing-edge lookups search (N(a) of
// Section 4, split by the orientation).  A neighbour twice in one row is a
// repeated pair, an invalid input (Section 1: a simple graph); both copies
// of a pair land in the same oriented row, so the sort finds every repeat.
//
// k_fwd decides the orientation of every entry at once and packs each
// forward entry's key (id << 32 | position in the weight-sorted row) into
// the first odeg[x] slots of its row's range in scratch (unordered: one
// atomic per row and warp).  A scan of odeg gives orowptr.  Rows are then
// sorted by their oriented degree d, on 64-bit keys (id << 32 | index of the
// key among the row's packed keys), unique within a row:
//   d <= 32           sub-warp bitonic network in registers (groups of 8, 16
//                     or 32 lanes, several rows per warp);
//   32 < d <= 512     one warp per row: bitonic network over 2..16 keys per
//                     lane in registers, transposed through shared memory;
//   512 < d           one block per row: stable LSD radix sort of the ids in
//                     shared memory (digits of at most 9 bits, ranked by warp
//                     ballots), slices of at most SR keys; rows above SR
//                     leave their sorted slices in global scratch, where one
//                     launch per merge level (many blocks, one row each)
//                     merges pairs of runs until the row is one run.
// A bitonic network spends log d (log d + 1) / 2 compare-exchange stages
// on every key, the radix sort a fixed number of passes (3 for 26-bit ids):
// the network wins on short rows, the radix sort from a few hundred keys.
// A vertex with d forward neighbours has d neighbours of degree >= d, so
// d <= sqrt(2m): the oriented rows are short even where the full rows are
// not.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "wtri_internal.cuh"

namespace wtri {
namespace rows {

constexpr int NT = 256;           // block kernels
constexpr int NWARPS = NT / 32;
constexpr int WMAX = 512;         // longest row sorted by one warp
constexpr int SR = 4096;          // longest slice a block radix-sorts in shared memory

// Size classes of a row (by oriented degree d): three sub-warp classes, four
// warp classes by keys per lane (2, 4, 8, 16), block rows, hub rows (> SR).
enum : int {
    CLS_NONE = 0, CLS_G8, CLS_G16, CLS_G32,
    CLS_W2, CLS_W4, CLS_W8, CLS_W16,
    CLS_BLOCK, CLS_HUB
};
constexpr int NCLS = 10;

__device__ __forceinline__ int row_class(int64_t d) {
    if (d <= 0) return CLS_NONE;
    if (d <= 8) return CLS_G8;
    if (d <= 16) return CLS_G16;
    if (d <= 32) return CLS_G32;
    if (d <= 64) return CLS_W2;
    if (d <= 128) return CLS_W4;
    if (d <= 256) return CLS_W8;
    if (d <= WMAX) return CLS_W16;
    if (d <= SR) return CLS_BLOCK;
    return CLS_HUB;
}

// Whether x (degree dx) comes before its neighbour c in the (degree, id)
// order.  The degrees saturated to 16 bits (a 2-byte-per-vertex table that
// mostly stays in L2) decide unless both saturate; then the exact degree of
// c comes from the row offsets.
constexpr uint32_t DEG_SAT = 65535;

// dc16: deg16[c], gathered by the caller.
__device__ __forceinline__ bool rank_before(int32_t x, int64_t dx, uint32_t dc16,
                                            const int64_t* __restrict__ rowptr, int32_t c) {
    uint64_t dc = dc16;
    if (dx >= DEG_SAT) {
        if (dc < DEG_SAT) return false;
        dc = (uint64_t)(__ldg(rowptr + c + 1) - __ldg(rowptr + c));
    }
    return (uint64_t)dx < dc || ((uint64_t)dx == dc && x < c);
}

struct RowsOut {
    const int64_t* rowptr;
    const int32_t* wwt;
    const int32_t* wrk;
    const unsigned long long* pk;    // packed forward keys, row x at [rowptr[x], rowptr[x] + odeg[x])
    const int32_t* odeg;             // oriented out-degrees
    const int64_t* orowptr;          // oriented row offsets
    int32_t* ocol;
    int32_t* owt;
    int32_t* ork;
    uint32_t* err;                   // build status: error bits
    unsigned long long* first_dup;   // smallest repeated pair, x << 32 | c
    const int32_t* list;             // rows of each class, class c at [cls_off[c], cls_off[c+1])
    const int32_t* cls_off;
};

// Gate of the row kernels: an earlier step failed.  A repeated pair found by
// another row kernel does not close it, so that every size class still runs
// and the smallest repeated entry is reported whatever the launch order.
__device__ __forceinline__ bool rows_gate_closed(const uint32_t* gate) {
    return (*(volatile const uint32_t*)gate & ~(uint32_t)DEV_ERR_DUPLICATE) != 0;
}

__device__ __forceinline__ void flag_dup(const RowsOut& R, int32_t x, int32_t c) {
    atomicOr(R.err, DEV_ERR_DUPLICATE);
    atomicMin(R.first_dup, ((unsigned long long)(uint32_t)x << 32) | (uint32_t)c);
}

// ---------------------------------------------------------------------------
// Row classes by oriented degree: counts, then the list of rows of each class.
// ---------------------------------------------------------------------------
// A block step covers NT * CLS_V rows: CLS_V strips of 32 rows per warp.
constexpr int CLS_V = 8;

// The classes of one warp's CLS_V strips, and (in lane k, 0 < k < NCLS) how
// many of them are of class k.
__device__ __forceinline__ int class_strips(int32_t n, const int32_t* __restrict__ odeg, int64_t xw,
                                            int (&cls)[CLS_V]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int j = 0; j < CLS_V; j++) {
        const int64_t x = xw + j * 32 + lane;
        cls[j] = x < n ? row_class(__ldg(odeg + x)) : CLS_NONE;
    }
    int mine = 0;
#pragma unroll
    for (int k = 1; k < NCLS; k++) {
        int t = 0;
#pragma unroll
        for (int j = 0; j < CLS_V; j++) t += __popc(__ballot_sync(0xffffffffu, cls[j] == k));
        if (lane == k) mine = t;
    }
    return mine;
}

__global__ void __launch_bounds__(NT) k_class_count(int32_t n, const int32_t* __restrict__ odeg,
                                                    int32_t* __restrict__ cls_cnt, const uint32_t* gate) {
    if (rows_gate_closed(gate)) return;
    __shared__ int32_t sc[NCLS];
    if (threadIdx.x < NCLS) sc[threadIdx.x] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    int acc = 0;  // lane k: rows of class k seen by this warp
    const int64_t span = (int64_t)NT * CLS_V;
    for (int64_t x0 = (int64_t)blockIdx.x * span; x0 < n; x0 += (int64_t)gridDim.x * span) {
        int cls[CLS_V];
        acc += class_strips(n, odeg, x0 + (int64_t)wp * 32 * CLS_V, cls);
    }
    if (lane > 0 && lane < NCLS && acc) atomicAdd(&sc[lane], acc);
    __syncthreads();
    if (threadIdx.x > 0 && threadIdx.x < NCLS && sc[threadIdx.x]) atomicAdd(cls_cnt + threadIdx.x, sc[threadIdx.x]);
}

// cls_cnt (NCLS counts) -> cls_off (NCLS + 1 offsets); fill cursors in cls_cur.
__global__ void k_class_offsets(const int32_t* cls_cnt, int32_t* cls_off, int32_t* cls_cur,
                                const uint32_t* gate) {
    if (rows_gate_closed(gate)) return;
    if (threadIdx.x == 0) {
        int32_t acc = 0;
        for (int c = 0; c < NCLS; c++) {
            cls_off[c] = acc;
            cls_cur[c] = acc;
            acc += (c == CLS_NONE) ? 0 : cls_cnt[c];
        }
        cls_off[NCLS] = acc;
    }
}

// Rows of each class into list[]: per block step, each warp's count of
// each class goes to shared memory, one global atomic per class reserves the
// block's slots, and each warp writes its rows at its offset in them.
__global__ void __launch_bounds__(NT) k_class_fill(int32_t n, const int32_t* __restrict__ odeg,
                                                   int32_t* __restrict__ cls_cur, int32_t* __restrict__ list,
                                                   const uint32_t* gate) {
    if (rows_gate_closed(gate)) return;
    constexpr int NWP = NT / 32;
    __shared__ int32_t woff[NWP][NCLS];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    const int64_t span = (int64_t)NT * CLS_V;
    for (int64_t x0 = (int64_t)blockIdx.x * span; x0 < n; x0 += (int64_t)gridDim.x * span) {
        const int64_t xw = x0 + (int64_t)wp * 32 * CLS_V;
        int cls[CLS_V];
        const int mine = class_strips(n, odeg, xw, cls);
        if (lane < NCLS) woff[wp][lane] = mine;
        __syncthreads();
        if (threadIdx.x > 0 && threadIdx.x < NCLS) {  // class k: warps' offsets, then the block's slots
            const int k = threadIdx.x;
            int32_t tot = 0;
            for (int w = 0; w < NWP; w++) {
                const int32_t c = woff[w][k];
                woff[w][k] = tot;
                tot += c;
            }
            const int32_t base = tot ? atomicAdd(cls_cur + k, tot) : 0;
            for (int w = 0; w < NWP; w++) woff[w][k] += base;
        }
        __syncthreads();
#pragma unroll
        for (int k = 1; k < NCLS; k++) {
            int32_t off = woff[wp][k];
#pragma unroll
            for (int j = 0; j < CLS_V; j++) {
                const uint32_t b = __ballot_sync(0xffffffffu, cls[j] == k);
                if (cls[j] == k) list[off + __popc(b & lt)] = (int32_t)(xw + j * 32 + lane);
                off += __popc(b);
            }
        }
        __syncthreads();  // woff is rewritten by the next step
    }
}

// ---------------------------------------------------------------------------
// Orientation of every entry: entry e of row x is forward if its neighbour c
// ranks above x (NodeIterator++ keeps the edge in x's row).  odeg[x] counts
// them; each forward entry's key (c << 32 | e - rowptr[x]) goes to slot
// rowptr[x] + (its arrival index) of pk.  Rows are contiguous, so a warp
// takes one atomic per row it touches.
// ---------------------------------------------------------------------------
constexpr unsigned long long KEY_NONE = ~0ull;  // sorts after every real key

__device__ __forceinline__ int32_t key_col(unsigned long long k) { return (int32_t)(k >> 32); }
__device__ __forceinline__ uint32_t key_pos(unsigned long long k) { return (uint32_t)k & 0x7fffffffu; }
__device__ __forceinline__ unsigned long long with_pos(unsigned long long k, uint32_t i) {
    return (k & 0xffffffff00000000ull) | i;
}

__device__ __forceinline__ uint32_t lane_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

constexpr int FWD_U = 4;  // strips of 32 entries per warp and iteration (loads issued together)

__global__ void __launch_bounds__(NT) k_fwd(int64_t n2, const int32_t* __restrict__ wrow,
                                            const int32_t* __restrict__ wcol,
                                            const int64_t* __restrict__ rowptr,
                                            const uint16_t* __restrict__ deg16,
                                            unsigned long long* __restrict__ pk,
                                            int32_t* __restrict__ odeg, const uint32_t* gate) {
    if (rows_gate_closed(gate)) return;
    const int lane = threadIdx.x & 31;
    const uint32_t lt = lane_lt();
    const int64_t nwarps = ((int64_t)gridDim.x * NT) >> 5;
    for (int64_t base = (((int64_t)blockIdx.x * NT + threadIdx.x) >> 5) * (32 * FWD_U); base < n2;
         base += nwarps * (32 * FWD_U)) {
        int32_t x[FWD_U], c[FWD_U];
        int64_t s[FWD_U], dx[FWD_U];
        uint32_t dc[FWD_U];
#pragma unroll
        for (int u = 0; u < FWD_U; u++) {
            const int64_t e = base + u * 32 + lane;
            x[u] = e < n2 ? __ldcs(wrow + e) : -1;
            c[u] = e < n2 ? __ldcs(wcol + e) : 0;
        }
#pragma unroll
        for (int u = 0; u < FWD_U; u++) {
            s[u] = x[u] >= 0 ? __ldg(rowptr + x[u]) : 0;
            dx[u] = x[u] >= 0 ? __ldg(rowptr + x[u] + 1) - s[u] : 0;
            dc[u] = x[u] >= 0 ? __ldg(deg16 + c[u]) : 0u;
        }
        int32_t slot[FWD_U];
        uint32_t bits[FWD_U], seg[FWD_U];
        int hl[FWD_U];
#pragma unroll
        for (int u = 0; u < FWD_U; u++) {
            const bool valid = x[u] >= 0;
            const bool f = valid && rank_before(x[u], dx[u], dc[u], rowptr, c[u]);
            bits[u] = __ballot_sync(0xffffffffu, f);
            const int32_t xp = __shfl_up_sync(0xffffffffu, x[u], 1);
            const bool head = valid && (lane == 0 || xp != x[u]);
            const uint32_t heads = __ballot_sync(0xffffffffu, head);
            // the segment of lanes sharing this lane's row starts at its head
            hl[u] = valid ? 31 - __clz(heads & (lt | (1u << lane))) : lane;
            const uint32_t after = heads & ~((2u << hl[u]) - 1u);  // heads after the segment's
            const int end = after ? __ffs(after) - 1 : 32;
            seg[u] = (end >= 32 ? 0xffffffffu : ((1u << end) - 1u)) & ~((1u << hl[u]) - 1u);
            slot[u] = 0;
            if (head) {
                const int cnt = __popc(bits[u] & seg[u]);
                if (cnt) slot[u] = atomicAdd(odeg + x[u], cnt);
            }
        }
#pragma unroll
        for (int u = 0; u < FWD_U; u++) {
            const int32_t sl = __shfl_sync(0xffffffffu, slot[u], hl[u]);
            if ((bits[u] >> lane) & 1u) {
                const int64_t e = base + u * 32 + lane;
                __stcg(pk + s[u] + sl + __popc(bits[u] & seg[u] & lt),
                       ((unsigned long long)(uint32_t)c[u] << 32) | (uint32_t)(e - s[u]));
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Oriented entry p of row x.  Outputs are written once and not read again
// by this pass: streaming stores, so that they do not displace the rows the
// pass gathers from.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void write_orient(const RowsOut& R, int64_t p, int32_t c, int32_t w,
                                             int32_t rk) {
    __stcs(R.ocol + p, c);
    __stcs(R.owt + p, w);
    __stcs(R.ork + p, rk);
}

// Weight and rank of a packed key (position in the weight-sorted row s..).
__device__ __forceinline__ void gather_wr(const RowsOut& R, int64_t s, unsigned long long kk, int32_t& w,
                                          int32_t& rk) {
    const uint32_t j = key_pos(kk);
    w = __ldg(R.wwt + s + j);
    rk = __ldg(R.wrk + s + j);
}

// ---------------------------------------------------------------------------
// Rows of at most G entries (G = 8, 16, 32): G lanes per row, a bitonic
// network across the group's lanes.
// ---------------------------------------------------------------------------
constexpr int SMALL_U = 4;  // rows per lane group and iteration (their loads issued together)

template <int G>
__global__ void __launch_bounds__(NT) k_rows_small(RowsOut R, int cls, const uint32_t* gate) {
    if (rows_gate_closed(gate)) return;
    const int lane = threadIdx.x & 31, gl = lane & (G - 1), grp = lane / G;
    constexpr int RPW = 32 / G;  // rows per warp and unrolled step
    const int64_t lo = R.cls_off[cls], hi = R.cls_off[cls + 1];
    const int64_t nwarps = ((int64_t)gridDim.x * NT) >> 5;
    for (int64_t wbase = lo + (((int64_t)blockIdx.x * NT + threadIdx.x) >> 5) * (RPW * SMALL_U); wbase < hi;
         wbase += nwarps * (RPW * SMALL_U)) {
        int32_t x[SMALL_U], d[SMALL_U];
        int64_t s[SMALL_U], ob[SMALL_U];
#pragma unroll
        for (int u = 0; u < SMALL_U; u++) {
            const int64_t ri = wbase + u * RPW + grp;
            x[u] = ri < hi ? __ldg(R.list + ri) : -1;
        }
#pragma unroll
        for (int u = 0; u < SMALL_U; u++) {
            s[u] = 0;
            d[u] = 0;
            ob[u] = 0;
            if (x[u] >= 0) {
                s[u] = __ldg(R.rowptr + x[u]);
                d[u] = __ldg(R.odeg + x[u]);
                ob[u] = __ldg(R.orowptr + x[u]);
            }
        }
        unsigned long long key[SMALL_U];
#pragma unroll
        for (int u = 0; u < SMALL_U; u++) key[u] = gl < d[u] ? __ldcs(R.pk + s[u] + gl) : KEY_NONE;
        int32_t w[SMALL_U], rk[SMALL_U];
#pragma unroll
        for (int u = 0; u < SMALL_U; u++) {
            w[u] = 0;
            rk[u] = 0;
            if (gl < d[u]) {
                gather_wr(R, s[u], key[u], w[u], rk[u]);
                key[u] = with_pos(key[u], gl);
            }
        }
#pragma unroll
        for (int k = 2; k <= G; k <<= 1) {
#pragma unroll
            for (int j = k >> 1; j > 0; j >>= 1) {
                const bool up = (gl & k) == 0, lower = (gl & j) == 0;
#pragma unroll
                for (int u = 0; u < SMALL_U; u++) {
                    const unsigned long long ok = __shfl_xor_sync(0xffffffffu, key[u], j, G);
                    key[u] = (lower == up) ? (ok < key[u] ? ok : key[u]) : (ok > key[u] ? ok : key[u]);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < SMALL_U; u++) {
            const int src = (int)key_pos(key[u]) & (G - 1);
            const int32_t ws = __shfl_sync(0xffffffffu, w[u], src, G);
            const int32_t rks = __shfl_sync(0xffffffffu, rk[u], src, G);
            const unsigned long long prev = __shfl_up_sync(0xffffffffu, key[u], 1, G);
            if (gl < d[u]) {
                const int32_t c = key_col(key[u]);
                write_orient(R, ob[u] + gl, c, ws, rks);
                if (gl > 0 && key_col(prev) == c) flag_dup(R, x[u], c);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Bitonic network over the 32 * EPL keys of a warp, in registers: key i of
// lane l is element l * EPL + i.  Stages with a partner distance below EPL
// stay inside a lane; the others exchange with lane l ^ (distance / EPL).
// Sorts ascending; keys must be distinct (KEY_NONE padding may repeat).
// ---------------------------------------------------------------------------
// Intra-lane compare-exchange stage at partner distance J (< EPL) of a
// bitonic merge of blocks of `size` elements.
template <int EPL, int J>
__device__ __forceinline__ void bitonic_intra(unsigned long long (&k)[EPL], int lane, int size) {
#pragma unroll
    for (int i = 0; i < EPL; i++) {
        const int p = i ^ J;
        if (p > i) {
            const bool up = ((lane * EPL + i) & size) == 0;
            const unsigned long long a = k[i], b = k[p];
            if ((a > b) == up) {
                k[i] = b;
                k[p] = a;
            }
        }
    }
}

template <int EPL>
__device__ __forceinline__ void warp_bitonic(unsigned long long (&k)[EPL]) {
    // The stage loops stay rolled (a fully unrolled network of 32 keys per
    // lane is tens of thousands of instructions, far beyond the instruction
    // cache); the element loops are unrolled, so registers stay registers.
    const int lane = threadIdx.x & 31;
#pragma unroll 1
    for (int size = 2; size <= 32 * EPL; size <<= 1) {
#pragma unroll 1
        for (int j = size >> 1; j > 0; j >>= 1) {
            if (j >= EPL) {
                const int lm = j / EPL;
                const bool lower = (lane & lm) == 0;
#pragma unroll
                for (int i = 0; i < EPL; i++) {
                    const unsigned long long o = __shfl_xor_sync(0xffffffffu, k[i], lm);
                    const bool up = ((lane * EPL + i) & size) == 0;
                    const bool keep_min = lower == up;
                    k[i] = keep_min ? (o < k[i] ? o : k[i]) : (o > k[i] ? o : k[i]);
                }
            } else {
                switch (j) {
                    case 16: if constexpr (EPL > 16) bitonic_intra<EPL, 16>(k, lane, size); break;
                    case 8: if constexpr (EPL > 8) bitonic_intra<EPL, 8>(k, lane, size); break;
                    case 4: if constexpr (EPL > 4) bitonic_intra<EPL, 4>(k, lane, size); break;
                    case 2: if constexpr (EPL > 2) bitonic_intra<EPL, 2>(k, lane, size); break;
                    default: if constexpr (EPL > 1) bitonic_intra<EPL, 1>(k, lane, size); break;
                }
            }
        }
    }
}

// Shared-memory index of element p of a warp's sorted run (lane-blocked
// stores of 8-byte keys would all hit one bank: swizzle the low five bits).
__device__ __forceinline__ int swz(int p) { return p ^ ((p >> 5) & 31); }

// ---------------------------------------------------------------------------
// Rows of 33..512 entries: one warp per row, 32 * EPL keys in registers
// (EPL = 2, 4, 8, 16 by class), sorted, transposed through the warp's
// shared memory (keys, and the row's weights and ranks by packed index).
// ---------------------------------------------------------------------------
template <int EPL>
__global__ void __launch_bounds__(NT) k_rows_warp(RowsOut R, int cls, const uint32_t* gate) {
    if (rows_gate_closed(gate)) return;
    extern __shared__ __align__(16) unsigned long long wsm[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned long long* run = wsm + (size_t)wid * 2 * 32 * EPL;
    int32_t* wv = reinterpret_cast<int32_t*>(run + 32 * EPL);  // weights by packed index
    int32_t* rv = wv + 32 * EPL;                                 // ranks by packed index
    const int64_t lo = R.cls_off[cls], hi = R.cls_off[cls + 1];
    const int64_t nwarps = ((int64_t)gridDim.x * NT) >> 5;
    for (int64_t ri = lo + (((int64_t)blockIdx.x * NT + threadIdx.x) >> 5); ri < hi; ri += nwarps) {
        const int32_t x = __ldg(R.list + ri);
        const int64_t s = __ldg(R.rowptr + x);
        const int d = __ldg(R.odeg + x);
        const int64_t ob = __ldg(R.orowptr + x);
        unsigned long long k[EPL];
#pragma unroll
        for (int i = 0; i < EPL; i++) {
            const int j = i * 32 + lane;  // coalesced loads; the network ignores input order
            if (j < d) {
                const unsigned long long kk = __ldcs(R.pk + s + j);
                gather_wr(R, s, kk, wv[j], rv[j]);
                k[i] = with_pos(kk, j);
            } else {
                k[i] = KEY_NONE;
            }
        }
        warp_bitonic<EPL>(k);
#pragma unroll
        for (int i = 0; i < EPL; i++) run[swz(lane * EPL + i)] = k[i];
        __syncwarp();
        for (int j = lane; j < d; j += 32) {
            const unsigned long long kk = run[swz(j)];
            const int32_t c = key_col(kk);
            const uint32_t src = key_pos(kk);
            write_orient(R, ob + j, c, wv[src], rv[src]);
            if (j > 0 && key_col(run[swz(j - 1)]) == c) flag_dup(R, x, c);
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// Merge path: split point of the diagonal `diag` between sorted runs a
// (na keys) and b (nb keys): i keys come from a, diag - i from b.
// ---------------------------------------------------------------------------
template <class RA, class RB>
__device__ __forceinline__ int64_t merge_split(const RA& a, int64_t na, const RB& b, int64_t nb,
                                               int64_t diag) {
    int64_t lo = diag > nb ? diag - nb : 0, hi = diag < na ? diag : na;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (a(mid) < b(diag - 1 - mid)) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Merges `cnt` outputs starting at diagonal diag into out(q) for q = diag...
template <class RA, class RB, class WO>
__device__ __forceinline__ void merge_out(const RA& a, int64_t na, const RB& b, int64_t nb, int64_t diag,
                                          int cnt, const WO& out) {
    int64_t i = merge_split(a, na, b, nb, diag), j = diag - i;
    for (int t = 0; t < cnt; t++) {
        const bool take_a = j >= nb || (i < na && a(i) < b(j));
        const unsigned long long v = take_a ? a(i) : b(j);
        if (take_a) i++;
        else j++;
        out(diag + t, v);
    }
}

// ---------------------------------------------------------------------------
// Block radix sort of one slice (cnt <= SR keys) in shared memory: LSD over
// the id bits [32, 32 + nbits) of the keys, digits of at most RBITS bits,
// each pass stable.  Item j of warp w, lane l is key w * 32 * IT + j * 32 + l
// of the source buffer (IT keys per thread, IT * NT >= cnt); within a warp
// the items are ranked strip by strip (a ballot per digit bit gives the
// lanes of equal digit, a per-warp counter per digit the keys before), the
// warps in order by a scan of the per-(warp, digit) counts.
// ---------------------------------------------------------------------------
constexpr int RBITS = 9;
constexpr int RBINS = 1 << RBITS;
constexpr int RDPT = RBINS / NT;  // digits owned by a thread in the scan
static_assert(RDPT == 2, "a thread owns two digits: one 4-byte word of each warp's counters");

struct RadixSmem {
    unsigned long long key[2][SR];   // ping-pong key buffers
    int32_t wv[SR];                  // weights of the slice by packed index
    int32_t rv[SR];                  // ranks of the slice by packed index
    uint16_t cnt[NWARPS][RBINS];     // per (warp, digit): count, then output offset
    uint32_t warp_tot[32];
    uint32_t total;
    int32_t item;
};

__device__ __forceinline__ uint32_t block_scan_excl(uint32_t x, uint32_t* warp_tot) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_tot[w] = inc;
    __syncthreads();
    uint32_t before = 0;
#pragma unroll
    for (int k = 0; k < NWARPS; k++) before += k < w ? warp_tot[k] : 0u;
    __syncthreads();
    return before + inc - x;
}

// Lanes whose valid item has the same digit as this lane's (invalid lanes
// group among themselves).
__device__ __forceinline__ uint32_t radix_peers(uint32_t d, int bits, bool valid) {
    const uint32_t vb = __ballot_sync(0xffffffffu, valid);
    uint32_t p = valid ? vb : ~vb;
#pragma unroll
    for (int k = 0; k < RBITS; k++) {
        if (k < bits) {
            const bool bit = (d >> k) & 1u;
            const uint32_t b = __ballot_sync(0xffffffffu, bit);
            p &= bit ? b : ~b;
        }
    }
    return p;
}

template <int IT>
__device__ __forceinline__ void radix_pass(const unsigned long long* src, unsigned long long* dst, int cnt,
                                           int shift, int bits, RadixSmem& S) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t lt = lane_lt();
    const uint32_t mask = (1u << bits) - 1u;
    for (int q = threadIdx.x; q < NWARPS * RBINS / 2; q += NT) reinterpret_cast<uint32_t*>(&S.cnt[0][0])[q] = 0;
    __syncthreads();
    unsigned long long k[IT];
    uint32_t rank[IT];
#pragma unroll
    for (int j = 0; j < IT; j++) {
        const int li = w * 32 * IT + j * 32 + lane;
        k[j] = li < cnt ? src[li] : KEY_NONE;
        rank[j] = radix_peers((uint32_t)(k[j] >> (32 + shift)) & mask, bits, li < cnt);
    }
#pragma unroll
    for (int j = 0; j < IT; j++) {
        const int li = w * 32 * IT + j * 32 + lane;
        const bool valid = li < cnt;
        const uint32_t d = (uint32_t)(k[j] >> (32 + shift)) & mask;
        const uint32_t peers = rank[j];
        const uint32_t b = valid ? (uint32_t)S.cnt[w][d] : 0u;
        rank[j] = b + __popc(peers & lt);
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) S.cnt[w][d] = (uint16_t)(b + __popc(peers));
        __syncwarp();
    }
    __syncthreads();
    // digit starts, then each warp's offset within its digit: thread t owns
    // digits 2t, 2t + 1 (one 4-byte word of every warp's counters)
    {
        const int d0 = threadIdx.x * RDPT;
        uint32_t t0 = 0, t1 = 0;
#pragma unroll
        for (int q = 0; q < NWARPS; q++) {
            const uint32_t r = *reinterpret_cast<const uint32_t*>(&S.cnt[q][d0]);
            t0 += r & 0xffffu;
            t1 += r >> 16;
        }
        uint32_t s0 = block_scan_excl(t0 + t1, S.warp_tot), s1 = s0 + t0;
#pragma unroll
        for (int q = 0; q < NWARPS; q++) {
            uint32_t* p = reinterpret_cast<uint32_t*>(&S.cnt[q][d0]);
            const uint32_t r = *p;
            *p = s0 | (s1 << 16);
            s0 += r & 0xffffu;
            s1 += r >> 16;
        }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < IT; j++) {
        const int li = w * 32 * IT + j * 32 + lane;
        if (li < cnt) dst[S.cnt[w][(uint32_t)(k[j] >> (32 + shift)) & mask] + rank[j]] = k[j];
    }
    __syncthreads();
}

// Loads packed keys [base, base + cnt) of a row (cnt <= SR) with their
// weights and ranks, sorts them by id (key positions relative to the slice);
// returns the buffer holding the sorted keys.
template <int IT>
__device__ __forceinline__ int radix_sort_slice(const RowsOut& R, int64_t s, int64_t base, int cnt, int nbits,
                                                RadixSmem& S) {
    for (int j = threadIdx.x; j < cnt; j += NT) {
        const unsigned long long kk = __ldcs(R.pk + s + base + j);
        gather_wr(R, s, kk, S.wv[j], S.rv[j]);
        S.key[0][j] = with_pos(kk, j);
    }
    __syncthreads();
    const int passes = (nbits + RBITS - 1) / RBITS;
    int cur = 0, shift = 0;
    for (int p = 0; p < passes; p++) {
        const int bits = nbits / passes + (p < nbits % passes ? 1 : 0);
        radix_pass<IT>(S.key[cur], S.key[cur ^ 1], cnt, shift, bits, S);
        shift += bits;
        cur ^= 1;
    }
    return cur;
}

__device__ __forceinline__ int radix_sort_any(const RowsOut& R, int64_t s, int64_t base, int cnt, int nbits,
                                              RadixSmem& S) {
    if (cnt <= 4 * NT) return radix_sort_slice<4>(R, s, base, cnt, nbits, S);
    if (cnt <= 8 * NT) return radix_sort_slice<8>(R, s, base, cnt, nbits, S);
    return radix_sort_slice<16>(R, s, base, cnt, nbits, S);
}
static_assert(16 * NT == SR, "the widest item count covers a slice");

// Epilogue of a row's sorted keys, readable by position p < cnt: oriented
// entry p at ob + p, its weight and rank from wget(key), repeats flagged.
template <class Keys, class WR>
__device__ __forceinline__ void block_epilogue(const RowsOut& R, int32_t x, int cnt, const Keys& key_at,
                                               const WR& wget, int64_t ob) {
    for (int p = threadIdx.x; p < cnt; p += NT) {
        const unsigned long long kk = key_at(p);
        const int32_t c = key_col(kk);
        int32_t w, rk;
        wget(kk, w, rk);
        write_orient(R, ob + p, c, w, rk);
        if (p > 0 && key_col(key_at(p - 1)) == c) flag_dup(R, x, c);
    }
}

// Rows of 513..SR oriented entries sort whole in shared memory; hub rows
// (above SR) sort each SR slice and leave it in g0 (global, at the row's
// offset rowptr[x]).  nbits: bit length of the largest vertex id.
__global__ void __launch_bounds__(NT, 2) k_rows_block(RowsOut R, unsigned long long* g0, int32_t* cursor,
                                                      int nbits, const uint32_t* gate) {
    if (rows_gate_closed(gate)) return;
    extern __shared__ __align__(16) unsigned char bsm_raw[];
    RadixSmem& S = *reinterpret_cast<RadixSmem*>(bsm_raw);
    const int64_t lo = R.cls_off[CLS_BLOCK], hi = R.cls_off[CLS_HUB + 1];  // block and hub rows
    for (;;) {
        if (threadIdx.x == 0) S.item = atomicAdd(cursor, 1);
        __syncthreads();
        const int64_t ri = lo + S.item;
        __syncthreads();
        if (ri >= hi) break;
        const int32_t x = __ldg(R.list + ri);
        const int64_t s = __ldg(R.rowptr + x);
        const int64_t d = __ldg(R.odeg + x);
        for (int64_t base = 0; base < d; base += SR) {
            const int cnt = (int)min((int64_t)SR, d - base);
            const int b = radix_sort_any(R, s, base, cnt, nbits, S);
            if (d <= SR) {
                block_epilogue(R, x, cnt, [&](int p) { return S.key[b][p]; },
                               [&](unsigned long long kk, int32_t& w, int32_t& rk) {
                                   const uint32_t src = key_pos(kk);
                                   w = S.wv[src];
                                   rk = S.rv[src];
                               },
                               __ldg(R.orowptr + x));
            } else {
                // positions in the key are relative to the slice: make them
                // packed indices of the row for the merges and the epilogue
                for (int j = threadIdx.x; j < cnt; j += NT)
                    g0[s + base + j] = S.key[b][j] + (unsigned long long)base;
            }
            __syncthreads();
        }
    }
}

// One merge level of the hub rows: runs of `len` keys at each hub row's
// offset in src become runs of 2 len in dst (rows with d <= len are done).
// A block takes MT consecutive outputs of one row: the two input windows
// (found by merge path in global memory) are staged in shared memory, merged
// there, and written in order.
constexpr int MT = 4096;

__global__ void __launch_bounds__(NT) k_rows_merge(RowsOut R, const unsigned long long* src,
                                                   unsigned long long* dst, int64_t len,
                                                   const uint32_t* gate) {
    if (rows_gate_closed(gate)) return;
    __shared__ unsigned long long win[MT];
    __shared__ int64_t split[2];
    const int64_t lo = R.cls_off[CLS_HUB], hi = R.cls_off[CLS_HUB + 1];
    for (int64_t ri = lo + blockIdx.x; ri < hi; ri += gridDim.x) {
        const int32_t x = __ldg(R.list + ri);
        const int64_t s = __ldg(R.rowptr + x);
        const int64_t d = __ldg(R.odeg + x);
        if (d <= len) continue;
        for (int64_t q0 = 0; q0 < d; q0 += MT) {
            const int64_t q1 = min(d, q0 + MT);
            const int64_t pb = (q0 / (2 * len)) * 2 * len;  // tiles never cross a pair (MT | 2 len)
            const int64_t na = min(len, d - pb), nb = max((int64_t)0, min(len, d - pb - len));
            const unsigned long long* a = src + s + pb;
            const unsigned long long* b = a + len;
            auto A = [&](int64_t i) { return a[i]; };
            auto B = [&](int64_t i) { return b[i]; };
            if (threadIdx.x < 2) split[threadIdx.x] = merge_split(A, na, B, nb, (threadIdx.x ? q1 : q0) - pb);
            __syncthreads();
            const int64_t i0 = split[0], i1 = split[1];
            const int64_t j0 = (q0 - pb) - i0, j1 = (q1 - pb) - i1;
            const int la = (int)(i1 - i0), lb = (int)(j1 - j0);
            for (int k = threadIdx.x; k < la; k += NT) win[k] = a[i0 + k];
            for (int k = threadIdx.x; k < lb; k += NT) win[la + k] = b[j0 + k];
            __syncthreads();
            const int per = MT / NT;
            const int d0 = threadIdx.x * per;
            if (d0 < la + lb) {
                const int cnt = min(per, la + lb - d0);
                merge_out([&](int64_t i) { return win[i]; }, la, [&](int64_t i) { return win[la + i]; }, lb, d0,
                          cnt, [&](int64_t q, unsigned long long v) { dst[s + q0 + q] = v; });
            }
            __syncthreads();
        }
    }
}

// Epilogue of the hub rows, from the buffer holding each row's last level:
// one block per row; weights and ranks gathered through the packed key
// (its position in the weight-sorted row).
__global__ void __launch_bounds__(NT) k_rows_hub_out(RowsOut R, const unsigned long long* g0,
                                                     const unsigned long long* g1,
                                                     const uint32_t* gate) {
    if (rows_gate_closed(gate)) return;
    const int64_t lo = R.cls_off[CLS_HUB], hi = R.cls_off[CLS_HUB + 1];
    for (int64_t ri = lo + blockIdx.x; ri < hi; ri += gridDim.x) {
        const int32_t x = __ldg(R.list + ri);
        const int64_t s = __ldg(R.rowptr + x);
        const int64_t d = __ldg(R.odeg + x);
        int levels = 0;
        for (int64_t len = SR; len < d; len <<= 1) levels++;
        const unsigned long long* g = ((levels & 1) ? g1 : g0) + s;
        block_epilogue(R, x, (int)d, [&](int64_t p) { return __ldcs(g + p); },
                       [&](unsigned long long kk, int32_t& w, int32_t& rk) {
                           gather_wr(R, s, __ldg(R.pk + s + key_pos(kk)), w, rk);
                       },
                       __ldg(R.orowptr + x));
    }
}

}  // namespace rows
}  // namespace wtri
