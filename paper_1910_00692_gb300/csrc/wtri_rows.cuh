// Id-sorted symmetric rows and the degree orientation, derived from the
// weight-sorted rows by a per-row segmented sort.
//
// Input: the weight-sorted rows (row x holds its neighbours in edge order at
// [rowptr[x], rowptr[x+1]) of wcol / wwt / wrk) and the row of each entry
// (wrow, build scratch).  Output, for every row x:
//   * scol / swt at the same positions, ascending by neighbour id (N(a) of
//     Section 4, the lists the closing-edge lookups search);
//   * the oriented row of NodeIterator++ (Section 5.2): the neighbours c of
//     higher (degree, id) rank than x, ascending by id, at
//     [orowptr[x], orowptr[x+1]) of ocol / owt / ork;
//   * repeated pairs (a neighbour twice in one row) flagged as an invalid
//     input (Section 1: a simple graph).
//
// Rows are sorted by size class, every sort on 64-bit keys (id << 32 |
// position in the row), unique within a row:
//   d <= 32           sub-warp bitonic network in registers (groups of 8, 16
//                     or 32 lanes, several rows per warp);
//   32 < d <= 1024    one warp per row: bitonic network over 2..32 keys per
//                     lane in registers, transposed through shared memory;
//   1024 < d          one block per row: warp-sorted runs of 1024 merged by
//                     merge path in shared memory into runs of SB; rows above
//                     SB leave their sorted runs in global scratch, where one
//                     launch per merge level (many blocks, one row each)
//                     merges pairs of runs until the row is one run.
// The orientation is decided first, for every entry at once (k_fwd: a bit
// per entry, whether the neighbour ranks above the row's vertex, and the
// oriented out-degree of each row); a scan gives the oriented offsets
// orowptr.  The bit then travels inside the sort key (id << 32 | bit << 31
// | position), so the sorts write the oriented entries in place with no
// gathers of their own.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "wtri_internal.cuh"

namespace wtri {
namespace rows {

constexpr int NT = 256;           // block kernels
constexpr int NWARPS = NT / 32;
constexpr int WMAX = 1024;        // longest row sorted by one warp
constexpr int SB = 8192;          // longest run a block sorts in shared memory
constexpr int MOPT = 16;          // merge path: outputs per thread and step

// Size classes of a row (by degree d): three sub-warp classes, five warp
// classes by keys per lane (2, 4, 8, 16, 32), block rows, hub rows (> SB).
enum : int {
    CLS_NONE = 0, CLS_G8, CLS_G16, CLS_G32,
    CLS_W2, CLS_W4, CLS_W8, CLS_W16, CLS_W32,
    CLS_BLOCK, CLS_HUB
};
constexpr int NCLS = 11;

__device__ __forceinline__ int row_class(int64_t d) {
    if (d <= 0) return CLS_NONE;
    if (d <= 8) return CLS_G8;
    if (d <= 16) return CLS_G16;
    if (d <= 32) return CLS_G32;
    if (d <= 64) return CLS_W2;
    if (d <= 128) return CLS_W4;
    if (d <= 256) return CLS_W8;
    if (d <= 512) return CLS_W16;
    if (d <= WMAX) return CLS_W32;
    if (d <= SB) return CLS_BLOCK;
    return CLS_HUB;
}

// Whether x (degree dx) comes before its neighbour c in the (degree, id)
// order.  The degrees saturated to 8 bits (a 1-byte-per-vertex table that
// stays in L2) decide unless both saturate; then the exact degree of c comes
// from the row offsets.
constexpr uint32_t DEG8_SAT = 255;

__device__ __forceinline__ bool rank_before(int32_t x, int64_t dx, const uint8_t* __restrict__ deg8,
                                            const int64_t* __restrict__ rowptr, int32_t c) {
    uint64_t dc = __ldg(deg8 + c);
    if (dx >= DEG8_SAT) {
        if (dc < DEG8_SAT) return false;
        dc = (uint64_t)(__ldg(rowptr + c + 1) - __ldg(rowptr + c));
    }
    return (uint64_t)dx < dc || ((uint64_t)dx == dc && x < c);
}

struct RowsOut {
    const int64_t* rowptr;
    const int32_t* wcol;
    const int32_t* wwt;
    const int32_t* wrk;
    const uint8_t* deg8;
    int32_t* scol;
    int32_t* swt;
    const uint32_t* fwd;             // bit j: entry j's neighbour ranks above its row's vertex
    const int64_t* orowptr;          // oriented row offsets
    int32_t* ocol;
    int32_t* owt;
    int32_t* ork;
    uint32_t* err;                   // build status: error bits
    unsigned long long* first_dup;   // smallest entry index of a repeated neighbour
    const int32_t* list;             // rows of each class, class c at [cls_off[c], cls_off[c+1])
    const int32_t* cls_off;
};

// Gate of the row kernels: an earlier step failed.  A repeated pair found by
// another row kernel does not close it, so that every size class still runs
// and the smallest repeated entry is reported whatever the launch order.
__device__ __forceinline__ bool rows_gate_closed(const uint32_t* gate) {
    return (*(volatile const uint32_t*)gate & ~(uint32_t)DEV_ERR_DUPLICATE) != 0;
}

__device__ __forceinline__ void flag_dup(const RowsOut& R, int64_t j) {
    atomicOr(R.err, DEV_ERR_DUPLICATE);
    atomicMin(R.first_dup, (unsigned long long)j);
}

// ---------------------------------------------------------------------------
// Row classes: counts, then the list of rows of each class.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NT) k_class_count(int32_t n, const int64_t* __restrict__ rowptr,
                                                    int32_t* __restrict__ cls_cnt, const uint32_t* gate) {
    if (rows_gate_closed(gate)) return;
    __shared__ int32_t sc[NCLS];
    if (threadIdx.x < NCLS) sc[threadIdx.x] = 0;
    __syncthreads();
    for (int64_t x = (int64_t)blockIdx.x * NT + threadIdx.x; x < n; x += (int64_t)gridDim.x * NT) {
        const int c = row_class(rowptr[x + 1] - rowptr[x]);
        if (c != CLS_NONE) atomicAdd(&sc[c], 1);
    }
    __syncthreads();
    if (threadIdx.x < NCLS && sc[threadIdx.x]) atomicAdd(cls_cnt + threadIdx.x, sc[threadIdx.x]);
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

__global__ void __launch_bounds__(NT) k_class_fill(int32_t n, const int64_t* __restrict__ rowptr,
                                                   int32_t* __restrict__ cls_cur, int32_t* __restrict__ list,
                                                   const uint32_t* gate) {
    if (rows_gate_closed(gate)) return;
    const int lane = threadIdx.x & 31;
    for (int64_t x0 = (int64_t)blockIdx.x * NT; x0 < n; x0 += (int64_t)gridDim.x * NT) {
        const int64_t x = x0 + threadIdx.x;
        const int c = x < n ? row_class(rowptr[x + 1] - rowptr[x]) : CLS_NONE;
        // one atomic per class present in the warp
        for (int k = 1; k < NCLS; k++) {
            const uint32_t b = __ballot_sync(0xffffffffu, c == k);
            if (!b) continue;
            int32_t base = 0;
            if (lane == __ffs(b) - 1) base = atomicAdd(cls_cur + k, __popc(b));
            base = __shfl_sync(0xffffffffu, base, __ffs(b) - 1);
            if (c == k) list[base + __popc(b & ((1u << lane) - 1u))] = (int32_t)x;
        }
    }
}

// ---------------------------------------------------------------------------
// Orientation of every entry: bit j of fwd says whether entry j's neighbour
// ranks above its row's vertex (NodeIterator++ keeps the edge in that row);
// odeg[x] counts them (rows are contiguous: a warp adds one count per row
// it touches).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NT) k_fwd(int64_t n2, const int32_t* __restrict__ wrow,
                                            const int32_t* __restrict__ wcol,
                                            const int64_t* __restrict__ rowptr,
                                            const uint8_t* __restrict__ deg8, uint32_t* __restrict__ fwd,
                                            int32_t* __restrict__ odeg, const uint32_t* gate) {
    if (rows_gate_closed(gate)) return;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * NT) >> 5;
    for (int64_t base = (((int64_t)blockIdx.x * NT + threadIdx.x) >> 5) * 32; base < n2;
         base += nwarps * 32) {
        const int64_t e = base + lane;
        const bool valid = e < n2;
        int32_t x = -1;
        bool f = false;
        if (valid) {
            x = __ldcs(wrow + e);
            const int32_t c = __ldcs(wcol + e);
            const int64_t dx = __ldg(rowptr + x + 1) - __ldg(rowptr + x);
            f = rank_before(x, dx, deg8, rowptr, c);
        }
        const uint32_t bits = __ballot_sync(0xffffffffu, f);
        if (lane == 0) fwd[base >> 5] = bits;  // base is a multiple of 32
        const int32_t xp = __shfl_up_sync(0xffffffffu, x, 1);
        const bool head = valid && (lane == 0 || xp != x);
        const uint32_t heads = __ballot_sync(0xffffffffu, head);
        if (head) {
            const uint32_t above = heads & ~((2u << lane) - 1u);  // heads after this lane
            const int end = above ? __ffs(above) - 1 : 32;
            const uint32_t seg = (end >= 32 ? 0xffffffffu : ((1u << end) - 1u)) & ~((1u << lane) - 1u);
            const int cnt = __popc(bits & seg);
            if (cnt) atomicAdd(odeg + x, cnt);
        }
    }
}

__device__ __forceinline__ bool fwd_bit(const uint32_t* fwd, int64_t j) {
    return (__ldg(fwd + (j >> 5)) >> (j & 31)) & 1u;
}

// ---------------------------------------------------------------------------
// Writes: the id-sorted entry; the oriented entry at its compact position.
// Outputs are written once and not read again by this pass: streaming
// stores, so that they do not displace the tables the pass gathers from.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void write_sym(const RowsOut& R, int64_t j, int32_t c, int32_t w) {
    __stcs(R.scol + j, c);
    __stcs(R.swt + j, w);
}
__device__ __forceinline__ void write_orient(const RowsOut& R, int64_t p, int32_t c, int32_t w,
                                             int32_t rk) {
    __stcs(R.ocol + p, c);
    __stcs(R.owt + p, w);
    __stcs(R.ork + p, rk);
}

__device__ __forceinline__ uint32_t lane_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

constexpr unsigned long long KEY_NONE = ~0ull;  // sorts after every real key

// Sort key of entry j of a row: neighbour id, then the orientation bit, then
// the position (unique within the row; the sorts order by id only, the rest
// rides along).
__device__ __forceinline__ unsigned long long row_key(int32_t c, bool f, int64_t j) {
    return ((unsigned long long)(uint32_t)c << 32) | ((unsigned long long)f << 31) |
           (unsigned long long)(uint32_t)j;
}
__device__ __forceinline__ int32_t key_col(unsigned long long k) { return (int32_t)(k >> 32); }
__device__ __forceinline__ bool key_fwd(unsigned long long k) { return (k >> 31) & 1ull; }
__device__ __forceinline__ uint32_t key_pos(unsigned long long k) { return (uint32_t)k & 0x7fffffffu; }

// ---------------------------------------------------------------------------
// Rows of at most G entries (G = 8, 16, 32): G lanes per row, a bitonic
// network across the group's lanes.
// ---------------------------------------------------------------------------
template <int G>
__global__ void __launch_bounds__(NT) k_rows_small(RowsOut R, int cls, const uint32_t* gate) {
    if (rows_gate_closed(gate)) return;
    const int lane = threadIdx.x & 31, gl = lane & (G - 1), grp = lane / G;
    constexpr int RPW = 32 / G;  // rows per warp
    const int64_t lo = R.cls_off[cls], hi = R.cls_off[cls + 1];
    const int64_t nwarps = ((int64_t)gridDim.x * NT) >> 5;
    const uint32_t gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (grp * G));
    for (int64_t wbase = lo + (((int64_t)blockIdx.x * NT + threadIdx.x) >> 5) * RPW; wbase < hi;
         wbase += nwarps * RPW) {
        const int64_t ri = wbase + grp;
        int32_t x = 0;
        int64_t s = 0, d = 0, ob = 0;
        if (ri < hi) {
            x = __ldg(R.list + ri);
            s = __ldg(R.rowptr + x);
            d = __ldg(R.rowptr + x + 1) - s;
            ob = __ldg(R.orowptr + x);
        }
        const bool valid = gl < d;
        unsigned long long key = KEY_NONE;
        int32_t w = 0, rk = 0;
        if (valid) {
            key = row_key(__ldcs(R.wcol + s + gl), fwd_bit(R.fwd, s + gl), gl);
            w = __ldcs(R.wwt + s + gl);
            rk = __ldcs(R.wrk + s + gl);
        }
#pragma unroll
        for (int k = 2; k <= G; k <<= 1) {
#pragma unroll
            for (int j = k >> 1; j > 0; j >>= 1) {
                const unsigned long long ok = __shfl_xor_sync(0xffffffffu, key, j, G);
                const bool up = (gl & k) == 0, lower = (gl & j) == 0;
                key = (lower == up) ? (ok < key ? ok : key) : (ok > key ? ok : key);
            }
        }
        const int src = (int)key_pos(key) & (G - 1);
        const int32_t ws = __shfl_sync(0xffffffffu, w, src, G);
        const int32_t rks = __shfl_sync(0xffffffffu, rk, src, G);
        const unsigned long long prev = __shfl_up_sync(0xffffffffu, key, 1, G);
        const int32_t c = key_col(key);
        const bool f = valid && key_fwd(key);
        if (valid) {
            write_sym(R, s + gl, c, ws);
            if (gl > 0 && key_col(prev) == c) flag_dup(R, s + gl);
        }
        const uint32_t b = __ballot_sync(0xffffffffu, f) & gmask;
        if (f) write_orient(R, ob + __popc(b & lane_lt()), c, ws, rks);
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
// Rows of 33..1024 entries: one warp per row, 32 * EPL keys in registers
// (EPL = 2, 4, 8, 16, 32 by class), sorted, transposed through the warp's
// shared memory (keys, and the row's weights and ranks by position).
// ---------------------------------------------------------------------------
template <int EPL>
__global__ void __launch_bounds__(NT) k_rows_warp(RowsOut R, int cls, const uint32_t* gate) {
    if (rows_gate_closed(gate)) return;
    extern __shared__ __align__(16) unsigned long long wsm[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t lt = lane_lt();
    unsigned long long* run = wsm + (size_t)wid * 2 * 32 * EPL;
    int32_t* wv = reinterpret_cast<int32_t*>(run + 32 * EPL);  // weights by position
    int32_t* rv = wv + 32 * EPL;                                 // ranks by position
    const int64_t lo = R.cls_off[cls], hi = R.cls_off[cls + 1];
    const int64_t nwarps = ((int64_t)gridDim.x * NT) >> 5;
    for (int64_t ri = lo + (((int64_t)blockIdx.x * NT + threadIdx.x) >> 5); ri < hi; ri += nwarps) {
        const int32_t x = __ldg(R.list + ri);
        const int64_t s = __ldg(R.rowptr + x);
        const int d = (int)(__ldg(R.rowptr + x + 1) - s);
        const int64_t ob = __ldg(R.orowptr + x);
        unsigned long long k[EPL];
#pragma unroll
        for (int i = 0; i < EPL; i++) {
            const int j = i * 32 + lane;  // coalesced loads; the network ignores input order
            if (j < d) {
                k[i] = row_key(__ldcs(R.wcol + s + j), fwd_bit(R.fwd, s + j), j);
                wv[j] = __ldcs(R.wwt + s + j);
                rv[j] = __ldcs(R.wrk + s + j);
            } else {
                k[i] = KEY_NONE;
            }
        }
        warp_bitonic<EPL>(k);
#pragma unroll
        for (int i = 0; i < EPL; i++) run[swz(lane * EPL + i)] = k[i];
        __syncwarp();
        int64_t orun = 0;
        for (int base = 0; base < d; base += 32) {
            const int j = base + lane;
            bool f = false;
            int32_t c = 0, w = 0, rk = 0;
            if (j < d) {
                const unsigned long long kk = run[swz(j)];
                c = key_col(kk);
                f = key_fwd(kk);
                const uint32_t src = key_pos(kk);
                w = wv[src];
                rk = rv[src];
                write_sym(R, s + j, c, w);
                if (j > 0 && key_col(run[swz(j - 1)]) == c) flag_dup(R, s + j);
            }
            const uint32_t b = __ballot_sync(0xffffffffu, f);
            if (f) write_orient(R, ob + orun + __popc(b & lt), c, w, rk);
            orun += __popc(b);
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

struct BlockSmem {
    unsigned long long buf[2][SB];   // runs, ping-pong (swizzled per 1024-key run)
    int32_t wv[SB];                  // weights of the slice by position
    int32_t rv[SB];                  // ranks of the slice by position
    uint32_t warp_tot[NWARPS];
    int32_t item;
};

// Sorts keys [base, base + cnt) of a row (cnt <= SB) into one run in
// S.buf[returned index] (element p at swz(p)); also stages the slice's
// weights and ranks by position.  nw = the power of two of 1024-key slices
// covering cnt; warp w < nw sorts slice w in registers; log2(nw) merge-path
// levels in shared memory make one run of nw * 1024 keys (the padding sorts
// last).
__device__ __forceinline__ int block_sort_run(const RowsOut& R, int64_t s, int64_t base, int cnt,
                                              BlockSmem& S) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int nw = 1;
    while (nw * 1024 < cnt) nw <<= 1;
    for (int j = threadIdx.x; j < cnt; j += NT) {
        S.wv[j] = __ldcs(R.wwt + s + base + j);
        S.rv[j] = __ldcs(R.wrk + s + base + j);
    }
    if (wid < nw) {
        unsigned long long k[32];
#pragma unroll
        for (int i = 0; i < 32; i++) {
            const int j = wid * 1024 + i * 32 + lane;
            k[i] = j < cnt ? row_key(__ldcs(R.wcol + s + base + j), fwd_bit(R.fwd, s + base + j), j)
                           : KEY_NONE;
        }
        warp_bitonic<32>(k);
#pragma unroll
        for (int i = 0; i < 32; i++) S.buf[0][swz(wid * 1024 + lane * 32 + i)] = k[i];
    }
    __syncthreads();
    // Every access below goes through swz (a bijection inside each group of
    // 32 keys): the merge path writes 4..32 consecutive keys per thread, which
    // unswizzled would put every lane of a warp on the same bank.
    int cur = 0;
    const int total = nw * 1024;
    const int per = total / NT;  // outputs per thread: 4 .. 32
    for (int len = 1024; len < total; len <<= 1) {
        const unsigned long long* src = S.buf[cur];
        unsigned long long* dst = S.buf[cur ^ 1];
        const int q0 = threadIdx.x * per;
        const int pair = q0 / (2 * len), pb = pair * 2 * len;
        auto A = [&](int64_t i) { return src[swz(pb + (int)i)]; };
        auto B = [&](int64_t i) { return src[swz(pb + len + (int)i)]; };
        merge_out(A, len, B, len, q0 - pb, per,
                  [&](int64_t q, unsigned long long v) { dst[swz(pb + (int)q)] = v; });
        __syncthreads();
        cur ^= 1;
    }
    return cur;
}

// Epilogue of sorted keys readable by position p < cnt (the positions of a
// row starting at p0): id-sorted entries at s + p0 + p, repeats, oriented
// entries at ob + orun + (rank among the oriented keys).  Weights and ranks
// come from wget(key).  Returns the number of oriented keys.  Block-wide:
// per 256 positions one ballot per warp and one barrier pair.
template <class Keys, class WR>
__device__ __forceinline__ int64_t block_epilogue(const RowsOut& R, int64_t s, int64_t p0, int cnt,
                                                  const Keys& key_at, const WR& wget, int64_t ob,
                                                  int64_t orun, unsigned long long prev_key,
                                                  uint32_t* warp_tot) {
    const int lane = threadIdx.x & 31, w_ = threadIdx.x >> 5;
    const uint32_t lt = lane_lt();
    for (int base = 0; base < cnt; base += NT) {
        const int p = base + threadIdx.x;
        bool f = false;
        int32_t c = 0, w = 0, rk = 0;
        if (p < cnt) {
            const unsigned long long kk = key_at(p);
            c = key_col(kk);
            f = key_fwd(kk);
            wget(kk, w, rk);
            write_sym(R, s + p0 + p, c, w);
            const unsigned long long pk = p > 0 ? key_at(p - 1) : prev_key;
            if ((p0 + p) > 0 && key_col(pk) == c) flag_dup(R, s + p0 + p);
        }
        const uint32_t b = __ballot_sync(0xffffffffu, f);
        if (lane == 0) warp_tot[w_] = __popc(b);
        __syncthreads();
        uint32_t before = 0, total = 0;
#pragma unroll
        for (int k = 0; k < NWARPS; k++) {
            const uint32_t t = warp_tot[k];
            before += k < w_ ? t : 0u;
            total += t;
        }
        if (f) write_orient(R, ob + orun + before + __popc(b & lt), c, w, rk);
        orun += total;
        __syncthreads();
    }
    return orun;
}

// Rows of 1025..SB entries sort whole in shared memory; hub rows (above SB)
// sort each SB slice and leave it in g0 (global, at the row's offset).
__global__ void __launch_bounds__(NT) k_rows_block(RowsOut R, unsigned long long* g0, int32_t* cursor,
                                                   const uint32_t* gate) {
    if (rows_gate_closed(gate)) return;
    extern __shared__ __align__(16) unsigned char bsm_raw[];
    BlockSmem& S = *reinterpret_cast<BlockSmem*>(bsm_raw);
    const int64_t lo = R.cls_off[CLS_BLOCK], hi = R.cls_off[CLS_HUB + 1];  // block and hub rows
    for (;;) {
        if (threadIdx.x == 0) S.item = atomicAdd(cursor, 1);
        __syncthreads();
        const int64_t ri = lo + S.item;
        __syncthreads();
        if (ri >= hi) break;
        const int32_t x = __ldg(R.list + ri);
        const int64_t s = __ldg(R.rowptr + x);
        const int64_t d = __ldg(R.rowptr + x + 1) - s;
        for (int64_t base = 0; base < d; base += SB) {
            const int cnt = (int)min((int64_t)SB, d - base);
            const int b = block_sort_run(R, s, base, cnt, S);
            if (d <= SB) {
                block_epilogue(R, s, 0, cnt, [&](int p) { return S.buf[b][swz(p)]; },
                               [&](unsigned long long kk, int32_t& w, int32_t& rk) {
                                   const uint32_t src = key_pos(kk);
                                   w = S.wv[src];
                                   rk = S.rv[src];
                               },
                               __ldg(R.orowptr + x), 0, KEY_NONE, S.warp_tot);
            } else {
                // positions in the key are relative to the slice: make them
                // row positions for the merges and the final epilogue
                for (int j = threadIdx.x; j < cnt; j += NT)
                    g0[s + base + j] = S.buf[b][swz(j)] + (unsigned long long)base;
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
        const int64_t d = __ldg(R.rowptr + x + 1) - s;
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
// one block per row, slices of SB positions staged in shared memory with
// their weights and ranks gathered from the weight-sorted row.
__global__ void __launch_bounds__(NT) k_rows_hub_out(RowsOut R, const unsigned long long* g0,
                                                     const unsigned long long* g1,
                                                     const uint32_t* gate) {
    if (rows_gate_closed(gate)) return;
    __shared__ uint32_t warp_tot[NWARPS];
    const int64_t lo = R.cls_off[CLS_HUB], hi = R.cls_off[CLS_HUB + 1];
    for (int64_t ri = lo + blockIdx.x; ri < hi; ri += gridDim.x) {
        const int32_t x = __ldg(R.list + ri);
        const int64_t s = __ldg(R.rowptr + x);
        const int64_t d = __ldg(R.rowptr + x + 1) - s;
        int levels = 0;
        for (int64_t len = SB; len < d; len <<= 1) levels++;
        const unsigned long long* g = ((levels & 1) ? g1 : g0) + s;
        block_epilogue(R, s, 0, (int)d, [&](int64_t p) { return __ldcs(g + p); },
                       [&](unsigned long long kk, int32_t& w, int32_t& rk) {
                           const uint32_t src = key_pos(kk);
                           w = __ldg(R.wwt + s + src);
                           rk = __ldg(R.wrk + s + src);
                       },
                       __ldg(R.orowptr + x), 0, KEY_NONE, warp_tot);
        __syncthreads();
    }
}

}  // namespace rows
}  // namespace wtri
