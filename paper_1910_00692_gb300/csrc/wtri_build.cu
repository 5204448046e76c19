// Device graph build: validation, degrees, the edge order, per-vertex
// weight-sorted lists, id-sorted lists and the degree orientation.
//
// Preprocessing named by the paper: "Sort E in decreasing order of weight"
// (Algorithm 2, first step), neighbour sets N(a) and degrees d_a (Section
// 4), and the NodeIterator++ degree ordering (Section 5.2).
//
// Pipeline (one stream, inputs read once from HBM or host):
//   1. k_validate: rejects bad edges, finds the max weight.
//   2. Edge order: stable LSD radix sort of key (wmax - w) carrying (u, v).
//   3. Weight-sorted lists: the virtual stream "two entries per edge, in edge
//      order" is stably radix-sorted by row, so each row keeps edge order.
//   4. Row offsets and degrees from the boundaries of the sorted rows (no
//      atomics), plus the list of long rows.
//   5. Id-sorted lists: the weight-sorted entries, read row by row (so the
//      stream is ascending in its row x), are mirrored to (row c, col x) and
//      stably sorted by row c, which leaves each row ascending in x.
//   6. Oriented lists: per row, keep neighbours of higher (degree, id) rank,
//      in place of the row's own slots; repeated pairs show up in the same
//      pass as equal neighbours next to each other.
#include <cuda_runtime.h>
#include <stdio.h>

#include <algorithm>
#include <string>

#include "wtri_internal.cuh"
#include "wtri_radix.cuh"

namespace wtri {

namespace {

constexpr int BLK = 256;

struct BuildStatus {
    uint32_t err;
    int32_t wmax;
    int32_t maxdeg;
    int32_t pad;
    unsigned long long first_bad;  // smallest offending edge index
};

__global__ void k_validate(int32_t n, int64_t m, const int32_t* __restrict__ u,
                           const int32_t* __restrict__ v, const int32_t* __restrict__ w,
                           BuildStatus* st) {
    int32_t wloc = 0;
    uint32_t eloc = 0;
    unsigned long long bad = ~0ull;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = __ldg(u + i), b = __ldg(v + i), x = __ldg(w + i);
        uint32_t e = 0;
        if (a < 0 || a >= n || b < 0 || b >= n) e |= DEV_ERR_RANGE;
        else if (a == b) e |= DEV_ERR_SELF_LOOP;
        if (x <= 0) e |= DEV_ERR_WEIGHT;
        if (e) {
            eloc |= e;
            if ((unsigned long long)i < bad) bad = (unsigned long long)i;
            continue;
        }
        wloc = max(wloc, x);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        wloc = max(wloc, __shfl_xor_sync(0xffffffffu, wloc, o));
        eloc |= __shfl_xor_sync(0xffffffffu, eloc, o);
        unsigned long long ob = __shfl_xor_sync(0xffffffffu, bad, o);
        bad = ob < bad ? ob : bad;
    }
    if ((threadIdx.x & 31) == 0) {
        if (wloc) atomicMax(&st->wmax, wloc);
        if (eloc) {
            atomicOr(&st->err, eloc);
            atomicMin(&st->first_bad, bad);
        }
    }
}

// ---- exclusive scan int32 -> int64 (3 kernels) ---------------------------
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = BLK * SCAN_ITEMS;

__device__ __forceinline__ int64_t block_scan_i64(int64_t x, int64_t* sh, int64_t* total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) sh[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        int64_t t = lane < (BLK / 32) ? sh[lane] : 0;
        int64_t ti = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, ti, o);
            if (lane >= o) ti += y;
        }
        if (lane < BLK / 32) sh[lane] = ti - t;
        if (lane == BLK / 32 - 1) *total = ti;
    }
    __syncthreads();
    int64_t r = sh[wid] + inc - x;
    __syncthreads();
    return r;
}

__global__ void k_scan_reduce(const int32_t* __restrict__ in, int64_t n, int64_t* tile_sums,
                              int32_t* maxval) {
    __shared__ int64_t sh[BLK / 32];
    __shared__ int64_t tot;
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    int64_t s = 0;
    int32_t mx = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; j++) {
        int64_t i = base + j * BLK + threadIdx.x;
        if (i < n) {
            int32_t x = in[i];
            s += x;
            mx = max(mx, x);
        }
    }
    block_scan_i64(s, sh, &tot);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0 && maxval) atomicMax(maxval, mx);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

__global__ void k_scan_tiles(int64_t* tile_sums, int64_t tiles, int64_t* out_total) {
    __shared__ int64_t sh[BLK / 32];
    __shared__ int64_t tot;
    int64_t carry = 0;
    for (int64_t b = 0; b < tiles; b += BLK) {
        int64_t i = b + threadIdx.x;
        int64_t x = i < tiles ? tile_sums[i] : 0;
        int64_t ex = block_scan_i64(x, sh, &tot);
        if (i < tiles) tile_sums[i] = carry + ex;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) *out_total = carry;
}

__global__ void k_scan_apply(const int32_t* __restrict__ in, int64_t n,
                             const int64_t* __restrict__ tile_offs, int64_t* __restrict__ out) {
    __shared__ int64_t sh[BLK / 32];
    __shared__ int64_t tot;
    // blocked arrangement: thread t owns items [t*ITEMS, (t+1)*ITEMS) of the tile
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int32_t x[SCAN_ITEMS];
    int64_t s = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; j++) {
        x[j] = (base + j < n) ? in[base + j] : 0;
        s += x[j];
    }
    int64_t run = block_scan_i64(s, sh, &tot) + tile_offs[blockIdx.x];
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; j++) {
        if (base + j < n) out[base + j] = run;
        run += x[j];
    }
}

// ---- radix loaders / storers for the build ---------------------------------
// A record is (key, v0, v1, v2); copied tiles hold each source array at a
// stride of radix::TT words.
using radix::TT;

// Edge order input: key = wmax - w, values (u, v).
struct EdgeLoader {
    static constexpr double REC_BYTES = 12.0;  // u, v, w
    static constexpr int NARR = 3;             // w, u, v
    static constexpr uint32_t TILE_WORDS = TT;
    const int32_t* u;
    const int32_t* v;
    const int32_t* w;
    int32_t wmax;
    __device__ __forceinline__ uint32_t key(int64_t i) const { return (uint32_t)(wmax - __ldg(w + i)); }
    __device__ __forceinline__ const void* tile_src(int a, int64_t tbase) const {
        return (a == 0 ? w : (a == 1 ? u : v)) + tbase;
    }
    __device__ __forceinline__ uint4 srec(const uint32_t* in, int li, int64_t) const {
        return make_uint4((uint32_t)(wmax - (int32_t)in[li]), in[TT + li], in[2 * TT + li], 0u);
    }
    __device__ __forceinline__ uint4 grec(int64_t i) const {
        return make_uint4(key(i), (uint32_t)__ldg(u + i), (uint32_t)__ldg(v + i), 0u);
    }
    bool tma_ok() const { return (((uintptr_t)u | (uintptr_t)v | (uintptr_t)w) & 15) == 0; }
};

// Final edge-order output.
struct EdgeOrderStorer {
    __host__ __device__ double rec_bytes() const { return 12.0; }
    int32_t* ou;
    int32_t* ov;
    int32_t* ow;
    int32_t wmax;
    __device__ __forceinline__ void store(int64_t p, const uint4& r) const {
        ow[p] = wmax - (int32_t)r.x;
        ou[p] = (int32_t)r.y;
        ov[p] = (int32_t)r.z;
    }
};

// Virtual stream of adjacency entries in edge order: entry i belongs to edge
// r = i / 2; side 0 is (row u, col v), side 1 is (row v, col u).  Record:
// (row, col, weight, r).
struct OrderEntryLoader {
    static constexpr double REC_BYTES = 6.0;  // u, v, w: 12 bytes per edge, two entries
    static constexpr int NARR = 3;            // ou, ov, ow (half a tile of edges each)
    static constexpr uint32_t TILE_WORDS = TT / 2;
    const int32_t* ou;
    const int32_t* ov;
    const int32_t* ow;
    __device__ __forceinline__ const void* tile_src(int a, int64_t tbase) const {
        return (a == 0 ? ou : (a == 1 ? ov : ow)) + (tbase >> 1);
    }
    __device__ __forceinline__ uint4 srec(const uint32_t* in, int li, int64_t tbase) const {
        const int e = li >> 1, side = li & 1;
        const uint32_t a = in[e], b = in[TT + e];
        return make_uint4(side ? b : a, side ? a : b, in[2 * TT + e], (uint32_t)((tbase >> 1) + e));
    }
    __device__ __forceinline__ uint4 grec(int64_t i) const {
        const int64_t r = i >> 1;
        const uint32_t a = (uint32_t)__ldg(ou + r), b = (uint32_t)__ldg(ov + r);
        return (i & 1) ? make_uint4(b, a, (uint32_t)__ldg(ow + r), (uint32_t)r)
                       : make_uint4(a, b, (uint32_t)__ldg(ow + r), (uint32_t)r);
    }
    __device__ __forceinline__ uint32_t key(int64_t i) const {
        return (uint32_t)__ldg(((i & 1) ? ov : ou) + (i >> 1));
    }
    bool tma_ok() const { return (((uintptr_t)ou | (uintptr_t)ov | (uintptr_t)ow) & 15) == 0; }
};

// Mirrored weight-sorted entries: entry i of row x (= wrow[i]) with
// neighbour c becomes the record (row c, col x, weight, r).
struct MirrorLoader {
    static constexpr double REC_BYTES = 16.0;  // wcol, wrow, wwt, wrk
    static constexpr int NARR = 4;
    static constexpr uint32_t TILE_WORDS = TT;
    const int32_t* wrow;
    const int32_t* wcol;
    const int32_t* wwt;
    const int32_t* wrk;
    __device__ __forceinline__ const void* tile_src(int a, int64_t tbase) const {
        return (a == 0 ? wcol : (a == 1 ? wrow : (a == 2 ? wwt : wrk))) + tbase;
    }
    __device__ __forceinline__ uint4 srec(const uint32_t* in, int li, int64_t) const {
        return make_uint4(in[li], in[TT + li], in[2 * TT + li], in[3 * TT + li]);
    }
    __device__ __forceinline__ uint4 grec(int64_t i) const {
        return make_uint4((uint32_t)__ldg(wcol + i), (uint32_t)__ldg(wrow + i), (uint32_t)__ldg(wwt + i),
                          (uint32_t)__ldg(wrk + i));
    }
    __device__ __forceinline__ uint32_t key(int64_t i) const { return (uint32_t)__ldg(wcol + i); }
    bool tma_ok() const {
        return (((uintptr_t)wrow | (uintptr_t)wcol | (uintptr_t)wwt | (uintptr_t)wrk) & 15) == 0;
    }
};

// Final row-sorted output: row (optional), col, weight, r.
struct RowsStorer {
    __host__ __device__ double rec_bytes() const { return row ? 16.0 : 12.0; }
    int32_t* row;  // may be null
    int32_t* col;
    int32_t* wt;
    int32_t* rk;
    __device__ __forceinline__ void store(int64_t p, const uint4& r) const {
        if (row) row[p] = (int32_t)r.x;
        col[p] = (int32_t)r.y;
        wt[p] = (int32_t)r.z;
        rk[p] = (int32_t)r.w;
    }
};

__global__ void k_copy_identity_order(int64_t m, const int32_t* u, const int32_t* v,
                                      const int32_t* w, int32_t* ou, int32_t* ov, int32_t* ow) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        ou[i] = u[i];
        ov[i] = v[i];
        ow[i] = w[i];
    }
}

// Row offsets from the row-sorted entry stream: entry i starts row x for
// every x in (row[i-1], row[i]]; rows past the last entry start at n2.
__global__ void k_rowptr_from_rows(int32_t n, int64_t n2, const int32_t* __restrict__ row,
                                   int64_t* __restrict__ rowptr) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t cur = __ldg(row + i);
        const int32_t prev = i == 0 ? -1 : __ldg(row + i - 1);
        for (int32_t x = prev + 1; x <= cur; x++) rowptr[x] = i;
        if (i == n2 - 1)
            for (int64_t x = (int64_t)cur + 1; x <= n; x++) rowptr[x] = n2;
    }
}

constexpr int SHORT_ROW = 32;   // rows below: one thread each
constexpr int LONG_ROW = 1024;  // rows from here: one block each; in between: one warp each

// Degrees (also saturated to 16 bits, the form the orientation test gathers),
// the maximum degree, and the lists of long rows (front of 'rows') and
// medium rows (back of 'rows').  counters: [0] long, [1] next long,
// [2] medium.
__global__ void k_degrees(int32_t n, const int64_t* __restrict__ rowptr, int32_t* __restrict__ deg,
                          uint16_t* __restrict__ deg16, BuildStatus* st, int32_t* rows,
                          int32_t* counters) {
    int32_t mx = 0;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x) {
        const int32_t d = (int32_t)(rowptr[x + 1] - rowptr[x]);
        deg[x] = d;
        deg16[x] = (uint16_t)min(d, 0xffff);
        mx = max(mx, d);
        // one atomic per warp and list
        const uint32_t act = __activemask();
        const int lane = threadIdx.x & 31;
        const uint32_t bl = __ballot_sync(act, d >= LONG_ROW);
        const uint32_t bm = __ballot_sync(act, d >= SHORT_ROW && d < LONG_ROW);
        const int leader = __ffs(act) - 1;
        int32_t base_l = 0, base_m = 0;
        if (lane == leader) {
            if (bl) base_l = atomicAdd(&counters[0], __popc(bl));
            if (bm) base_m = atomicAdd(&counters[2], __popc(bm));
        }
        base_l = __shfl_sync(act, base_l, leader);
        base_m = __shfl_sync(act, base_m, leader);
        const uint32_t below = (1u << lane) - 1u;
        if (d >= LONG_ROW) rows[base_l + __popc(bl & below)] = (int32_t)x;
        else if (d >= SHORT_ROW) rows[n - 1 - (base_m + __popc(bm & below))] = (int32_t)x;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0 && mx) atomicMax(&st->maxdeg, mx);
}

// Whether x (degree dx) comes before its neighbour c in the (degree, id)
// order.  The 16-bit degrees decide unless both saturate.
__device__ __forceinline__ bool before(int32_t x, int32_t dx, const uint16_t* __restrict__ deg16,
                                       const int32_t* __restrict__ deg, int32_t c) {
    uint32_t dc = __ldg(deg16 + c);
    if (dx >= 0xffff) {
        if (dc < 0xffffu) return false;
        dc = (uint32_t)__ldg(deg + c);
    }
    return (uint32_t)dx < dc || ((uint32_t)dx == dc && x < c);
}

constexpr int OBLK = 512;

// Degree orientation, in the slots of the symmetric rows: row x keeps its
// neighbours of higher (degree, id) rank, in id order, at
// [rowptr[x], rowptr[x] + odeg[x]).  The same pass finds repeated pairs
// (equal neighbours next to each other in an id-sorted row).
//
// Every pass loads an entry's id, weight and rank together (the weight and
// rank of a dropped entry are read but unused), so the only dependent load
// is the neighbour's degree.
//
// Short rows: one thread per row walks its entries, eight at a time.
__global__ void k_orient_short(int32_t n, const int64_t* __restrict__ rowptr,
                               const int32_t* __restrict__ scol, const int32_t* __restrict__ swt,
                               const int32_t* __restrict__ srk, const uint16_t* __restrict__ deg16,
                               const int32_t* __restrict__ deg, int32_t* __restrict__ ocol,
                               int32_t* __restrict__ owt, int32_t* __restrict__ ork,
                               int32_t* __restrict__ odeg, BuildStatus* st) {
    constexpr int B = 8;
    unsigned long long dup = ~0ull;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = rowptr[x], e = rowptr[x + 1];
        const int32_t dx = (int32_t)(e - s);
        if (dx >= SHORT_ROW) continue;
        int64_t out = s;
        int32_t prev = -1;
        for (int64_t j0 = s; j0 < e; j0 += B) {
            int32_t c[B], wv[B], rv[B];
            bool f[B];
#pragma unroll
            for (int i = 0; i < B; i++) {
                const bool ok = j0 + i < e;
                c[i] = ok ? __ldcs(scol + j0 + i) : -1;
                wv[i] = ok ? __ldcs(swt + j0 + i) : 0;
                rv[i] = ok ? __ldcs(srk + j0 + i) : 0;
            }
#pragma unroll
            for (int i = 0; i < B; i++) f[i] = c[i] >= 0 && before((int32_t)x, dx, deg16, deg, c[i]);
#pragma unroll
            for (int i = 0; i < B; i++) {
                if (c[i] < 0) break;
                if (c[i] == prev) dup = min(dup, (unsigned long long)(j0 + i));
                prev = c[i];
                if (f[i]) {
                    ocol[out] = c[i];
                    owt[out] = wv[i];
                    ork[out] = rv[i];
                    out++;
                }
            }
        }
        odeg[x] = (int32_t)(out - s);
    }
    if (dup != ~0ull) {
        atomicOr(&st->err, DEV_ERR_DUPLICATE);
        atomicMin(&st->first_bad, dup);
    }
}

// Long rows: blocks take them from a queue; then medium rows: warp i takes
// entries i, i + warps, ... of their list, four 32-entry chunks at a time.
__global__ void __launch_bounds__(OBLK) k_orient(
    int32_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ scol,
    const int32_t* __restrict__ swt, const int32_t* __restrict__ srk,
    const uint16_t* __restrict__ deg16, const int32_t* __restrict__ deg, int32_t* __restrict__ ocol,
    int32_t* __restrict__ owt, int32_t* __restrict__ ork, int32_t* __restrict__ odeg,
    const int32_t* __restrict__ rows, int32_t* counters, BuildStatus* st) {
    __shared__ uint32_t warp_cnt[OBLK / 32];
    __shared__ uint32_t tot;
    __shared__ int32_t item;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t below = (1u << lane) - 1u;
    unsigned long long dup = ~0ull;
    const int nlong = counters[0];
    for (;;) {
        if (threadIdx.x == 0) item = atomicAdd(&counters[1], 1);
        __syncthreads();
        const int it = item;
        __syncthreads();
        if (it >= nlong) break;
        const int32_t x = rows[it];
        const int64_t s = rowptr[x], e = rowptr[x + 1];
        const int32_t dx = (int32_t)(e - s);
        int64_t out = s;
        for (int64_t j0 = s; j0 < e; j0 += OBLK) {
            const int64_t j = j0 + threadIdx.x;
            bool fwd = false;
            int32_t c = 0, wv = 0, rv = 0, cp = -1;
            if (j < e) {
                c = __ldcs(scol + j);
                wv = __ldcs(swt + j);
                rv = __ldcs(srk + j);
                if (j > s) cp = __ldg(scol + j - 1);
            }
            if (j < e) {
                if (cp == c) dup = min(dup, (unsigned long long)j);
                fwd = before(x, dx, deg16, deg, c);
            }
            const uint32_t b = __ballot_sync(0xffffffffu, fwd);
            if (lane == 0) warp_cnt[wid] = __popc(b);
            __syncthreads();
            if (threadIdx.x == 0) {
                uint32_t acc = 0;
                for (int k = 0; k < OBLK / 32; k++) {
                    const uint32_t t = warp_cnt[k];
                    warp_cnt[k] = acc;
                    acc += t;
                }
                tot = acc;
            }
            __syncthreads();
            if (fwd) {
                const int64_t p = out + warp_cnt[wid] + __popc(b & below);
                ocol[p] = c;
                owt[p] = wv;
                ork[p] = rv;
            }
            out += tot;
            __syncthreads();
        }
        if (threadIdx.x == 0) odeg[x] = (int32_t)(out - s);
    }
    constexpr int CH = 4;
    const int nmed = counters[2];
    const int64_t nwarps = ((int64_t)gridDim.x * OBLK) >> 5;
    for (int64_t it = ((int64_t)blockIdx.x * OBLK + threadIdx.x) >> 5; it < nmed; it += nwarps) {
        const int32_t x = rows[n - 1 - it];
        const int64_t s = rowptr[x], e = rowptr[x + 1];
        const int32_t dx = (int32_t)(e - s);
        int64_t out = s;
        int32_t carry = -1;  // id of the entry before the current chunk
        for (int64_t j0 = s; j0 < e; j0 += 32 * CH) {
            int32_t c[CH], wv[CH], rv[CH];
            bool f[CH];
#pragma unroll
            for (int i = 0; i < CH; i++) {
                const int64_t j = j0 + 32 * i + lane;
                const bool ok = j < e;
                c[i] = ok ? __ldcs(scol + j) : -1;
                wv[i] = ok ? __ldcs(swt + j) : 0;
                rv[i] = ok ? __ldcs(srk + j) : 0;
            }
#pragma unroll
            for (int i = 0; i < CH; i++) f[i] = c[i] >= 0 && before(x, dx, deg16, deg, c[i]);
#pragma unroll
            for (int i = 0; i < CH; i++) {
                const int32_t up = __shfl_up_sync(0xffffffffu, c[i], 1);
                const int32_t pc = lane == 0 ? carry : up;
                const int64_t j = j0 + 32 * i + lane;
                if (c[i] >= 0 && pc == c[i]) dup = min(dup, (unsigned long long)j);
                carry = __shfl_sync(0xffffffffu, c[i], 31);
                const uint32_t b = __ballot_sync(0xffffffffu, f[i]);
                if (f[i]) {
                    const int64_t p = out + __popc(b & below);
                    ocol[p] = c[i];
                    owt[p] = wv[i];
                    ork[p] = rv[i];
                }
                out += __popc(b);
            }
        }
        if (lane == 0) odeg[x] = (int32_t)(out - s);
    }
    if (dup != ~0ull) {
        atomicOr(&st->err, DEV_ERR_DUPLICATE);
        atomicMin(&st->first_bad, dup);  // entry index of the repeat
    }
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Graphs and scratch come from the device's stream-ordered pool; keep freed
// blocks in the pool (no release at synchronization) so that rebuilding a
// graph of the same size reuses memory instead of paying for cudaMalloc.
void keep_pool_memory(int dev) {
    static int done_mask = 0;  // benign race: the attribute write is idempotent
    if (dev < 0 || dev >= 31 || (done_mask >> dev) & 1) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    done_mask |= 1 << dev;
}

}  // namespace

int exclusive_scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, cudaStream_t s) {
    // out has n+1 entries; out[n] = total.
    const int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    int64_t* tile_sums = nullptr;
    WTRI_CUDA(cudaMallocAsync((void**)&tile_sums, sizeof(int64_t) * (size_t)std::max<int64_t>(tiles, 1), s));
    if (tiles > 0) {
        ProfScope ps("scan_offsets", s, 4.0 * n * 2 + 8.0 * (n + 1), 3);
        k_scan_reduce<<<(unsigned)tiles, BLK, 0, s>>>(in, n, tile_sums, nullptr);
        k_scan_tiles<<<1, BLK, 0, s>>>(tile_sums, tiles, out + n);
        k_scan_apply<<<(unsigned)tiles, BLK, 0, s>>>(in, n, tile_sums, out);
    } else {
        WTRI_CUDA(cudaMemsetAsync(out, 0, sizeof(int64_t), s));
    }
    WTRI_CUDA(cudaGetLastError());
    WTRI_CUDA(cudaFreeAsync(tile_sums, s));
    return WTRI_OK;
}

namespace {

struct Scratch {
    cudaStream_t s;
    void* p = nullptr;
    explicit Scratch(cudaStream_t st) : s(st) {}
    ~Scratch() {
        if (p) cudaFreeAsync(p, s);
    }
};

unsigned grid_for(int64_t work, int per_block = BLK) {
    int64_t g = (work + per_block - 1) / per_block;
    const int64_t cap = (int64_t)sm_count() * 16;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (unsigned)g;
}

}  // namespace

int build_graph(int32_t n, int64_t m, const int32_t* u_in, const int32_t* v_in,
                const int32_t* w_in, int on_device, cudaStream_t s, wtri_graph** out) {
    *out = nullptr;
    if (n <= 0) return set_error(WTRI_EINVAL, "n must be positive");
    if (m < 0) return set_error(WTRI_EINVAL, "m must be non-negative");
    if (m > (int64_t(1) << 30)) return set_error(WTRI_EUNSUPPORTED, "m above 2^30 edges");
    if (m > 0 && (!u_in || !v_in || !w_in)) return set_error(WTRI_EINVAL, "null edge arrays");

    int dev = 0;
    WTRI_CUDA(cudaGetDevice(&dev));
    keep_pool_memory(dev);

    // Inputs on the device.
    Scratch in_buf(s);
    const int32_t *u = u_in, *v = v_in, *w = w_in;
    if (!on_device && m > 0) {
        WTRI_CUDA(cudaMallocAsync(&in_buf.p, sizeof(int32_t) * 3 * (size_t)m, s));
        int32_t* d = (int32_t*)in_buf.p;
        WTRI_CUDA(cudaMemcpyAsync(d, u_in, sizeof(int32_t) * m, cudaMemcpyHostToDevice, s));
        WTRI_CUDA(cudaMemcpyAsync(d + m, v_in, sizeof(int32_t) * m, cudaMemcpyHostToDevice, s));
        WTRI_CUDA(cudaMemcpyAsync(d + 2 * m, w_in, sizeof(int32_t) * m, cudaMemcpyHostToDevice, s));
        u = d;
        v = d + m;
        w = d + 2 * m;
    }

    // One allocation for every resident array (256-byte aligned pieces, with
    // 16 bytes of slack after each so bulk copies may round sizes up).
    const size_t N1 = (size_t)n, M = (size_t)m, M2 = 2 * (size_t)m;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align_up(off + bytes + 16, 256);
        return o;
    };
    const size_t o_deg = take(4 * N1), o_odeg = take(4 * N1);
    const size_t o_rowptr = take(8 * (N1 + 1));
    const size_t o_ou = take(4 * M), o_ov = take(4 * M), o_ow = take(4 * M);
    const size_t o_wcol = take(4 * M2), o_wwt = take(4 * M2), o_wrk = take(4 * M2);
    const size_t o_scol = take(4 * M2), o_swt = take(4 * M2), o_srk = take(4 * M2);
    const size_t o_ocol = take(4 * M2), o_owt = take(4 * M2), o_ork = take(4 * M2);
    const size_t total = off;

    wtri_graph* g = new (std::nothrow) wtri_graph();
    if (!g) return set_error(WTRI_ENOMEM, "host allocation failed");
    g->stream = s;
    g->device = dev;
    g->bytes = (int64_t)total;
    cudaError_t e = cudaMallocAsync(&g->base, total, s);
    if (e != cudaSuccess) {
        delete g;
        cudaGetLastError();
        return set_error(WTRI_ENOMEM, "device allocation of " + std::to_string(total) + " bytes failed");
    }
    char* B = (char*)g->base;
    int32_t* deg = (int32_t*)(B + o_deg);
    int32_t* odeg = (int32_t*)(B + o_odeg);
    int64_t* rowptr = (int64_t*)(B + o_rowptr);
    int32_t *ou = (int32_t*)(B + o_ou), *ov = (int32_t*)(B + o_ov), *ow = (int32_t*)(B + o_ow);
    int32_t *wcol = (int32_t*)(B + o_wcol), *wwt = (int32_t*)(B + o_wwt), *wrk = (int32_t*)(B + o_wrk);
    int32_t *scol = (int32_t*)(B + o_scol), *swt = (int32_t*)(B + o_swt), *srk = (int32_t*)(B + o_srk);
    int32_t *ocol = (int32_t*)(B + o_ocol), *owt = (int32_t*)(B + o_owt), *ork = (int32_t*)(B + o_ork);

    auto fail = [&](int rc) {
        cudaFreeAsync(g->base, s);
        cudaStreamSynchronize(s);
        delete g;
        return rc;
    };

    BuildStatus* d_st = nullptr;
    BuildStatus h_st;
    Scratch st_buf(s);
    if (cudaMallocAsync(&st_buf.p, sizeof(BuildStatus), s) != cudaSuccess)
        return fail(set_error(WTRI_ENOMEM, "status allocation failed"));
    d_st = (BuildStatus*)st_buf.p;
    {
        BuildStatus init = {0u, 0, 0, 0, ~0ull};
        if (cudaMemcpyAsync(d_st, &init, sizeof(init), cudaMemcpyHostToDevice, s) != cudaSuccess)
            return fail(cuda_error(cudaGetLastError(), "status init", __FILE__, __LINE__));
    }

    // 1. validation + max weight
    if (m > 0) {
        ProfScope ps("validate", s, 12.0 * m, 1);
        k_validate<<<grid_for(m), BLK, 0, s>>>(n, m, u, v, w, d_st);
    }
    if (cudaMemcpyAsync(&h_st, d_st, sizeof(h_st), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return fail(cuda_error(cudaGetLastError(), "validation", __FILE__, __LINE__));
    if (h_st.err) {
        std::string what = (h_st.err & DEV_ERR_RANGE) ? "vertex id outside [0, n)"
                           : (h_st.err & DEV_ERR_SELF_LOOP) ? "self-loop"
                                                            : "non-positive weight";
        return fail(set_error(WTRI_EINVAL, "invalid edge " + std::to_string(h_st.first_bad) +
                                               ": " + what));
    }
    g->d.n = n;
    g->d.m = m;
    g->d.wmax = h_st.wmax;
    g->d.maxdeg = 0;

    if (m > 0) {
        // Scratch: two buffers of 16-byte records and one of 16-bit digits for
        // 2m records, the radix counts, the row keys of the weight-sorted
        // layout, long rows.
        const int64_t n2 = 2 * m;
        const size_t rec_words = 4 * (size_t)n2 + 4;
        const size_t dig_words = ((size_t)n2 + 1) / 2 + 4;
        const size_t cnt_words = radix::scratch_words(n2);
        const size_t words = 2 * rec_words + dig_words + cnt_words + (size_t)n2 + N1 + 8 + (N1 + 1) / 2 + 4;
        Scratch tmp(s);
        if (cudaMallocAsync(&tmp.p, words * 4, s) != cudaSuccess) {
            cudaGetLastError();
            return fail(set_error(WTRI_ENOMEM, "device scratch allocation failed"));
        }
        uint4* rec_a = (uint4*)tmp.p;
        uint4* rec_b = rec_a + rec_words / 4;
        uint16_t* dig = (uint16_t*)(rec_b + rec_words / 4);
        uint32_t* counts = (uint32_t*)dig + dig_words;
        int32_t* wrow = (int32_t*)(counts + cnt_words);
        int32_t* row_list = wrow + n2;                    // long rows first, medium rows last
        int32_t* row_counters = row_list + n;             // 8 words, see k_degrees
        uint16_t* deg16 = (uint16_t*)(row_counters + 8);  // n half-words
        if (cudaMemsetAsync(row_counters, 0, 32, s) != cudaSuccess)
            return fail(cuda_error(cudaGetLastError(), "memset", __FILE__, __LINE__));

        // 2. edge order
        const int wbits = radix::bit_length((uint64_t)(h_st.wmax - 1));
        if (wbits == 0) {
            ProfScope ps("edge_order_copy", s, 24.0 * m, 1);
            k_copy_identity_order<<<grid_for(m), BLK, 0, s>>>(m, u, v, w, ou, ov, ow);
        } else {
            EdgeLoader el{u, v, w, h_st.wmax};
            EdgeOrderStorer es{ou, ov, ow, h_st.wmax};
            int rc = radix::lsd_sort(el, es, m, wbits, rec_a, rec_b, dig, counts, s, &d_st->err);
            if (rc != WTRI_OK) return fail(rc);
        }
        // 3. weight-sorted rows (row key kept in wrow)
        const int nbits = std::max(1, radix::bit_length((uint64_t)(n - 1)));
        {
            OrderEntryLoader ol{ou, ov, ow};
            RowsStorer rs{wrow, wcol, wwt, wrk};
            int rc = radix::lsd_sort(ol, rs, n2, nbits, rec_a, rec_b, dig, counts, s, &d_st->err);
            if (rc != WTRI_OK) return fail(rc);
        }
        // 4. row offsets, degrees, long rows
        {
            ProfScope ps("row_offsets", s, 4.0 * n2 + 8.0 * (n + 1) + 4.0 * n, 2);
            k_rowptr_from_rows<<<grid_for(n2), BLK, 0, s>>>(n, n2, wrow, rowptr);
            k_degrees<<<grid_for(n), BLK, 0, s>>>(n, rowptr, deg, deg16, d_st, row_list, row_counters);
        }
        // 5. id-sorted rows
        {
            MirrorLoader ml{wrow, wcol, wwt, wrk};
            RowsStorer rs{nullptr, scol, swt, srk};
            int rc = radix::lsd_sort(ml, rs, n2, nbits, rec_a, rec_b, dig, counts, s, &d_st->err);
            if (rc != WTRI_OK) return fail(rc);
        }
        // 6. orientation + repeated pairs
        {
            {
                ProfScope ps("orient_short", s, 0.0, 1);
                k_orient_short<<<grid_for(n), BLK, 0, s>>>(n, rowptr, scol, swt, srk, deg16, deg, ocol,
                                                           owt, ork, odeg, d_st);
            }
            // reads every id-sorted neighbour, weight and rank, writes m
            // oriented entries and the out-degrees (bytes of both launches)
            ProfScope ps("orient", s, 12.0 * n2 + 12.0 * m + 4.0 * n + 8.0 * (n + 1), 1);
            // persistent: as many blocks as fit at once (rows are dealt by block and warp index)
            static int per_sm = 0;
            if (per_sm == 0 &&
                (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_orient, OBLK, 0) != cudaSuccess ||
                 per_sm < 1))
                per_sm = 1;
            k_orient<<<sm_count() * per_sm, OBLK, 0, s>>>(n, rowptr, scol, swt, srk, deg16, deg, ocol,
                                                          owt, ork, odeg, row_list, row_counters, d_st);
        }
        if (cudaGetLastError() != cudaSuccess)
            return fail(set_error(WTRI_ECUDA, "build kernel launch failed"));
        if (cudaMemcpyAsync(&h_st, d_st, sizeof(h_st), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return fail(cuda_error(cudaGetLastError(), "build", __FILE__, __LINE__));
        if (h_st.err & DEV_ERR_TIMEOUT)
            return fail(set_error(WTRI_ETIMEOUT, "a bounded wait in the radix sort ran out"));
        if (h_st.err & DEV_ERR_DUPLICATE) {
            int32_t col[2] = {-1, -1};
            const int64_t j = (int64_t)h_st.first_bad;
            cudaMemcpyAsync(&col[0], scol + j, 4, cudaMemcpyDeviceToHost, s);
            cudaStreamSynchronize(s);
            return fail(set_error(WTRI_EINVAL, "repeated undirected pair: neighbour " +
                                                   std::to_string(col[0]) +
                                                   " appears twice in one row"));
        }
        g->d.maxdeg = h_st.maxdeg;
    } else {
        if (cudaMemsetAsync(rowptr, 0, 8 * (N1 + 1), s) != cudaSuccess ||
            cudaMemsetAsync(deg, 0, 4 * N1, s) != cudaSuccess ||
            cudaMemsetAsync(odeg, 0, 4 * N1, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return fail(cuda_error(cudaGetLastError(), "build", __FILE__, __LINE__));
    }

    g->d.deg = deg;
    g->d.odeg = odeg;
    g->d.rowptr = rowptr;
    g->d.ord_u = ou;
    g->d.ord_v = ov;
    g->d.ord_w = ow;
    g->d.wcol = wcol;
    g->d.wwt = wwt;
    g->d.wrk = wrk;
    g->d.scol = scol;
    g->d.swt = swt;
    g->d.srk = srk;
    g->d.ocol = ocol;
    g->d.owt = owt;
    g->d.ork = ork;
    *out = g;
    return WTRI_OK;
}

}  // namespace wtri
