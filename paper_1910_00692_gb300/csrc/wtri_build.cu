// Device graph build: validation, degrees, the edge order, per-vertex
// weight-sorted lists and the degree-oriented id-sorted lists.
//
// Preprocessing named by the paper: "Sort E in decreasing order of weight"
// (Algorithm 2, first step), neighbour sets N(a) and degrees d_a (Section
// 4), and the NodeIterator++ degree ordering (Section 5.2).
//
// Pipeline (one stream, inputs read once from HBM or host; no host round
// trip until the end: every kernel after validation reads the device status
// word and returns at once if an earlier step failed):
//   1. k_validate: rejects bad edges, finds the max weight.
//   2. Edge order: stable LSD radix sort of key ~w carrying (u, v), planned
//      for 31-bit weights; the passes above the max weight's bit length
//      skip themselves on the device.
//   3. Weight-sorted lists: the virtual stream "two entries per edge, in edge
//      order" is stably radix-sorted by row, so each row keeps edge order.
//   4. Row offsets and degrees from the boundaries of the sorted rows (no
//      atomics).
//   5. Orientation of every entry (neighbour of higher (degree, id) rank),
//      the oriented out-degrees and their scan (the oriented row offsets);
//      per-row segmented sort of the forward entries by neighbour id
//      (wtri_rows.cuh): the oriented rows, and repeated pairs (equal
//      neighbours next to each other in one oriented row).
#include <cuda_runtime.h>
#include <stdio.h>

#include <algorithm>
#include <cmath>
#include <string>

#include "wtri_internal.cuh"
#include "wtri_radix.cuh"
#include "wtri_rows.cuh"

namespace wtri {

namespace {

constexpr int BLK = 256;

struct BuildStatus {
    uint32_t err;
    int32_t wmax;
    int32_t maxdeg;
    int32_t pad;
    unsigned long long first_bad;  // smallest offending edge index; for a repeated
                                   // pair, the smallest x << 32 | c of its oriented row
};

// Float weights (fw): positive finite fp32 values, whose bit patterns are
// the positive int32 below 0x7f800000 (+inf; NaN lies above it).
struct ValidateAcc {
    int32_t wmax = 0;
    uint32_t err = 0;
    unsigned long long bad = ~0ull;
    __device__ __forceinline__ void edge(int32_t n, int fw, int64_t i, int32_t a, int32_t b, int32_t x) {
        uint32_t e = 0;
        if (a < 0 || a >= n || b < 0 || b >= n) e |= DEV_ERR_RANGE;
        else if (a == b) e |= DEV_ERR_SELF_LOOP;
        if (x <= 0 || (fw && x >= 0x7f800000)) e |= DEV_ERR_WEIGHT;
        if (e) {
            err |= e;
            if ((unsigned long long)i < bad) bad = (unsigned long long)i;
            return;
        }
        wmax = max(wmax, x);
    }
};

// VEC: the three arrays are 16-byte aligned; four edges per 16-byte load of
// each (enough bytes in flight to stream the input at HBM rate), the last
// m % 4 edges one by one.
template <bool VEC>
__global__ void k_validate(int32_t n, int64_t m, const int32_t* __restrict__ u,
                           const int32_t* __restrict__ v, const int32_t* __restrict__ w,
                           int fw, BuildStatus* st) {
    ValidateAcc acc;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    const int64_t nq = VEC ? m / 4 : 0;
    for (int64_t q = tid; q < nq; q += nth) {
        const int4 a = __ldg(reinterpret_cast<const int4*>(u) + q);
        const int4 b = __ldg(reinterpret_cast<const int4*>(v) + q);
        const int4 x = __ldg(reinterpret_cast<const int4*>(w) + q);
        acc.edge(n, fw, 4 * q, a.x, b.x, x.x);
        acc.edge(n, fw, 4 * q + 1, a.y, b.y, x.y);
        acc.edge(n, fw, 4 * q + 2, a.z, b.z, x.z);
        acc.edge(n, fw, 4 * q + 3, a.w, b.w, x.w);
    }
    for (int64_t i = 4 * nq + tid; i < m; i += nth) acc.edge(n, fw, i, __ldg(u + i), __ldg(v + i), __ldg(w + i));
    int32_t wloc = acc.wmax;
    uint32_t eloc = acc.err;
    unsigned long long bad = acc.bad;
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

// Edge order input: key ~w (ascending key = weight descending), values (u, v).
struct EdgeLoader {
    static constexpr double REC_BYTES = 12.0;  // u, v, w
    static constexpr int NARR = 3;             // w, u, v
    static constexpr uint32_t TILE_WORDS = TT;
    const int32_t* u;
    const int32_t* v;
    const int32_t* w;
    __device__ __forceinline__ uint32_t key(int64_t i) const { return ~(uint32_t)__ldg(w + i); }
    __device__ __forceinline__ const void* tile_src(int a, int64_t tbase) const {
        return (a == 0 ? w : (a == 1 ? u : v)) + tbase;
    }
    __device__ __forceinline__ uint4 srec(const uint32_t* in, int li, int64_t) const {
        return make_uint4(~in[li], in[TT + li], in[2 * TT + li], 0u);
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
    __device__ __forceinline__ void prepare() {}
    __device__ __forceinline__ void store(int64_t p, const uint4& r) const {
        ow[p] = (int32_t)~r.x;
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

// Final row-sorted output: row, col, weight, r.
struct RowsStorer {
    __host__ __device__ double rec_bytes() const { return 16.0; }
    int32_t* row;
    int32_t* col;
    int32_t* wt;
    int32_t* rk;
    __device__ __forceinline__ void prepare() {}
    __device__ __forceinline__ void store(int64_t p, const uint4& r) const {
        row[p] = (int32_t)r.x;
        col[p] = (int32_t)r.y;
        wt[p] = (int32_t)r.z;
        rk[p] = (int32_t)r.w;
    }
};

// Row offsets from the row-sorted entry stream: entry i starts row x for
// every x in (row[i-1], row[i]]; rows past the last entry start at n2.
// Rows start where the sorted row keys change.  Eight keys per thread from
// two 16-byte loads (row is 16-byte aligned), the key before them from the
// previous group.
__global__ void k_rowptr_from_rows(int32_t n, int64_t n2, const int32_t* __restrict__ row,
                                   int64_t* __restrict__ rowptr, const uint32_t* gate) {
    if (*(volatile const uint32_t*)gate) return;
    constexpr int G = 8;
    const int64_t ng = (n2 + G - 1) / G;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < ng;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i0 = G * q;
        int32_t cur[G];
        if (i0 + G <= n2) {
            const int4 r0 = __ldg(reinterpret_cast<const int4*>(row) + 2 * q);
            const int4 r1 = __ldg(reinterpret_cast<const int4*>(row) + 2 * q + 1);
            cur[0] = r0.x;
            cur[1] = r0.y;
            cur[2] = r0.z;
            cur[3] = r0.w;
            cur[4] = r1.x;
            cur[5] = r1.y;
            cur[6] = r1.z;
            cur[7] = r1.w;
        } else {
#pragma unroll
            for (int t = 0; t < G; t++) cur[t] = i0 + t < n2 ? __ldg(row + i0 + t) : n;
        }
        int32_t prev = q == 0 ? -1 : __ldg(row + i0 - 1);
#pragma unroll
        for (int t = 0; t < G; t++) {
            // past the end the key is n: rows after the last key start at n2
            const int64_t i = i0 + t < n2 ? i0 + t : n2;
            for (int64_t x = (int64_t)prev + 1; x <= cur[t]; x++) rowptr[x] = i;
            prev = max(prev, cur[t]);
        }
        if (i0 + G == n2)
            for (int64_t x = (int64_t)prev + 1; x <= n; x++) rowptr[x] = n2;
    }
}
__global__ void k_degrees(int32_t n, const int64_t* __restrict__ rowptr, uint16_t* __restrict__ deg16,
                          BuildStatus* st) {
    if (*(volatile const uint32_t*)&st->err) return;
    int32_t mx = 0;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t d = rowptr[x + 1] - rowptr[x];
        deg16[x] = (uint16_t)min(d, (int64_t)rows::DEG_SAT);
        mx = max(mx, (int32_t)min(d, (int64_t)INT32_MAX));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0 && mx) atomicMax(&st->maxdeg, mx);
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
        ProfScope ps("scan_offsets", s, 0.0, 3, 4.0 * n * 2 + 8.0 * (n + 1));
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

// Per-row sorts (wtri_rows.cuh): launches of every size class, each under its
// own phase timer (the bytes of the whole step are declared by the caller).
// g0/g1: the hub rows' runs (8 bytes per entry each).  max_deg_bound: an
// upper bound on any degree (sets the number of hub merge levels launched;
// levels that no row needs return at once).
int sort_rows(const rows::RowsOut& R, unsigned long long* g0, unsigned long long* g1, int32_t* cursor,
              int64_t max_deg_bound, int nbits, const uint32_t* gate, cudaStream_t s) {
    const int sms = sm_count();
    {
        ProfScope ps("rows_sort_small", s, 0.0, 3);
        rows::k_rows_small<8><<<sms * 8, rows::NT, 0, s>>>(R, rows::CLS_G8, gate);
        rows::k_rows_small<16><<<sms * 8, rows::NT, 0, s>>>(R, rows::CLS_G16, gate);
        rows::k_rows_small<32><<<sms * 8, rows::NT, 0, s>>>(R, rows::CLS_G32, gate);
    }
    {
        ProfScope ps("rows_sort_warp", s, 0.0, 4);
        auto launch = [&](auto kern, int epl, int cls) -> int {
            static std::atomic<uint64_t> done[6];
            const int smem = rows::NWARPS * 32 * epl * 16;  // keys + weights + ranks
            int slot = 0;
            for (int e = epl; e > 2; e >>= 1) slot++;
            WTRI_TRY(smem_optin((const void*)kern, smem, done[slot]));
            kern<<<sms * 4, rows::NT, smem, s>>>(R, cls, gate);
            return WTRI_OK;
        };
        WTRI_TRY(launch(rows::k_rows_warp<2>, 2, rows::CLS_W2));
        WTRI_TRY(launch(rows::k_rows_warp<4>, 4, rows::CLS_W4));
        WTRI_TRY(launch(rows::k_rows_warp<8>, 8, rows::CLS_W8));
        WTRI_TRY(launch(rows::k_rows_warp<16>, 16, rows::CLS_W16));
    }
    {
        ProfScope ps("rows_sort_block", s, 0.0, 1);
        static std::atomic<uint64_t> done{0};
        const int smem = (int)sizeof(rows::RadixSmem);
        WTRI_TRY(smem_optin((const void*)rows::k_rows_block, smem, done));
        rows::k_rows_block<<<sms * 2, rows::NT, smem, s>>>(R, g0, cursor, nbits, gate);
    }
    {
        int levels = 0;
        for (int64_t len = rows::SR; len < max_deg_bound; len <<= 1) levels++;
        ProfScope ps("rows_sort_hub", s, 0.0, levels + 1);
        int64_t len = rows::SR;
        for (int l = 0; l < levels; l++, len <<= 1)
            rows::k_rows_merge<<<sms * 4, rows::NT, 0, s>>>(R, (l & 1) ? g1 : g0, (l & 1) ? g0 : g1, len,
                                                            gate);
        rows::k_rows_hub_out<<<sms * 4, rows::NT, 0, s>>>(R, g0, g1, gate);
    }
    WTRI_CUDA(cudaGetLastError());
    return WTRI_OK;
}

}  // namespace

int build_graph(int32_t n, int64_t m, const int32_t* u_in, const int32_t* v_in,
                const int32_t* w_in, int on_device, cudaStream_t s, wtri_graph** out, int fw) {
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
        // each array starts 16-byte aligned (validation loads four edges at once)
        const size_t mp = align_up((size_t)m, 4);
        WTRI_CUDA(cudaMallocAsync(&in_buf.p, sizeof(int32_t) * 3 * mp, s));
        int32_t* d = (int32_t*)in_buf.p;
        WTRI_CUDA(cudaMemcpyAsync(d, u_in, sizeof(int32_t) * m, cudaMemcpyHostToDevice, s));
        WTRI_CUDA(cudaMemcpyAsync(d + mp, v_in, sizeof(int32_t) * m, cudaMemcpyHostToDevice, s));
        WTRI_CUDA(cudaMemcpyAsync(d + 2 * mp, w_in, sizeof(int32_t) * m, cudaMemcpyHostToDevice, s));
        u = d;
        v = d + mp;
        w = d + 2 * mp;
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
    const size_t o_rowptr = take(8 * (N1 + 1)), o_orowptr = take(8 * (N1 + 1));
    const size_t o_ou = take(4 * M), o_ov = take(4 * M), o_ow = take(4 * M);
    const size_t o_wcol = take(4 * M2), o_wwt = take(4 * M2), o_wrk = take(4 * M2);
    const size_t o_ocol = take(4 * M), o_owt = take(4 * M), o_ork = take(4 * M);
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
    int64_t* rowptr = (int64_t*)(B + o_rowptr);
    int64_t* orowptr = (int64_t*)(B + o_orowptr);
    int32_t *ou = (int32_t*)(B + o_ou), *ov = (int32_t*)(B + o_ov), *ow = (int32_t*)(B + o_ow);
    int32_t *wcol = (int32_t*)(B + o_wcol), *wwt = (int32_t*)(B + o_wwt), *wrk = (int32_t*)(B + o_wrk);
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
    if (cudaMallocAsync(&st_buf.p, sizeof(BuildStatus) + 64, s) != cudaSuccess)
        return fail(set_error(WTRI_ENOMEM, "status allocation failed"));
    d_st = (BuildStatus*)st_buf.p;
    {
        static const BuildStatus init = {0u, 0, 0, 0, ~0ull};
        if (cudaMemcpyAsync(d_st, &init, sizeof(init), cudaMemcpyHostToDevice, s) != cudaSuccess)
            return fail(cuda_error(cudaGetLastError(), "status init", __FILE__, __LINE__));
    }
    const uint32_t* gate = &d_st->err;

    // 1. validation + max weight
    if (m > 0) {
        ProfScope ps("validate", s, 12.0 * m, 1);  // the COO input, read once
        if ((((uintptr_t)u | (uintptr_t)v | (uintptr_t)w) & 15) == 0)
            k_validate<true><<<grid_for(m / 4 + 1), BLK, 0, s>>>(n, m, u, v, w, fw, d_st);
        else
            k_validate<false><<<grid_for(m), BLK, 0, s>>>(n, m, u, v, w, fw, d_st);
    }
    g->d.n = n;
    g->d.m = m;
    g->d.fw = fw;
    g->d.wmax = 0;
    g->d.maxdeg = 0;

    if (m > 0) {
        // Scratch: two buffers of 16-byte records and one of 16-bit digits for
        // 2m records (the record buffers are reused by the per-row sort of
        // the longest rows), the radix counts, the row of each weight-sorted
        // entry, 16-bit degrees, oriented out-degrees, the class lists.
        const int64_t n2 = 2 * m;
        const size_t rec_words = 4 * (size_t)n2 + 4;
        // (multiples of four words: wrow below starts 16-byte aligned)
        const size_t dig_words = align_up(((size_t)n2 + 1) / 2 + 4, 4);
        const size_t cnt_words = align_up(radix::scratch_words(n2), 4);
        const size_t words = 2 * rec_words + dig_words + cnt_words + (size_t)n2 + (N1 + 1) / 2 + 4 +
                             N1 + 4 + N1 + 4 + 64;
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
        uint16_t* deg16 = (uint16_t*)(wrow + n2);  // n halfwords
        int32_t* odeg = (int32_t*)(deg16 + 2 * ((N1 + 1) / 2 + 4));
        int32_t* list = odeg + N1 + 4;
        int32_t* small = list + N1 + 4;  // class counts, offsets, fill cursors, block-row cursor
        int32_t* cls_cnt = small;
        int32_t* cls_off = small + 16;
        int32_t* cls_cur = small + 32;
        int32_t* cursor = small + 48;
        static_assert(rows::NCLS + 1 <= 16, "class arrays fit their 16-word slots");
        if (cudaMemsetAsync(small, 0, 64 * 4, s) != cudaSuccess ||
            cudaMemsetAsync(odeg, 0, 4 * N1, s) != cudaSuccess)
            return fail(cuda_error(cudaGetLastError(), "memset", __FILE__, __LINE__));

        // 2. edge order (weights up to 31 bits; passes above the max weight's
        //    bit length skip themselves)
        {
            EdgeLoader el{u, v, w};
            EdgeOrderStorer es{ou, ov, ow};
            // one read + one write of (edge id, weight): 16 B per edge
            int rc = radix::lsd_sort_device_width(el, es, m, 31, &d_st->wmax, rec_a, rec_b, dig, counts,
                                                  s, &d_st->err, 16.0 * m, 2);
            if (rc != WTRI_OK) return fail(rc);
        }
        // 3. weight-sorted rows (row key kept in wrow)
        const int nbits = std::max(1, radix::bit_length((uint64_t)(n - 1)));
        {
            OrderEntryLoader ol{ou, ov, ow};
            RowsStorer rs{wrow, wcol, wwt, wrk};
            // one read + one write of (neighbour, weight, rank): 24 + 24 B per edge
            int rc = radix::lsd_sort(ol, rs, n2, nbits, rec_a, rec_b, dig, counts, s, &d_st->err,
                                     48.0 * m);
            if (rc != WTRI_OK) return fail(rc);
        }
        // 4. row offsets, degrees
        {
            ProfScope ps("row_offsets", s, 8.0 * (n + 1), 2, 4.0 * n2 + 8.0 * (n + 1) + 2.0 * n);
            k_rowptr_from_rows<<<grid_for(n2 / 8 + 1), BLK, 0, s>>>(n, n2, wrow, rowptr, gate);
            k_degrees<<<grid_for(n), BLK, 0, s>>>(n, rowptr, deg16, d_st);
        }
        // 5. orientation of every entry and the oriented out-degrees (the
        //    forward entries' keys packed per row in rec_b), their scan (the
        //    oriented row offsets), the rows' size classes by oriented degree,
        //    then the per-row sort by id writing the oriented rows.  Scratch:
        //    the record buffers, free once the radix sorts are done (g0/g1:
        //    the hub rows' runs, 8 bytes per entry each, in rec_a).
        {
            // reads the weight-sorted rows once; writes the oriented rows
            // (12 B per edge) and their offsets (8 B per vertex)
            ProfScope ps("rows_sort", s, 12.0 * m + 8.0 * (n + 1), 0,
                         8.0 * n2 + n2 + 8.0 * m + 8.0 * m + 8.0 * m + 12.0 * m + 8.0 * (n + 1));
            unsigned long long* g0 = (unsigned long long*)rec_a;
            unsigned long long* g1 = g0 + n2;
            unsigned long long* pk = (unsigned long long*)rec_b;
            {
                ProfScope pf("rows_sort_fwd", s, 0.0, 1);
                rows::k_fwd<<<grid_for(n2, rows::NT), rows::NT, 0, s>>>(n2, wrow, wcol, rowptr, deg16, pk, odeg,
                                                                        gate);
            }
            WTRI_TRY(exclusive_scan_i32_to_i64(odeg, orowptr, n, s));
            {
                ProfScope pc("orient_classes", s, 0.0, 3, 4.0 * n + 8.0 * n);
                const unsigned cg = grid_for(n, rows::NT * rows::CLS_V);
                rows::k_class_count<<<cg, rows::NT, 0, s>>>(n, odeg, cls_cnt, gate);
                rows::k_class_offsets<<<1, 32, 0, s>>>(cls_cnt, cls_off, cls_cur, gate);
                rows::k_class_fill<<<cg, rows::NT, 0, s>>>(n, odeg, cls_cur, list, gate);
            }
            rows::RowsOut R{rowptr, wwt, wrk, pk, odeg, orowptr, ocol, owt, ork,
                            &d_st->err, &d_st->first_bad, list, cls_off};
            // d forward neighbours all have degree >= d: d^2 <= 2m
            int64_t od_max = (int64_t)std::sqrt(2.0 * (double)m) + 1;
            od_max = std::min<int64_t>(od_max, std::min<int64_t>((int64_t)n - 1, m));
            WTRI_TRY(sort_rows(R, g0, g1, cursor, od_max, nbits, gate, s));
        }
        if (cudaGetLastError() != cudaSuccess)
            return fail(set_error(WTRI_ECUDA, "build kernel launch failed"));
    } else {
        if (cudaMemsetAsync(rowptr, 0, 8 * (N1 + 1), s) != cudaSuccess ||
            cudaMemsetAsync(orowptr, 0, 8 * (N1 + 1), s) != cudaSuccess)
            return fail(cuda_error(cudaGetLastError(), "build", __FILE__, __LINE__));
    }
    // The one host round trip: the status of every step.
    if (cudaMemcpyAsync(&h_st, d_st, sizeof(h_st), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return fail(cuda_error(cudaGetLastError(), "build", __FILE__, __LINE__));
    if (h_st.err & (DEV_ERR_RANGE | DEV_ERR_SELF_LOOP | DEV_ERR_WEIGHT)) {
        std::string what = (h_st.err & DEV_ERR_RANGE) ? "vertex id outside [0, n)"
                           : (h_st.err & DEV_ERR_SELF_LOOP) ? "self-loop"
                                                            : (fw ? "weight not a positive finite float"
                                                                  : "non-positive weight");
        return fail(set_error(WTRI_EINVAL, "invalid edge " + std::to_string(h_st.first_bad) +
                                               ": " + what));
    }
    if (h_st.err & DEV_ERR_TIMEOUT)
        return fail(set_error(WTRI_ETIMEOUT, "a bounded wait in the radix sort ran out"));
    if (h_st.err & DEV_ERR_DUPLICATE) {
        const uint64_t pr = (uint64_t)h_st.first_bad;
        return fail(set_error(WTRI_EINVAL, "repeated undirected pair {" + std::to_string((uint32_t)(pr >> 32)) +
                                               ", " + std::to_string((uint32_t)pr) + "}"));
    }
    if (h_st.err) return fail(set_error(WTRI_ECUDA, "internal error in the build"));
    g->d.wmax = h_st.wmax;
    g->d.maxdeg = h_st.maxdeg;
    g->d.rowptr = rowptr;
    g->d.orowptr = orowptr;
    g->d.ord_u = ou;
    g->d.ord_v = ov;
    g->d.ord_w = ow;
    g->d.wcol = wcol;
    g->d.wwt = wwt;
    g->d.wrk = wrk;
    g->d.ocol = ocol;
    g->d.owt = owt;
    g->d.ork = ork;
    *out = g;
    return WTRI_OK;
}

}  // namespace wtri
