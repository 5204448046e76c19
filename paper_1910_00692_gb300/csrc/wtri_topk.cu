// Exact top-k query, weighted edge sampling and the allocation-free query:
// host orchestration of the kernels in wtri_query.cuh.
#include "wtri_query.cuh"

#include <mutex>

namespace wtri {
namespace {

// First-wait poll limit of the long-scan kernel's row staging (a test hook
// lowers it; see wtri_debug_set_wait_limit).
std::atomic<uint32_t> g_stage_wait{WAIT_LIMIT};
uint32_t stage_wait_limit() { return g_stage_wait.load(std::memory_order_relaxed); }

template <int P>
int run_query(const wtri_graph* g, int32_t k, wtri_tri* d_tris, double* d_weight, int32_t* d_count,
              cudaStream_t s, int scale, int shard, int nshards, unsigned long long* d_keys,
              double gp) {
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
    q.long_count = &q.st->long_count;
    q.qid = 0;
    q.shard = shard;
    q.nshards = nshards;
    q.t_short = g->tune.t_short;
    q.qbytes = query_bytes_on() ? query_bytes_counter() : nullptr;
    q.gp = gp;
    q.fw = g->d.fw;
    q.wait_first = stage_wait_limit();
    WTRI_CUDA(cudaMemsetAsync(q.st, 0, sizeof(QState), s));

    const size_t lsmem = LONG_SMEM;
    WTRI_TRY((long_optin<P, false>()));
    const int long_grid = sm_count() * 2;
    ProfScope whole(query_name(P), s, 0.0, 0);
    // p = -inf on one shard: NodeIterator++ rounds (no deferred scans)
    const bool oriented = P == P_MIN && nshards == 1;
    int64_t lo = 0, size = g->tune.first_round;
    while (lo < m) {
        const int64_t hi = std::min(m, lo + size);
        if (oriented) {
            ProfScope ps("topk_round_min", s, 0.0, 1);
            k_round_min<<<round_grid_warps(hi - lo), RBLK, 0, s>>>(G, q, lo, hi);
        } else {
            {
                ProfScope ps("topk_round", s, 0.0, 1);
                if (hi - lo <= WARP_ROUND_MAX)  // small early rounds: a warp per edge
                    k_round_warp<P><<<round_grid_warps(hi - lo), RBLK, 0, s>>>(G, q, lo, hi);
                else
                    k_round<P><<<round_grid(hi - lo), RBLK, 0, s>>>(G, q, lo, hi);
            }
            {
                ProfScope ps("topk_long", s, 0.0, 1);
                k_long<P><<<long_grid, LBLK, lsmem, s>>>(G, q);
            }
        }
        {
            ProfScope ps("topk_select", s, 0.0, 1);
            k_select<<<1, SBLK, 0, s>>>(q);
        }
        lo = hi;
        size *= g->tune.growth;
    }
    {
        ProfScope ps("topk_final", s, 0.0, 2);
        k_final_select<<<1, SBLK, 0, s>>>(q);
        k_rank_scatter<P><<<ceil_div_u(std::max(k, 1), 8), 256, 0, s>>>(q, d_tris, d_weight, d_count,
                                                                        d_keys);
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
            // w^p: p = 2 squares, p = 1 keeps, p = 0 gives 1 (uniform draws)
            x = (u128)(uint64_t)(cstart[c + 1] - cstart[c]) *
                (P == P_TWO ? wv * wv : (P == P_GEO ? (u128)1 : wv));
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
        const u128 wp = P == P_TWO ? wv * wv : (P == P_GEO ? (u128)1 : wv);
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
    q.long_count = &q.st->long_count;
    q.qid = 0;
    q.shard = 0;
    q.nshards = 1;
    q.t_short = g->tune.t_short;
    q.qbytes = nullptr;
    q.gp = 0.0;
    q.fw = 0;
    q.wait_first = stage_wait_limit();
    WTRI_CUDA(cudaMemsetAsync(q.st, 0, sizeof(QState), s));
    ProfScope whole(P == P_ONE ? "sample_p=1" : (P == P_TWO ? "sample_p=2" : "sample_p=0"), s, 0.0, 0);
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
    const size_t lsmem = LONG_SMEM;
    WTRI_TRY((long_optin<P, true>()));
    const int long_grid = sm_count() * 2;
    int64_t lo = 0, size = g->tune.first_round;
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
        size *= g->tune.growth;
    }
    {
        ProfScope ps("topk_final", s, 0.0, 2);
        k_final_select<<<1, SBLK, 0, s>>>(q);
        k_rank_scatter<P><<<ceil_div_u(std::max(k, 1), 8), 256, 0, s>>>(q, d_tris, d_weight, d_count,
                                                                    nullptr);
    }
    WTRI_CUDA(cudaGetLastError());
    WTRI_CUDA(cudaFreeAsync(buf, s));
    return WTRI_OK;
}

}  // namespace

int topk_device(const wtri_graph* g, int pcode, int32_t k, wtri_tri* d_tris, double* d_weight,
                int32_t* d_count, cudaStream_t stream, int retry_scale, int shard, int nshards,
                unsigned long long* d_keys, double gp) {
    switch (pcode) {
        case P_MIN:
            return run_query<P_MIN>(g, k, d_tris, d_weight, d_count, stream, retry_scale, shard, nshards, d_keys, gp);
        case P_ONE:
            return run_query<P_ONE>(g, k, d_tris, d_weight, d_count, stream, retry_scale, shard, nshards, d_keys, gp);
        case P_TWO:
            return run_query<P_TWO>(g, k, d_tris, d_weight, d_count, stream, retry_scale, shard, nshards, d_keys, gp);
        case P_GEO:
            return run_query<P_GEO>(g, k, d_tris, d_weight, d_count, stream, retry_scale, shard, nshards, d_keys, gp);
        case P_GEN:
            return run_query<P_GEN>(g, k, d_tris, d_weight, d_count, stream, retry_scale, shard, nshards, d_keys, gp);
        default:
            return run_query<P_MAX>(g, k, d_tris, d_weight, d_count, stream, retry_scale, shard, nshards, d_keys, gp);
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
                      int32_t* d_count, cudaStream_t s, double gp) {
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
    q.long_count = &q.st->long_count;
    q.qid = 0;
    q.shard = 0;
    q.nshards = 1;
    q.t_short = g->tune.t_short;
    q.qbytes = nullptr;
    q.gp = gp;
    q.fw = g->d.fw;
    q.wait_first = stage_wait_limit();
    // The array keeps the previous call's contents: reset the status word
    // (counters, threshold, stop flag, error bits).
    WTRI_CUDA(cudaMemsetAsync(q.st, 0, sizeof(QState), s));

    const size_t lsmem = LONG_SMEM;
    WTRI_TRY((long_optin<P, false>()));
    const int long_grid = sm_count() * 2;
    int64_t lo = 0, size = g->tune.first_round;
    while (lo < m) {
        const int64_t hi = std::min(m, lo + size);
        if (P == P_MIN) {  // NodeIterator++ rounds, as in run_query
            k_round_min<<<round_grid_warps(hi - lo), RBLK, 0, s>>>(G, q, lo, hi);
            count_launches(1);
        } else {
            if (hi - lo <= WARP_ROUND_MAX)
                k_round_warp<P><<<round_grid_warps(hi - lo), RBLK, 0, s>>>(G, q, lo, hi);
            else
                k_round<P><<<round_grid(hi - lo), RBLK, 0, s>>>(G, q, lo, hi);
            k_long<P><<<long_grid, LBLK, lsmem, s>>>(G, q);
            count_launches(2);
        }
        k_select<<<1, SBLK, 0, s>>>(q);
        count_launches(1);
        lo = hi;
        size *= g->tune.growth;
    }
    k_final_select<<<1, SBLK, 0, s>>>(q);
    k_rank_scatter<P><<<ceil_div_u(std::max(k, 1), 8), 256, 0, s>>>(q, d_tris, d_weight, d_count,
                                                                    nullptr);
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
    if (pcode == P_GEO)
        return run_sample<P_GEO>(g, k, nsamples, seed, d_tris, d_weight, d_count, stream, retry_scale);
    return run_sample<P_TWO>(g, k, nsamples, seed, d_tris, d_weight, d_count, stream, retry_scale);
}

int sample_edges_device(const wtri_graph* g, int pcode, int64_t nsamples, uint64_t seed,
                        uint32_t* d_mark, cudaStream_t stream) {
    if (pcode == P_ONE) return draw_samples<P_ONE>(g, nsamples, seed, d_mark, stream);
    if (pcode == P_GEO) return draw_samples<P_GEO>(g, nsamples, seed, d_mark, stream);
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
    WTRI_TRY(p_to_code_for(p, g, &code));
    if (!d_tris || !d_weight || !d_count) return set_error(WTRI_EINVAL, "output pointers are NULL");
    cudaStream_t s = stream ? (cudaStream_t)stream : g->stream;
    if (g->d.m == 0) {
        WTRI_CUDA(cudaMemsetAsync(d_count, 0, sizeof(int32_t), s));
        return WTRI_OK;
    }
    switch (code) {
        case P_MIN: return run_query_noalloc<P_MIN>(g, k, d_tris, d_weight, d_count, s, p);
        case P_ONE: return run_query_noalloc<P_ONE>(g, k, d_tris, d_weight, d_count, s, p);
        case P_TWO: return run_query_noalloc<P_TWO>(g, k, d_tris, d_weight, d_count, s, p);
        case P_GEO: return run_query_noalloc<P_GEO>(g, k, d_tris, d_weight, d_count, s, p);
        case P_GEN: return run_query_noalloc<P_GEN>(g, k, d_tris, d_weight, d_count, s, p);
        default: return run_query_noalloc<P_MAX>(g, k, d_tris, d_weight, d_count, s, p);
    }
}


// ---------------------------------------------------------------------------
// Instrumented query byte counter (one per device).
// ---------------------------------------------------------------------------
namespace wtri {
namespace {
__device__ unsigned long long g_query_bytes;
std::atomic<int> g_query_bytes_on{0};
std::mutex g_qb_mu;
unsigned long long* g_qb_ptr[64] = {};
}  // namespace

bool query_bytes_on() { return g_query_bytes_on.load(std::memory_order_relaxed) != 0; }

unsigned long long* query_bytes_counter() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(g_qb_mu);
    if (!g_qb_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_query_bytes) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        g_qb_ptr[dev] = (unsigned long long*)p;
    }
    return g_qb_ptr[dev];
}

}  // namespace wtri

extern "C" WTRI_API int wtri_query_bytes(int on, int reset, unsigned long long* bytes) {
    using namespace wtri;
    unsigned long long* d = query_bytes_counter();
    if (!d) return set_error(WTRI_ECUDA, "query byte counter unavailable on this device");
    WTRI_CUDA(cudaDeviceSynchronize());
    if (bytes) WTRI_CUDA(cudaMemcpy(bytes, d, sizeof(unsigned long long), cudaMemcpyDeviceToHost));
    if (reset) WTRI_CUDA(cudaMemset(d, 0, sizeof(unsigned long long)));
    g_query_bytes_on.store(on ? 1 : 0);
    return WTRI_OK;
}

extern "C" WTRI_API int wtri_debug_set_wait_limit(int64_t polls) {
    wtri::g_stage_wait.store(polls < 0 ? wtri::WAIT_LIMIT : (uint32_t)std::min<int64_t>(polls, UINT32_MAX));
    return WTRI_OK;
}
