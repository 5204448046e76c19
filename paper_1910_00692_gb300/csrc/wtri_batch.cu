// Batched exact top-k: many (graph, p, k) queries in one launch sequence.
//
// Every query keeps its own state (threshold, stop point, candidate buffer)
// exactly as in the single query; the kernels of each phase run over all
// queries at once:
//   k_round_offsets one block: each query's live range for this round (cut
//                   at its stop point) and their prefix offsets;
//   k_round_batch   threads stride over the concatenated live ranges (a
//                   binary search maps a work item to its query);
//   k_long_batch    deferred long scans of all queries (items carry the
//                   query index);
//   k_select_batch  one block per query: k-th key, compaction, threshold;
//   k_final_batch / k_rank_batch: exact selection and ranking per query.
// The whole sequence (rounds x 4 + 2 launches) is captured in one CUDA
// graph and launched once.
#include "wtri_query.cuh"

#include <vector>

#ifndef WTRI_BATCH_FIRST
#define WTRI_BATCH_FIRST 64  // first round of a batched query (edges)
#endif
#ifndef WTRI_BATCH_GROWTH
#define WTRI_BATCH_GROWTH 8  // growth of the batch's rounds
#endif

namespace wtri {
namespace {

struct BatchDev {
    const DevGraph* graphs;
    const Query* queries;
    const int32_t* pcodes;
    int32_t nq;
};

// Last q with offs[q] <= t (offs non-decreasing, offs[0] = 0 <= t).
__device__ __forceinline__ int find_q(const int64_t* offs, int nq, int64_t t) {
    int lo = 0, hi = nq;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(offs + mid) <= t) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Per round: each query's live range is [lo, min(hi, its stop point)); the
// exclusive prefix of the live sizes maps work items to queries, so
// queries that have stopped cost nothing in later rounds.
__global__ void __launch_bounds__(1024) k_round_offsets(BatchDev B, const int64_t* __restrict__ lo,
                                                        const int64_t* __restrict__ hi,
                                                        int64_t* __restrict__ offs) {
    __shared__ int64_t warp_sum[32];
    __shared__ int64_t carry;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < B.nq; base += 1024) {
        const int qi = base + threadIdx.x;
        int64_t sz = 0;
        if (qi < B.nq) {
            const int64_t stop = (int64_t)(STOP_NONE - *(volatile const uint32_t*)&B.queries[qi].st->stop_rev);
            const int64_t e = min(hi[qi], stop);
            sz = e > lo[qi] ? e - lo[qi] : 0;
        }
        int64_t inc = sz;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) warp_sum[wid] = inc;
        __syncthreads();
        if (threadIdx.x == 0) {
            int64_t acc = carry;
            for (int k = 0; k < 32; k++) {
                const int64_t t = warp_sum[k];
                warp_sum[k] = acc;
                acc += t;
            }
            carry = acc;
        }
        __syncthreads();
        if (qi < B.nq) offs[qi] = warp_sum[wid] + inc - sz;
        __syncthreads();
    }
    if (threadIdx.x == 0) offs[B.nq] = carry;
}

__global__ void __launch_bounds__(RBLK) k_round_batch(BatchDev B, const int64_t* __restrict__ offs,
                                                      const int64_t* __restrict__ lo) {
    const int64_t total = offs[B.nq];
    const int64_t stride = (int64_t)gridDim.x * RBLK;
    for (int64_t t = (int64_t)blockIdx.x * RBLK + threadIdx.x; t < total; t += stride) {
        const int qi = find_q(offs, B.nq, t);
        const Query& q = B.queries[qi];
        const int64_t idx = lo[qi] + (t - offs[qi]);
        if (idx >= (int64_t)(STOP_NONE - *(volatile const uint32_t*)&q.st->stop_rev)) continue;
        const unsigned long long tau = ld_volatile_u64(&q.st->tau);
        const DevGraph& G = B.graphs[qi];
        Tally tb;  // batched queries are not instrumented
        switch (B.pcodes[qi]) {
            case P_MIN: process_edge<P_MIN, false>(G, q, tau, (int32_t)idx, tb); break;
            case P_ONE: process_edge<P_ONE, false>(G, q, tau, (int32_t)idx, tb); break;
            case P_TWO: process_edge<P_TWO, false>(G, q, tau, (int32_t)idx, tb); break;
            case P_GEO: process_edge<P_GEO, false>(G, q, tau, (int32_t)idx, tb); break;
            default: process_edge<P_MAX, false>(G, q, tau, (int32_t)idx, tb); break;
        }
    }
}

__global__ void __launch_bounds__(LBLK) k_long_batch(BatchDev B, const LongItem* __restrict__ longs,
                                                     const uint32_t* long_count, uint32_t long_cap) {
    extern __shared__ __align__(128) unsigned char lsm[];
    int32_t* srow = reinterpret_cast<int32_t*>(lsm);
    __shared__ __align__(8) uint64_t bar;
    __shared__ int timed_out;
    const uint32_t n_items = min(*(volatile const uint32_t*)long_count, long_cap);
    if (blockIdx.x >= n_items) return;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        timed_out = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    uint32_t phase = 0;
    for (uint32_t it = blockIdx.x; it < n_items; it += gridDim.x) {
        const LongItem item = longs[it];
        const int qi = item.pad;
        const Query& q = B.queries[qi];
        const DevGraph& G = B.graphs[qi];
        const unsigned long long tau = ld_volatile_u64(&q.st->tau);
        const int64_t dy = __ldg(G.rowptr + item.y + 1) - __ldg(G.rowptr + item.y);
        const int64_t obeg = __ldg(G.orowptr + item.y);
        const int32_t ody = (int32_t)(__ldg(G.orowptr + item.y + 1) - obeg);
        const bool staged = ody > 0 && ody <= STAGE_MAX;
        int32_t off = 0;
        if (staged && !stage_row(G, obeg, ody, srow, &bar, phase, off, &q.st->err, &timed_out,
                                 WAIT_LIMIT))
            return;
        Tally tb;
        switch (B.pcodes[qi]) {
            case P_MIN: long_scan<P_MIN, false>(G, q, tau, item, srow, off, obeg, ody, dy, staged, tb); break;
            case P_ONE: long_scan<P_ONE, false>(G, q, tau, item, srow, off, obeg, ody, dy, staged, tb); break;
            case P_TWO: long_scan<P_TWO, false>(G, q, tau, item, srow, off, obeg, ody, dy, staged, tb); break;
            case P_GEO: long_scan<P_GEO, false>(G, q, tau, item, srow, off, obeg, ody, dy, staged, tb); break;
            default: long_scan<P_MAX, false>(G, q, tau, item, srow, off, obeg, ody, dy, staged, tb); break;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(SBLK) k_select_batch(BatchDev B) {
    __shared__ SelectSmem S;
    select_round(B.queries[blockIdx.x], S);
}

__global__ void __launch_bounds__(SBLK) k_final_batch(BatchDev B) {
    __shared__ SelectSmem S;
    final_select(B.queries[blockIdx.x], S);
}

__global__ void __launch_bounds__(256) k_rank_batch(BatchDev B, const int64_t* __restrict__ koffs,
                                                    wtri_tri* out_tri, double* out_w,
                                                    int32_t* status) {
    const int64_t total = koffs[B.nq];
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t wv = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; wv < total;
         wv += nwarps) {
        const int qi = find_q(koffs, B.nq, wv);
        const uint32_t i = (uint32_t)(wv - koffs[qi]);
        const Query& q = B.queries[qi];
        wtri_tri* ot = out_tri + koffs[qi];
        double* ow = out_w + koffs[qi];
        switch (B.pcodes[qi]) {
            case P_MIN: rank_one<P_MIN>(q, i, ot, ow, status + qi); break;
            case P_ONE: rank_one<P_ONE>(q, i, ot, ow, status + qi); break;
            case P_TWO: rank_one<P_TWO>(q, i, ot, ow, status + qi); break;
            case P_GEO: rank_one<P_GEO>(q, i, ot, ow, status + qi); break;
            default: rank_one<P_MAX>(q, i, ot, ow, status + qi); break;
        }
    }
}

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

}  // namespace wtri

// ---------------------------------------------------------------------------
// Host side: a batch plan (schedule, buffer layout, descriptors), launching
// it on a stream into one device scratch block, and collecting results.
// Used by wtri_topk_batch and by the serving loop.
// ---------------------------------------------------------------------------
struct wtri_batch_plan {
    int32_t nq = 0;
    int R = 0;
    std::vector<wtri::DevGraph> hg;
    std::vector<int32_t> pcodes, ks, tshort;
    std::vector<uint32_t> caps;
    std::vector<int64_t> offs, los, totals, koffs;
    std::vector<unsigned char> hq;  // Query descriptors (filled at launch)
    size_t cand_total = 0;
    uint32_t long_cap = 1u << 18;
    size_t o_st, o_key, o_tri, o_long, o_lcnt, o_g, o_q, o_pc, o_offs, o_live, o_los, o_koffs, o_otri,
        o_ow, o_stat, bytes;
    std::vector<int32_t> stat;
    std::vector<wtri_tri> otri;
    std::vector<double> ow;
};

namespace wtri {

// Candidate slots of one batched query: enough for k plus ties, and for the
// first rounds of a large graph (enumerated before the threshold exists).
uint32_t batch_query_cap(int32_t k, int64_t m) {
    int64_t cap = std::max<int64_t>(16 * (int64_t)k, m / 16);
    cap = std::min<int64_t>(cap, int64_t(1) << 20);
    return (uint32_t)std::max<int64_t>(cap, 16384);
}

BatchPlan* batch_plan_create(const wtri_graph* const* gs, const int32_t* pcodes, const int32_t* ks,
                             int32_t nq) {
    BatchPlan* P = new (std::nothrow) BatchPlan();
    if (!P) return nullptr;
    P->nq = nq;
    P->hg.resize((size_t)nq);
    P->pcodes.assign(pcodes, pcodes + nq);
    P->ks.assign(ks, ks + nq);
    P->caps.resize((size_t)nq);
    P->tshort.resize((size_t)nq);
    P->koffs.assign((size_t)nq + 1, 0);
    int64_t mmax = 0;
    for (int i = 0; i < nq; i++) {
        P->hg[(size_t)i] = gs[i]->d;
        P->tshort[(size_t)i] = gs[i]->tune.t_short;
        mmax = std::max<int64_t>(mmax, gs[i]->d.m);
        P->koffs[(size_t)i + 1] = P->koffs[(size_t)i] + ks[i];
        P->caps[(size_t)i] = batch_query_cap(ks[i], gs[i]->d.m);
        P->cand_total += P->caps[(size_t)i];
    }
    // Round schedule: one for the whole batch (first round, growth: the
    // WTRI_BATCH_* switches), since every batch round costs a launch sequence and a
    // select over all queries and the smallest growth would set the round
    // count of all; each query keeps its own graph's short/long boundary
    // (t_short).  Round r of the batch runs round r of every query (empty
    // once a query's schedule has covered its edges).
    (void)mmax;
    const int64_t first = WTRI_BATCH_FIRST;
    const int64_t growth = WTRI_BATCH_GROWTH;
    int R = 0;
    std::vector<std::vector<int64_t>> his((size_t)nq);
    for (int i = 0; i < nq; i++) {
        const int64_t m = gs[i]->d.m;
        for (int64_t lo = 0, size = first; lo < m; lo += size, size *= growth)
            his[(size_t)i].push_back(std::min(m, lo + size));
        R = std::max<int>(R, (int)his[(size_t)i].size());
    }
    P->R = R;
    // offs: per round, the query ranges' hi ends (the device computes the
    // live offsets from them and the stop points); totals bound the grids.
    P->offs.resize((size_t)R * nq);
    P->los.resize((size_t)R * nq);
    P->totals.resize((size_t)R);
    for (int r = 0; r < R; r++) {
        int64_t acc = 0;
        for (int i = 0; i < nq; i++) {
            const auto& h = his[(size_t)i];
            const int64_t m = gs[i]->d.m;
            const int64_t a = r == 0 ? 0 : (r - 1 < (int)h.size() ? h[(size_t)r - 1] : m);
            const int64_t b = r < (int)h.size() ? h[(size_t)r] : m;
            P->offs[(size_t)r * nq + i] = b;
            P->los[(size_t)r * nq + i] = a;
            acc += b - a;
        }
        P->totals[(size_t)r] = acc;
    }
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = al256(off + bytes);
        return o;
    };
    P->o_st = take(sizeof(QState) * (size_t)nq);
    P->o_key = take(8 * P->cand_total);
    P->o_tri = take(16 * P->cand_total);
    P->o_long = take(sizeof(LongItem) * (size_t)P->long_cap);
    P->o_lcnt = take(64);
    P->o_g = take(sizeof(DevGraph) * (size_t)nq);
    P->o_q = take(sizeof(Query) * (size_t)nq);
    P->o_pc = take(4 * (size_t)nq);
    P->o_offs = take(8 * std::max<size_t>(P->offs.size(), 1));
    P->o_live = take(8 * ((size_t)nq + 1) * std::max(R, 1));
    P->o_los = take(8 * std::max<size_t>(P->los.size(), 1));
    P->o_koffs = take(8 * P->koffs.size());
    P->o_otri = take(sizeof(wtri_tri) * (size_t)P->koffs[(size_t)nq]);
    P->o_ow = take(8 * (size_t)P->koffs[(size_t)nq]);
    P->o_stat = take(4 * (size_t)nq);
    P->bytes = off;
    return P;
}

size_t batch_plan_bytes(const BatchPlan* P) { return P->bytes; }

void batch_plan_destroy(BatchPlan* P) { delete P; }

// The last instantiated batch graph of this thread on each device.
struct GraphCache {
    cudaGraphExec_t exec = nullptr;
    cudaStream_t stream = nullptr;
    uint64_t instantiations = 0, updates = 0;
};

GraphCache& graph_cache() {
    static thread_local GraphCache cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
    return cache[dev];
}

// Uploads the descriptors (small, from pageable memory: the call returns
// once they are staged) and enqueues every kernel of the batch on s.
int batch_plan_launch(BatchPlan* P, void* dbuf, cudaStream_t s, int use_graph) {
    const int nq = P->nq;
    char* B0 = (char*)dbuf;
    QState* st = (QState*)(B0 + P->o_st);
    unsigned long long* ckey = (unsigned long long*)(B0 + P->o_key);
    int4* ctri = (int4*)(B0 + P->o_tri);
    LongItem* longs = (LongItem*)(B0 + P->o_long);
    uint32_t* lcnt = (uint32_t*)(B0 + P->o_lcnt);
    std::vector<Query> hq((size_t)nq);
    size_t c0 = 0;
    for (int i = 0; i < nq; i++) {
        Query& q = hq[(size_t)i];
        q.st = st + i;
        q.ckey = ckey + c0;
        q.ctri = ctri + c0;
        q.cap = P->caps[(size_t)i];
        q.longs = longs;
        q.long_cap = P->long_cap;
        q.k = P->ks[(size_t)i];
        q.smark = nullptr;
        q.slist = nullptr;
        q.long_count = lcnt;
        q.qid = i;
        q.shard = 0;
        q.nshards = 1;
        q.t_short = P->tshort[(size_t)i];
        q.qbytes = nullptr;
        q.gp = 0.0;  // batched queries take the exact-key p values only
        q.fw = 0;    // and integer weights
        q.wait_first = WAIT_LIMIT;
        c0 += P->caps[(size_t)i];
    }
    BatchDev Bd;
    Bd.graphs = (const DevGraph*)(B0 + P->o_g);
    Bd.queries = (const Query*)(B0 + P->o_q);
    Bd.pcodes = (const int32_t*)(B0 + P->o_pc);
    Bd.nq = nq;
    int64_t* d_offs = (int64_t*)(B0 + P->o_offs);
    int64_t* d_live = (int64_t*)(B0 + P->o_live);
    int64_t* d_los = (int64_t*)(B0 + P->o_los);
    int64_t* d_koffs = (int64_t*)(B0 + P->o_koffs);
    wtri_tri* d_otri = (wtri_tri*)(B0 + P->o_otri);
    double* d_ow = (double*)(B0 + P->o_ow);
    int32_t* d_stat = (int32_t*)(B0 + P->o_stat);
    WTRI_CUDA(cudaMemcpyAsync((void*)Bd.graphs, P->hg.data(), sizeof(DevGraph) * nq, cudaMemcpyHostToDevice, s));
    WTRI_CUDA(cudaMemcpyAsync((void*)Bd.queries, hq.data(), sizeof(Query) * nq, cudaMemcpyHostToDevice, s));
    WTRI_CUDA(cudaMemcpyAsync((void*)Bd.pcodes, P->pcodes.data(), 4 * (size_t)nq, cudaMemcpyHostToDevice, s));
    WTRI_CUDA(cudaMemcpyAsync(d_offs, P->offs.data(), 8 * P->offs.size(), cudaMemcpyHostToDevice, s));
    if (!P->los.empty())
        WTRI_CUDA(cudaMemcpyAsync(d_los, P->los.data(), 8 * P->los.size(), cudaMemcpyHostToDevice, s));
    WTRI_CUDA(cudaMemcpyAsync(d_koffs, P->koffs.data(), 8 * P->koffs.size(), cudaMemcpyHostToDevice, s));

    const size_t lsmem = LONG_SMEM;
    {
        static std::atomic<uint64_t> done{0};
        WTRI_TRY(smem_optin((const void*)k_long_batch, (int)lsmem, done));
    }
    const int long_grid = sm_count() * 2;
    const int R = P->R;
    auto launch_all = [&]() {
        cudaMemsetAsync(st, 0, sizeof(QState) * (size_t)nq, s);
        cudaMemsetAsync(lcnt, 0, 64, s);
        for (int r = 0; r < R; r++) {
            int64_t* live = d_live + (size_t)r * (nq + 1);
            k_round_offsets<<<1, 1024, 0, s>>>(Bd, d_los + (size_t)r * nq, d_offs + (size_t)r * nq, live);
            k_round_batch<<<round_grid(P->totals[(size_t)r]), RBLK, 0, s>>>(Bd, live,
                                                                            d_los + (size_t)r * nq);
            k_long_batch<<<long_grid, LBLK, lsmem, s>>>(Bd, longs, lcnt, P->long_cap);
            k_select_batch<<<nq, SBLK, 0, s>>>(Bd);
        }
        k_final_batch<<<nq, SBLK, 0, s>>>(Bd);
        const int64_t warps = P->koffs[(size_t)nq];
        k_rank_batch<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((warps + 7) / 8,
                                                                        sm_count() * 16)),
                       256, 0, s>>>(Bd, d_koffs, d_otri, d_ow, d_stat);
    };
    int rc = WTRI_OK;
    ProfScope ps("topk_batch", s, 0.0, 4 * R + 2);
    if (use_graph) {
        // The descriptors must have landed before the captured work refers
        // to them only through device pointers: that holds, the copies are
        // ordered on s before the graph launch.  The instantiated graph is
        // kept (per thread and device) and refreshed with
        // cudaGraphExecUpdate when the next batch has the same launch
        // topology (same number of rounds), so a repeated batch shape is
        // instantiated once.
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            launch_all();
            e = cudaStreamEndCapture(s, &graph);  // always leave capture mode
        }
        cudaGraphExec_t exec = nullptr;
        if (e == cudaSuccess) {
            GraphCache& gc = graph_cache();
            if (gc.exec && gc.stream == s) {
                cudaGraphExecUpdateResultInfo info;
                if (cudaGraphExecUpdate(gc.exec, graph, &info) == cudaSuccess) {
                    exec = gc.exec;
                    gc.updates++;
                } else {
                    cudaGetLastError();
                    cudaGraphExecDestroy(gc.exec);
                    gc.exec = nullptr;
                }
            }
            if (!exec) {
                e = cudaGraphInstantiate(&exec, graph, 0);
                if (e == cudaSuccess) {
                    gc.exec = exec;
                    gc.stream = s;
                    gc.instantiations++;
                }
            }
        }
        if (e == cudaSuccess) e = cudaGraphLaunch(exec, s);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) rc = cuda_error(e, "batch graph", __FILE__, __LINE__);
    } else {
        launch_all();
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_error(e, "batch launch", __FILE__, __LINE__);
    }
    return rc;
}

// Copies statuses and results to the plan's host vectors (synchronizes s).
int batch_plan_collect(BatchPlan* P, void* dbuf, cudaStream_t s) {
    const int nq = P->nq;
    char* B0 = (char*)dbuf;
    P->stat.assign((size_t)nq, 0);
    P->otri.resize((size_t)P->koffs[(size_t)nq]);
    P->ow.resize((size_t)P->koffs[(size_t)nq]);
    WTRI_CUDA(cudaMemcpyAsync(P->stat.data(), B0 + P->o_stat, 4 * (size_t)nq, cudaMemcpyDeviceToHost, s));
    WTRI_CUDA(cudaMemcpyAsync(P->otri.data(), B0 + P->o_otri, sizeof(wtri_tri) * P->otri.size(),
                              cudaMemcpyDeviceToHost, s));
    WTRI_CUDA(cudaMemcpyAsync(P->ow.data(), B0 + P->o_ow, 8 * P->ow.size(), cudaMemcpyDeviceToHost, s));
    WTRI_CUDA(cudaStreamSynchronize(s));
    return WTRI_OK;
}

int32_t batch_plan_status(const BatchPlan* P, int i) { return P->stat[(size_t)i]; }
const wtri_tri* batch_plan_tris(const BatchPlan* P, int i) { return P->otri.data() + P->koffs[(size_t)i]; }
const double* batch_plan_weights(const BatchPlan* P, int i) { return P->ow.data() + P->koffs[(size_t)i]; }

// One query with larger bounded buffers (for queries that overflowed a
// batch's); results to host arrays.
int topk_retry_host(const wtri_graph* g, int pcode, int32_t k, cudaStream_t s, wtri_tri* htri,
                    double* hw, int32_t* count) {
    void* dbuf = nullptr;
    WTRI_CUDA(cudaMallocAsync(&dbuf, (sizeof(wtri_tri) + 8) * (size_t)k + 64, s));
    wtri_tri* dt = (wtri_tri*)dbuf;
    double* dw = (double*)((char*)dbuf + ((sizeof(wtri_tri) * (size_t)k + 15) & ~size_t(15)));
    int32_t* dc = (int32_t*)(dw + k);
    int32_t cnt = WTRI_ENOMEM;
    int rc = WTRI_OK;
    for (int scale = 8; scale <= 64 && cnt == WTRI_ENOMEM && rc == WTRI_OK; scale *= 8) {
        rc = topk_device(g, pcode, k, dt, dw, dc, s, scale);
        if (rc == WTRI_OK) {
            cudaError_t e = cudaMemcpyAsync(&cnt, dc, 4, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) rc = cuda_error(e, "retry", __FILE__, __LINE__);
        }
    }
    if (rc == WTRI_OK && cnt < 0) rc = set_error(cnt, "query failed on retry with larger buffers");
    if (rc == WTRI_OK && cnt > 0) {
        cudaError_t e = cudaMemcpyAsync(htri, dt, sizeof(wtri_tri) * (size_t)cnt, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hw, dw, 8 * (size_t)cnt, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = cuda_error(e, "retry copy", __FILE__, __LINE__);
    }
    cudaFreeAsync(dbuf, s);
    if (rc == WTRI_OK) *count = cnt;
    return rc;
}

cudaStream_t own_stream() {
    static thread_local cudaStream_t own[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    if (!own[dev] && cudaStreamCreateWithFlags(&own[dev], cudaStreamNonBlocking) != cudaSuccess)
        return nullptr;
    return own[dev];
}

// Runs nq queries; results to caller host arrays.  Queries whose bounded
// buffers overflowed are re-run one by one with larger buffers.
int topk_batch(const wtri_graph* const* gs, const int32_t* pcodes, const int32_t* ks, int32_t nq,
               wtri_result* outs, cudaStream_t user_stream, int use_graph) {
    // The batch runs on a stream of its own (the legacy default stream cannot
    // be captured), ordered after the work already queued on the caller's.
    cudaStream_t s = own_stream();
    if (!s) return set_error(WTRI_ECUDA, "could not create the batch stream");
    {
        cudaEvent_t ev;
        WTRI_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        cudaError_t e = cudaEventRecord(ev, user_stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev, 0);
        cudaEventDestroy(ev);
        WTRI_CUDA(e);
    }
    BatchPlan* P = batch_plan_create(gs, pcodes, ks, nq);
    if (!P) return set_error(WTRI_ENOMEM, "host allocation failed");
    void* buf = nullptr;
    if (cudaMallocAsync(&buf, P->bytes, s) != cudaSuccess) {
        cudaGetLastError();
        batch_plan_destroy(P);
        return set_error(WTRI_ENOMEM, "batch scratch allocation failed");
    }
    int rc = batch_plan_launch(P, buf, s, use_graph);
    if (rc == WTRI_OK) rc = batch_plan_collect(P, buf, s);
    cudaFreeAsync(buf, s);
    for (int i = 0; i < nq && rc == WTRI_OK; i++) {
        const int32_t c = P->stat[(size_t)i];
        if (c == WTRI_ENOMEM) {
            rc = topk_retry_host(gs[i], pcodes[i], ks[i], s, outs[i].tris, outs[i].weight, &outs[i].count);
            continue;
        }
        if (c < 0) {
            rc = set_error(c, "device-side error in batched query " + std::to_string(i));
            break;
        }
        std::copy(P->otri.begin() + P->koffs[(size_t)i], P->otri.begin() + P->koffs[(size_t)i] + c,
                  outs[i].tris);
        std::copy(P->ow.begin() + P->koffs[(size_t)i], P->ow.begin() + P->koffs[(size_t)i] + c,
                  outs[i].weight);
        outs[i].count = c;
    }
    batch_plan_destroy(P);
    return rc;
}

}  // namespace wtri
