// Batched exact top-k: many (graph, p, k) queries in one launch sequence.
//
// Every query keeps its own state (threshold, stop point, candidate buffer)
// exactly as in the single query; the kernels of each phase run over all
// queries at once:
//   k_round_batch   threads stride over the concatenated edge ranges of all
//                   queries for this round (host-computed offsets; a binary
//                   search maps a work item to its query);
//   k_long_batch    deferred long scans of all queries (items carry the
//                   query index);
//   k_select_batch  one block per query: k-th key, compaction, threshold;
//   k_final_batch / k_rank_batch: exact selection and ranking per query.
// The whole sequence (rounds x 3 + 2 launches) is captured in one CUDA
// graph and launched once.
#include "wtri_query.cuh"

#include <vector>

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
        switch (B.pcodes[qi]) {
            case P_MIN: process_edge<P_MIN, false>(G, q, tau, (int32_t)idx); break;
            case P_ONE: process_edge<P_ONE, false>(G, q, tau, (int32_t)idx); break;
            case P_TWO: process_edge<P_TWO, false>(G, q, tau, (int32_t)idx); break;
            default: process_edge<P_MAX, false>(G, q, tau, (int32_t)idx); break;
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
        const int64_t ybeg = __ldg(G.rowptr + item.y), yend = __ldg(G.rowptr + item.y + 1);
        const int32_t dy = (int32_t)(yend - ybeg);
        const bool staged = dy <= STAGE_MAX;
        int32_t off = 0;
        if (staged && !stage_row(G, ybeg, dy, srow, &bar, phase, off, &q.st->err, &timed_out))
            return;
        switch (B.pcodes[qi]) {
            case P_MIN: long_scan<P_MIN, false>(G, q, tau, item, srow, off, ybeg, dy, staged); break;
            case P_ONE: long_scan<P_ONE, false>(G, q, tau, item, srow, off, ybeg, dy, staged); break;
            case P_TWO: long_scan<P_TWO, false>(G, q, tau, item, srow, off, ybeg, dy, staged); break;
            default: long_scan<P_MAX, false>(G, q, tau, item, srow, off, ybeg, dy, staged); break;
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
            default: rank_one<P_MAX>(q, i, ot, ow, status + qi); break;
        }
    }
}

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

// Runs nq queries; results to caller host arrays.  Queries whose bounded
// buffers overflowed are re-run one by one with larger buffers.
int topk_batch(const wtri_graph* const* gs, const int32_t* pcodes, const int32_t* ks, int32_t nq,
               wtri_result* outs, cudaStream_t user_stream, int use_graph) {
    // The batch runs on a stream of its own (the legacy default stream cannot
    // be captured), ordered after the work already queued on the caller's.
    static thread_local cudaStream_t own[64] = {};
    int dev = 0;
    WTRI_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return set_error(WTRI_EUNSUPPORTED, "device index above 63");
    if (!own[dev]) WTRI_CUDA(cudaStreamCreateWithFlags(&own[dev], cudaStreamNonBlocking));
    cudaStream_t s = own[dev];
    {
        cudaEvent_t ev;
        WTRI_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        cudaError_t e = cudaEventRecord(ev, user_stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev, 0);
        cudaEventDestroy(ev);
        WTRI_CUDA(e);
    }
    std::vector<DevGraph> hg((size_t)nq);
    std::vector<Query> hq((size_t)nq);
    std::vector<int64_t> koffs((size_t)nq + 1, 0);
    int64_t mmax = 0;
    size_t cand_total = 0;
    std::vector<uint32_t> caps((size_t)nq);
    for (int i = 0; i < nq; i++) {
        hg[(size_t)i] = gs[i]->d;
        mmax = std::max<int64_t>(mmax, gs[i]->d.m);
        koffs[(size_t)i + 1] = koffs[(size_t)i] + ks[i];
        caps[(size_t)i] = (uint32_t)std::max<int64_t>(16384, 16 * (int64_t)ks[i]);
        cand_total += caps[(size_t)i];
    }
    // Round schedule (same as a single query), per query clipped to its m.
    std::vector<int64_t> r_lo, r_hi;
    for (int64_t lo = 0, size = FIRST_ROUND; lo < mmax; lo += size, size *= ROUND_GROWTH) {
        r_lo.push_back(lo);
        r_hi.push_back(std::min(mmax, lo + size));
    }
    const int R = (int)r_lo.size();
    std::vector<int64_t> offs((size_t)R * (nq + 1)), los((size_t)R * nq);
    std::vector<int64_t> totals((size_t)R);
    for (int r = 0; r < R; r++) {
        int64_t acc = 0;
        for (int i = 0; i < nq; i++) {
            const int64_t m = gs[i]->d.m;
            const int64_t a = std::min(m, r_lo[(size_t)r]), b = std::min(m, r_hi[(size_t)r]);
            offs[(size_t)r * (nq + 1) + i] = acc;
            los[(size_t)r * nq + i] = a;
            acc += b - a;
        }
        offs[(size_t)r * (nq + 1) + nq] = acc;
        totals[(size_t)r] = acc;
    }
    const uint32_t long_cap = 1u << 18;
    // Device scratch: states, candidates, deferred list, descriptors, outputs.
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = al256(off + bytes);
        return o;
    };
    const size_t o_st = take(sizeof(QState) * (size_t)nq);
    const size_t o_key = take(8 * cand_total);
    const size_t o_tri = take(16 * cand_total);
    const size_t o_long = take(sizeof(LongItem) * (size_t)long_cap);
    const size_t o_lcnt = take(64);
    const size_t o_g = take(sizeof(DevGraph) * (size_t)nq);
    const size_t o_q = take(sizeof(Query) * (size_t)nq);
    const size_t o_pc = take(4 * (size_t)nq);
    const size_t o_offs = take(8 * offs.size());
    const size_t o_los = take(8 * std::max<size_t>(los.size(), 1));
    const size_t o_koffs = take(8 * koffs.size());
    const size_t o_otri = take(sizeof(wtri_tri) * (size_t)koffs[(size_t)nq]);
    const size_t o_ow = take(8 * (size_t)koffs[(size_t)nq]);
    const size_t o_stat = take(4 * (size_t)nq);
    void* buf = nullptr;
    if (cudaMallocAsync(&buf, off, s) != cudaSuccess) {
        cudaGetLastError();
        return set_error(WTRI_ENOMEM, "batch scratch allocation failed");
    }
    char* B0 = (char*)buf;
    QState* st = (QState*)(B0 + o_st);
    unsigned long long* ckey = (unsigned long long*)(B0 + o_key);
    int4* ctri = (int4*)(B0 + o_tri);
    LongItem* longs = (LongItem*)(B0 + o_long);
    uint32_t* lcnt = (uint32_t*)(B0 + o_lcnt);
    size_t c0 = 0;
    for (int i = 0; i < nq; i++) {
        Query& q = hq[(size_t)i];
        q.st = st + i;
        q.ckey = ckey + c0;
        q.ctri = ctri + c0;
        q.cap = caps[(size_t)i];
        q.longs = longs;
        q.long_cap = long_cap;
        q.k = ks[i];
        q.smark = nullptr;
        q.slist = nullptr;
        q.long_count = lcnt;
        q.qid = i;
        c0 += caps[(size_t)i];
    }
    BatchDev Bd;
    Bd.graphs = (const DevGraph*)(B0 + o_g);
    Bd.queries = (const Query*)(B0 + o_q);
    Bd.pcodes = (const int32_t*)(B0 + o_pc);
    Bd.nq = nq;
    int64_t* d_offs = (int64_t*)(B0 + o_offs);
    int64_t* d_los = (int64_t*)(B0 + o_los);
    int64_t* d_koffs = (int64_t*)(B0 + o_koffs);
    wtri_tri* d_otri = (wtri_tri*)(B0 + o_otri);
    double* d_ow = (double*)(B0 + o_ow);
    int32_t* d_stat = (int32_t*)(B0 + o_stat);
    int rc = WTRI_OK;
    auto cu = [&](cudaError_t e, const char* what) {
        if (e != cudaSuccess && rc == WTRI_OK) rc = cuda_error(e, what, __FILE__, __LINE__);
    };
    cu(cudaMemcpyAsync((void*)Bd.graphs, hg.data(), sizeof(DevGraph) * nq, cudaMemcpyHostToDevice, s), "upload");
    cu(cudaMemcpyAsync((void*)Bd.queries, hq.data(), sizeof(Query) * nq, cudaMemcpyHostToDevice, s), "upload");
    cu(cudaMemcpyAsync((void*)Bd.pcodes, pcodes, 4 * (size_t)nq, cudaMemcpyHostToDevice, s), "upload");
    cu(cudaMemcpyAsync(d_offs, offs.data(), 8 * offs.size(), cudaMemcpyHostToDevice, s), "upload");
    if (!los.empty())
        cu(cudaMemcpyAsync(d_los, los.data(), 8 * los.size(), cudaMemcpyHostToDevice, s), "upload");
    cu(cudaMemcpyAsync(d_koffs, koffs.data(), 8 * koffs.size(), cudaMemcpyHostToDevice, s), "upload");
    // Uploads come from pageable memory: finish them before the capture.
    cu(cudaStreamSynchronize(s), "upload");

    const size_t lsmem = (size_t)STAGE_MAX * 4 + 16;
    static bool attr_done = false;
    if (!attr_done && rc == WTRI_OK) {
        cu(cudaFuncSetAttribute(k_long_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lsmem),
           "attribute");
        attr_done = true;
    }
    const int long_grid = sm_count() * 2;
    auto launch_all = [&]() {
        cudaMemsetAsync(st, 0, sizeof(QState) * (size_t)nq, s);
        cudaMemsetAsync(lcnt, 0, 64, s);
        for (int r = 0; r < R; r++) {
            k_round_batch<<<round_grid(totals[(size_t)r]), RBLK, 0, s>>>(
                Bd, d_offs + (size_t)r * (nq + 1), d_los + (size_t)r * nq);
            k_long_batch<<<long_grid, LBLK, lsmem, s>>>(Bd, longs, lcnt, long_cap);
            k_select_batch<<<nq, SBLK, 0, s>>>(Bd);
        }
        k_final_batch<<<nq, SBLK, 0, s>>>(Bd);
        const int64_t warps = koffs[(size_t)nq];
        k_rank_batch<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((warps + 7) / 8,
                                                                        sm_count() * 16)),
                       256, 0, s>>>(Bd, d_koffs, d_otri, d_ow, d_stat);
    };
    if (rc == WTRI_OK) {
        ProfScope ps("topk_batch", s, 0.0, 3 * R + 2);
        if (use_graph) {
            cudaGraph_t graph = nullptr;
            cudaGraphExec_t exec = nullptr;
            const cudaError_t eb = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
            cu(eb, "begin capture");
            if (eb == cudaSuccess) {
                launch_all();
                // always leave capture mode, even if a launch failed
                cu(cudaStreamEndCapture(s, &graph), "end capture");
            }
            if (rc == WTRI_OK) cu(cudaGraphInstantiate(&exec, graph, 0), "instantiate");
            if (rc == WTRI_OK) cu(cudaGraphLaunch(exec, s), "graph launch");
            if (exec) cudaGraphExecDestroy(exec);
            if (graph) cudaGraphDestroy(graph);
        } else {
            launch_all();
            cu(cudaGetLastError(), "batch launch");
        }
    }
    std::vector<int32_t> stat((size_t)nq, 0);
    std::vector<wtri_tri> otri((size_t)koffs[(size_t)nq]);
    std::vector<double> ow((size_t)koffs[(size_t)nq]);
    if (rc == WTRI_OK) {
        cu(cudaMemcpyAsync(stat.data(), d_stat, 4 * (size_t)nq, cudaMemcpyDeviceToHost, s), "status");
        cu(cudaMemcpyAsync(otri.data(), d_otri, sizeof(wtri_tri) * otri.size(), cudaMemcpyDeviceToHost, s),
           "results");
        cu(cudaMemcpyAsync(ow.data(), d_ow, 8 * ow.size(), cudaMemcpyDeviceToHost, s), "results");
        cu(cudaStreamSynchronize(s), "results");
    }
    cudaFreeAsync(buf, s);
    if (rc != WTRI_OK) return rc;
    std::vector<int> redo;
    for (int i = 0; i < nq; i++) {
        const int32_t c = stat[(size_t)i];
        if (c == WTRI_ENOMEM) {
            redo.push_back(i);
            continue;
        }
        if (c < 0) return set_error(c, "device-side error in batched query " + std::to_string(i));
        std::copy(otri.begin() + koffs[(size_t)i], otri.begin() + koffs[(size_t)i] + c, outs[i].tris);
        std::copy(ow.begin() + koffs[(size_t)i], ow.begin() + koffs[(size_t)i] + c, outs[i].weight);
        outs[i].count = c;
    }
    for (int i : redo) {
        // Larger bounded buffers, one query at a time.
        const int32_t k = ks[i];
        void* dbuf = nullptr;
        WTRI_CUDA(cudaMallocAsync(&dbuf, (sizeof(wtri_tri) + 8) * (size_t)k + 64, s));
        wtri_tri* dt = (wtri_tri*)dbuf;
        double* dw = (double*)((char*)dbuf + ((sizeof(wtri_tri) * (size_t)k + 15) & ~size_t(15)));
        int32_t* dc = (int32_t*)(dw + k);
        int32_t cnt = WTRI_ENOMEM;
        for (int scale = 8; scale <= 64 && cnt == WTRI_ENOMEM; scale *= 8) {
            WTRI_TRY(topk_device(gs[i], pcodes[i], k, dt, dw, dc, s, scale));
            WTRI_CUDA(cudaMemcpyAsync(&cnt, dc, 4, cudaMemcpyDeviceToHost, s));
            WTRI_CUDA(cudaStreamSynchronize(s));
        }
        if (cnt < 0) {
            cudaFreeAsync(dbuf, s);
            return set_error(cnt, "batched query " + std::to_string(i) + " failed on retry");
        }
        WTRI_CUDA(cudaMemcpyAsync(outs[i].tris, dt, sizeof(wtri_tri) * (size_t)cnt, cudaMemcpyDeviceToHost, s));
        WTRI_CUDA(cudaMemcpyAsync(outs[i].weight, dw, 8 * (size_t)cnt, cudaMemcpyDeviceToHost, s));
        WTRI_CUDA(cudaStreamSynchronize(s));
        cudaFreeAsync(dbuf, s);
        outs[i].count = cnt;
    }
    return WTRI_OK;
}

}  // namespace wtri
