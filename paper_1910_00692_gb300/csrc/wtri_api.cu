// C ABI entry points (include/wtri.h): argument checks, error reporting and
// host-side result copies around the device paths.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <string>
#include <algorithm>
#include <vector>

#include "wtri_internal.cuh"

namespace wtri {

static thread_local std::string t_last_error;

int set_error(int code, const std::string& msg) {
    t_last_error = msg;
    return code;
}

int cuda_error(cudaError_t e, const char* what, const char* file, int line) {
    std::string msg = std::string(what) + ": " + cudaGetErrorString(e) + " (" + file + ":" +
                      std::to_string(line) + ")";
    if (e == cudaErrorMemoryAllocation) return set_error(WTRI_ENOMEM, msg);
    return set_error(WTRI_ECUDA, msg);
}

int p_to_code(double p, int* code) {
    if (isnan(p)) return set_error(WTRI_EINVAL, "p is NaN");
    if (p == 1.0) *code = P_ONE;
    else if (p == 2.0) *code = P_TWO;
    else if (isinf(p) && p > 0) *code = P_MAX;
    else if (isinf(p) && p < 0) *code = P_MIN;
    else if (p == 0.0) *code = P_GEO;
    else *code = P_GEN;  // any other finite p: fp64 key
    return WTRI_OK;
}

int p_to_code_for(double p, const wtri_graph* g, int* code) {
    WTRI_TRY(p_to_code(p, code));
    if (g && g->d.fw) {  // real weights: every finite p ranks by the fp64 mean
        if (*code == P_ONE || *code == P_TWO || *code == P_GEO) *code = P_GEN;
        return WTRI_OK;
    }
    if (*code == P_GEO && g && g->d.wmax > GEO_WMAX)
        return set_error(WTRI_EUNSUPPORTED, "p = 0 needs weights below 2^21 (exact product key)");
    return WTRI_OK;
}

int need_integer_weights(const wtri_graph* g, const char* what) {
    if (g && g->d.fw)
        return set_error(WTRI_EUNSUPPORTED, std::string(what) + " takes integer weights (exact w^p or keys)");
    return WTRI_OK;
}

int sm_count() {
    static std::atomic<int> cached[64];
    int dev = 0, c = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 132;
    if (dev >= 0 && dev < 64 && (c = cached[dev].load(std::memory_order_relaxed)) > 0) return c;
    if (cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || c <= 0)
        return 132;
    if (dev >= 0 && dev < 64) cached[dev].store(c, std::memory_order_relaxed);
    return c;
}

int smem_optin(const void* fn, int bytes, std::atomic<uint64_t>& done) {
    int dev = 0;
    WTRI_CUDA(cudaGetDevice(&dev));
    const uint64_t bit = (dev >= 0 && dev < 64) ? (1ull << dev) : 0ull;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return WTRI_OK;
    WTRI_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    if (bit) done.fetch_or(bit, std::memory_order_acq_rel);
    return WTRI_OK;
}

const char* query_name(int pcode) {
    static const char* const names[P_COUNT] = {"query_p=-inf", "query_p=1", "query_p=2",
                                               "query_p=+inf", "query_p=0", "query_p=general"};
    static_assert(P_MIN < P_COUNT && P_ONE < P_COUNT && P_TWO < P_COUNT && P_MAX < P_COUNT &&
                      P_GEO < P_COUNT && P_GEN < P_COUNT,
                  "every p code names a query");
    return (pcode >= 0 && pcode < P_COUNT) ? names[pcode] : "query_p=?";
}

namespace {

constexpr int32_t K_MAX = 65536;

int check_query(const wtri_graph* g, int32_t k) {
    if (!g) return set_error(WTRI_EINVAL, "graph is NULL");
    if (k <= 0) return set_error(WTRI_EINVAL, "k must be positive");
    if (k > K_MAX) return set_error(WTRI_EUNSUPPORTED, "k above 65536");
    return WTRI_OK;
}

// Runs a device query into scratch outputs, copies them to the caller's host
// result, retrying with larger device buffers if a bounded buffer filled.
template <class Launch>
int host_result_query(const wtri_graph* g, int32_t k, wtri_result* out, Launch launch,
                      uint64_t* hkeys = nullptr) {
    cudaStream_t s = g->stream;
    const size_t tri_bytes = sizeof(wtri_tri) * (size_t)k;
    const size_t w_bytes = sizeof(double) * (size_t)k;
    void* buf = nullptr;
    WTRI_CUDA(cudaMallocAsync(&buf, tri_bytes + 2 * w_bytes + 64, s));
    wtri_tri* d_tri = (wtri_tri*)buf;
    double* d_w = (double*)((char*)buf + ((tri_bytes + 15) & ~size_t(15)));
    unsigned long long* d_key = (unsigned long long*)((char*)d_w + w_bytes);
    int32_t* d_cnt = (int32_t*)((char*)d_key + w_bytes);
    int rc = WTRI_OK;
    int32_t status = 0;
    for (int scale = 1; scale <= 64; scale *= 8) {
        rc = launch(d_tri, d_w, d_cnt, s, scale, hkeys ? d_key : nullptr);
        if (rc != WTRI_OK) break;
        cudaError_t e = cudaMemcpyAsync(&status, d_cnt, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            rc = cuda_error(e, "query", __FILE__, __LINE__);
            break;
        }
        if (status == WTRI_ENOMEM && scale < 64) continue;  // bounded buffer overflowed: retry
        break;
    }
    if (rc == WTRI_OK && status < 0) {
        rc = set_error(status, status == WTRI_ENOMEM     ? "device candidate buffer overflow"
                               : status == WTRI_ETIMEOUT ? "bounded device wait ran out"
                                                         : "device-side error in query");
    }
    if (rc == WTRI_OK && status > 0) {
        cudaError_t e = cudaMemcpyAsync(out->tris, d_tri, sizeof(wtri_tri) * (size_t)status,
                                        cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(out->weight, d_w, sizeof(double) * (size_t)status,
                                cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && hkeys)
            e = cudaMemcpyAsync(hkeys, d_key, 8 * (size_t)status, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = cuda_error(e, "result copy", __FILE__, __LINE__);
    }
    cudaFreeAsync(buf, s);
    if (rc == WTRI_OK) out->count = status;
    return rc;
}

}  // namespace
}  // namespace wtri

using namespace wtri;

extern "C" {

WTRI_API const char* wtri_last_error(void) { return t_last_error.c_str(); }

WTRI_API const char* wtri_version(void) { return "wtri 0.1 (sm_103a)"; }

WTRI_API int wtri_build_csr(int32_t n, int64_t m, const int32_t* u, const int32_t* v,
                            const int32_t* w, int on_device, void* cuda_stream, wtri_graph** out) {
    if (!out) return set_error(WTRI_EINVAL, "out is NULL");
    *out = nullptr;
    t_last_error.clear();
    return build_graph(n, m, u, v, w, on_device, (cudaStream_t)cuda_stream, out);
}

WTRI_API int wtri_build_csr_f32(int32_t n, int64_t m, const int32_t* u, const int32_t* v, const float* w,
                                int on_device, void* cuda_stream, wtri_graph** out) {
    if (!out) return set_error(WTRI_EINVAL, "out is NULL");
    *out = nullptr;
    t_last_error.clear();
    // positive floats order like their bit patterns: the build sorts the bits
    return build_graph(n, m, u, v, reinterpret_cast<const int32_t*>(w), on_device,
                       (cudaStream_t)cuda_stream, out, 1);
}

WTRI_API void wtri_graph_free(wtri_graph* g) {
    if (!g) return;
    // Queries may have run on other streams: let all device work finish.
    cudaDeviceSynchronize();
    cudaFreeAsync(g->base, g->stream);
    cudaStreamSynchronize(g->stream);
    delete g;
}

WTRI_API int wtri_graph_info(const wtri_graph* g, int32_t* n, int64_t* m, int32_t* max_degree,
                             int32_t* max_weight, int64_t* device_bytes) {
    if (!g) return set_error(WTRI_EINVAL, "graph is NULL");
    if (n) *n = g->d.n;
    if (m) *m = g->d.m;
    if (max_degree) *max_degree = g->d.maxdeg;
    if (max_weight) *max_weight = g->d.wmax;
    if (device_bytes) *device_bytes = g->bytes;
    return WTRI_OK;
}

WTRI_API int wtri_topk(const wtri_graph* g, double p, int32_t k, wtri_result* out) {
    if (!out) return set_error(WTRI_EINVAL, "out is NULL");
    out->count = 0;
    int code = 0;
    WTRI_TRY(check_query(g, k));
    WTRI_TRY(p_to_code_for(p, g, &code));
    if (!out->tris || !out->weight) return set_error(WTRI_EINVAL, "result arrays are NULL");
    if (out->capacity < k) return set_error(WTRI_EINVAL, "result capacity below k");
    if (g->d.m == 0) return WTRI_OK;
    return host_result_query(g, k, out,
                             [&](wtri_tri* t, double* wv, int32_t* c, cudaStream_t s, int scale,
                                 unsigned long long*) {
                                 return topk_device(g, code, k, t, wv, c, s, scale, 0, 1, nullptr, p);
                             });
}

WTRI_API int wtri_topk_shard(const wtri_graph* g, double p, int32_t k, int32_t shard,
                             int32_t nshards, wtri_result* out, uint64_t* keys) {
    if (!out) return set_error(WTRI_EINVAL, "out is NULL");
    out->count = 0;
    int code = 0;
    WTRI_TRY(check_query(g, k));
    WTRI_TRY(p_to_code_for(p, g, &code));
    if (nshards < 1 || shard < 0 || shard >= nshards)
        return set_error(WTRI_EINVAL, "need 0 <= shard < nshards");
    if (!out->tris || !out->weight || !keys) return set_error(WTRI_EINVAL, "result arrays are NULL");
    if (out->capacity < k) return set_error(WTRI_EINVAL, "result capacity below k");
    if (g->d.m == 0) return WTRI_OK;
    return host_result_query(g, k, out,
                             [&](wtri_tri* t, double* wv, int32_t* c, cudaStream_t s, int scale,
                                 unsigned long long* dk) {
                                 return topk_device(g, code, k, t, wv, c, s, scale, shard, nshards, dk,
                                                    p);
                             },
                             keys);
}

WTRI_API int wtri_merge_topk(int32_t nparts, const int32_t* counts, const wtri_tri* const* tris,
                             const double* const* weights, const uint64_t* const* keys, int32_t k,
                             wtri_result* out, uint64_t* out_keys) {
    if (!out) return set_error(WTRI_EINVAL, "out is NULL");
    out->count = 0;
    if (nparts < 0 || k <= 0) return set_error(WTRI_EINVAL, "need nparts >= 0 and k > 0");
    if (nparts > 0 && (!counts || !tris || !weights || !keys))
        return set_error(WTRI_EINVAL, "NULL part arrays");
    if (!out->tris || !out->weight || out->capacity < k)
        return set_error(WTRI_EINVAL, "result arrays NULL or too small");
    struct Ent {
        uint64_t key;
        wtri_tri t;
        double w;
    };
    std::vector<Ent> all;
    for (int32_t i = 0; i < nparts; i++) {
        if (counts[i] < 0) return set_error(WTRI_EINVAL, "negative part count");
        for (int32_t j = 0; j < counts[i]; j++) all.push_back({keys[i][j], tris[i][j], weights[i][j]});
    }
    auto before = [](const Ent& x, const Ent& y) {
        if (x.key != y.key) return x.key > y.key;
        if (x.t.a != y.t.a) return x.t.a < y.t.a;
        if (x.t.b != y.t.b) return x.t.b < y.t.b;
        return x.t.c < y.t.c;
    };
    const size_t keep = std::min<size_t>(all.size(), (size_t)k);
    std::partial_sort(all.begin(), all.begin() + (long)keep, all.end(), before);
    for (size_t i = 1; i < keep; i++)
        if (!before(all[i - 1], all[i]))
            return set_error(WTRI_EINVAL, "the parts share a triangle (shards must be disjoint)");
    for (size_t i = 0; i < keep; i++) {
        out->tris[i] = all[i].t;
        out->weight[i] = all[i].w;
        if (out_keys) out_keys[i] = all[i].key;
    }
    out->count = (int32_t)keep;
    return WTRI_OK;
}

WTRI_API int wtri_set_tune(wtri_graph* g, int64_t first_round, int32_t growth, int32_t t_short) {
    if (!g) return set_error(WTRI_EINVAL, "graph is NULL");
    if (first_round < 1 || growth < 2 || t_short < 1)
        return set_error(WTRI_EINVAL, "need first_round >= 1, growth >= 2, t_short >= 1");
    g->tune.first_round = first_round;
    g->tune.growth = growth;
    g->tune.t_short = t_short;
    return WTRI_OK;
}

WTRI_API int wtri_autotune(wtri_graph* g, int32_t k, int32_t reps, wtri_tune_info* info) {
    if (!g) return set_error(WTRI_EINVAL, "graph is NULL");
    WTRI_TRY(check_query(g, k));
    if (reps < 1) return set_error(WTRI_EINVAL, "reps must be positive");
    if (g->d.m == 0) {
        if (info) *info = wtri_tune_info{g->tune.first_round, g->tune.growth, g->tune.t_short, 0, 0, 0};
        return WTRI_OK;
    }
    cudaStream_t s = g->stream;
    void* buf = nullptr;
    const size_t tb = sizeof(wtri_tri) * (size_t)k, wb = 8 * (size_t)k;
    WTRI_CUDA(cudaMallocAsync(&buf, tb + wb + 64, s));
    wtri_tri* dt = (wtri_tri*)buf;
    double* dw = (double*)((char*)buf + ((tb + 15) & ~size_t(15)));
    int32_t* dc = (int32_t*)(dw + k);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // Median device time of one pass over the four p of the paper's configs.
    auto time_cfg = [&](const wtri::Tune& t, double* ms_out) -> int {
        const wtri::Tune keep = g->tune;
        g->tune = t;
        std::vector<float> ts;
        int rc = WTRI_OK;
        for (int r = 0; r <= reps && rc == WTRI_OK; r++) {  // first pass warms up
            cudaEventRecord(e0, s);
            for (int pc = 0; pc < 4 && rc == WTRI_OK; pc++) rc = topk_device(g, pc, k, dt, dw, dc, s, 1);
            cudaEventRecord(e1, s);
            cudaError_t e = cudaEventSynchronize(e1);
            if (e != cudaSuccess) rc = cuda_error(e, "autotune", __FILE__, __LINE__);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (r > 0) ts.push_back(ms);
        }
        int32_t status = 0;
        if (rc == WTRI_OK && cudaMemcpy(&status, dc, 4, cudaMemcpyDeviceToHost) == cudaSuccess && status < 0)
            rc = WTRI_ENOMEM;  // a bounded buffer filled: this setting is not usable
        g->tune = keep;
        if (rc != WTRI_OK) return rc;
        std::sort(ts.begin(), ts.end());
        *ms_out = ts[ts.size() / 2];
        return WTRI_OK;
    };
    const wtri::Tune dflt;
    double best_ms = 0, dflt_ms = 0;
    int rc = time_cfg(dflt, &dflt_ms);
    wtri::Tune best = dflt;
    best_ms = dflt_ms;
    int tried = 1;
    const int64_t firsts[] = {32, 64, 256, 1024};
    const int32_t growths[] = {4, 8, 16};
    const int32_t shorts[] = {8, 16, 32, 64, 128};
    for (int64_t f : firsts)
        for (int32_t gr : growths)
            for (int32_t ts : shorts) {
                if (rc != WTRI_OK) break;
                wtri::Tune t;
                t.first_round = f;
                t.growth = gr;
                t.t_short = ts;
                if (f == dflt.first_round && gr == dflt.growth && ts == dflt.t_short) continue;
                double ms = 0;
                const int r2 = time_cfg(t, &ms);
                tried++;
                if (r2 == WTRI_ENOMEM) continue;
                if (r2 != WTRI_OK) {
                    rc = r2;
                    break;
                }
                if (ms < best_ms) {
                    best_ms = ms;
                    best = t;
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(buf, s);
    if (rc != WTRI_OK) return rc;
    g->tune = best;
    if (info) {
        info->first_round = best.first_round;
        info->growth = best.growth;
        info->t_short = best.t_short;
        info->default_ms = dflt_ms;
        info->tuned_ms = best_ms;
        info->configs_tried = tried;
    }
    return WTRI_OK;
}

WTRI_API int wtri_autotune_buckets(wtri_graph* const* gs, int32_t ngraphs, int32_t k, int32_t reps,
                                   int32_t* buckets_tuned) {
    if (ngraphs < 0 || (ngraphs > 0 && !gs)) return set_error(WTRI_EINVAL, "bad graph array");
    // size buckets: graphs whose edge counts have the same bit length
    std::vector<int> best(65, -1);
    for (int32_t i = 0; i < ngraphs; i++) {
        if (!gs[i]) return set_error(WTRI_EINVAL, "graph " + std::to_string(i) + " is NULL");
        int b = 0;
        for (uint64_t m = (uint64_t)gs[i]->d.m; m; m >>= 1) b++;
        if (best[(size_t)b] < 0 || gs[i]->d.m > gs[(size_t)best[(size_t)b]]->d.m) best[(size_t)b] = i;
    }
    int32_t tuned = 0;
    std::vector<wtri::Tune> setting(65);
    for (int b = 0; b <= 64; b++) {
        if (best[(size_t)b] < 0) continue;
        wtri_graph* g = gs[(size_t)best[(size_t)b]];
        WTRI_TRY(wtri_autotune(g, k, reps, nullptr));
        setting[(size_t)b] = g->tune;
        tuned++;
    }
    for (int32_t i = 0; i < ngraphs; i++) {
        int b = 0;
        for (uint64_t m = (uint64_t)gs[i]->d.m; m; m >>= 1) b++;
        gs[i]->tune = setting[(size_t)b];
    }
    if (buckets_tuned) *buckets_tuned = tuned;
    return WTRI_OK;
}

WTRI_API int wtri_topk_device(const wtri_graph* g, double p, int32_t k, wtri_tri* d_tris,
                              double* d_weight, int32_t* d_count, void* stream) {
    int code = 0;
    WTRI_TRY(check_query(g, k));
    WTRI_TRY(p_to_code_for(p, g, &code));
    if (!d_tris || !d_weight || !d_count) return set_error(WTRI_EINVAL, "output pointers are NULL");
    cudaStream_t s = stream ? (cudaStream_t)stream : g->stream;
    if (g->d.m == 0) {
        WTRI_CUDA(cudaMemsetAsync(d_count, 0, sizeof(int32_t), s));
        return WTRI_OK;
    }
    return topk_device(g, code, k, d_tris, d_weight, d_count, s, 1, 0, 1, nullptr, p);
}

WTRI_API int wtri_sample_topk(const wtri_graph* g, double p, int32_t k, int64_t nsamples,
                              uint64_t seed, wtri_result* out) {
    if (!out) return set_error(WTRI_EINVAL, "out is NULL");
    out->count = 0;
    int code = 0;
    WTRI_TRY(check_query(g, k));
    WTRI_TRY(p_to_code_for(p, g, &code));
    WTRI_TRY(need_integer_weights(g, "edge sampling"));
    if (code != P_ONE && code != P_TWO && code != P_GEO)
        return set_error(WTRI_EUNSUPPORTED, "edge sampling needs p = 0, 1 or 2 (exact integer w^p)");
    if (nsamples < 0) return set_error(WTRI_EINVAL, "nsamples must be non-negative");
    if (!out->tris || !out->weight) return set_error(WTRI_EINVAL, "result arrays are NULL");
    if (out->capacity < k) return set_error(WTRI_EINVAL, "result capacity below k");
    if (g->d.m == 0 || nsamples == 0) return WTRI_OK;
    return host_result_query(g, k, out,
                             [&](wtri_tri* t, double* wv, int32_t* c, cudaStream_t s, int scale,
                                 unsigned long long*) {
                                 return sample_topk_device(g, code, k, nsamples, seed, t, wv, c, s,
                                                           scale);
                             });
}

WTRI_API int wtri_wedge_topk(const wtri_graph* g, double p, int32_t k, int64_t nsamples,
                             uint64_t seed, wtri_result* out) {
    if (!out) return set_error(WTRI_EINVAL, "out is NULL");
    out->count = 0;
    int code = 0;
    WTRI_TRY(check_query(g, k));
    WTRI_TRY(p_to_code_for(p, g, &code));
    WTRI_TRY(need_integer_weights(g, "wedge sampling"));
    if (code != P_ONE && code != P_TWO && code != P_GEO)
        return set_error(WTRI_EUNSUPPORTED, "wedge sampling needs p = 0, 1 or 2 (exact integer w^p)");
    if (nsamples < 0) return set_error(WTRI_EINVAL, "nsamples must be non-negative");
    if (nsamples >= (int64_t(1) << 31)) return set_error(WTRI_EUNSUPPORTED, "nsamples of 2^31 or more");
    if (!out->tris || !out->weight) return set_error(WTRI_EINVAL, "result arrays are NULL");
    if (out->capacity < k) return set_error(WTRI_EINVAL, "result capacity below k");
    if (g->d.m == 0 || nsamples == 0) return WTRI_OK;
    return host_result_query(g, k, out,
                             [&](wtri_tri* t, double* wv, int32_t* c, cudaStream_t s, int,
                                 unsigned long long*) {
                                 return wedge_topk_device(g, code, k, nsamples, seed, t, wv, c, s);
                             });
}

WTRI_API int wtri_sample_wedges(const wtri_graph* g, double p, int64_t nsamples, uint64_t seed,
                                int32_t* center, int32_t* jb, int32_t* jc, int32_t* tri) {
    if (!g) return set_error(WTRI_EINVAL, "graph is NULL");
    int code = 0;
    WTRI_TRY(p_to_code_for(p, g, &code));
    WTRI_TRY(need_integer_weights(g, "wedge sampling"));
    if (code != P_ONE && code != P_TWO && code != P_GEO)
        return set_error(WTRI_EUNSUPPORTED, "wedge sampling needs p = 0, 1 or 2 (exact integer w^p)");
    if (nsamples < 0) return set_error(WTRI_EINVAL, "nsamples must be non-negative");
    if (nsamples == 0) return WTRI_OK;
    if (!center || !jb || !jc || !tri) return set_error(WTRI_EINVAL, "output arrays are NULL");
    if (g->d.m == 0) {
        for (int64_t s = 0; s < nsamples; s++) {
            center[s] = jb[s] = jc[s] = -1;
            tri[3 * s] = tri[3 * s + 1] = tri[3 * s + 2] = -1;
        }
        return WTRI_OK;
    }
    return wedge_draws_host(g, code, nsamples, seed, center, jb, jc, tri);
}

WTRI_API int wtri_sample_cliques(const wtri_graph* g, int32_t q, double p, int32_t k, int64_t nsamples,
                                 uint64_t seed, int32_t* cliques, double* weights, uint64_t* keys,
                                 int32_t* count) {
    if (!g) return set_error(WTRI_EINVAL, "graph is NULL");
    if (count) *count = 0;
    if (q != 4 && q != 5) return set_error(WTRI_EINVAL, "clique size must be 4 or 5");
    if (k <= 0 || k > 65536) return set_error(WTRI_EINVAL, "k must be in [1, 65536]");
    if (!cliques || !weights || !count) return set_error(WTRI_EINVAL, "output arrays are NULL");
    int code = 0;
    WTRI_TRY(p_to_code(p, &code));
    WTRI_TRY(need_integer_weights(g, "clique sampling"));
    if (code != P_MIN && code != P_ONE && code != P_TWO && code != P_MAX)
        return set_error(WTRI_EUNSUPPORTED, "cliques rank at p in {-inf, 1, 2, +inf}");
    if (nsamples >= 0 && code != P_ONE && code != P_TWO)
        return set_error(WTRI_EUNSUPPORTED, "edge draws need w^p with p = 1 or 2");
    if (code == P_TWO && g->d.wmax > (1 << 30))
        return set_error(WTRI_EUNSUPPORTED, "p = 2 ranks cliques by a sum of squares: weights up to 2^30");
    if (g->d.m == 0) return WTRI_OK;
    return clique_topk_host(g, q, code, k, nsamples, seed, cliques, weights, keys, count);
}

WTRI_API int wtri_topk_batch(const wtri_graph* const* gs, const double* p, const int32_t* k,
                             int32_t nq, wtri_result* outs) {
    if (nq < 0) return set_error(WTRI_EINVAL, "nq must be non-negative");
    if (nq == 0) return WTRI_OK;
    if (!gs || !p || !k || !outs) return set_error(WTRI_EINVAL, "NULL batch arrays");
    std::vector<int32_t> codes((size_t)nq);
    for (int32_t i = 0; i < nq; i++) outs[i].count = 0;
    int dev = -1;
    for (int32_t i = 0; i < nq; i++) {
        if (!gs[i]) return set_error(WTRI_EINVAL, "graph " + std::to_string(i) + " is NULL");
        if (dev < 0) dev = gs[i]->device;
        if (gs[i]->device != dev) return set_error(WTRI_EINVAL, "batch graphs on different devices");
        int c = 0;
        int rc = p_to_code_for(p[i], gs[i], &c);
        if (rc == WTRI_OK) rc = need_integer_weights(gs[i], "the batched call");
        if (rc != WTRI_OK) return rc;
        if (c == P_GEN)
            return set_error(WTRI_EUNSUPPORTED,
                             "batched queries take p in {-inf, 0, 1, 2, +inf}; other p through wtri_topk");
        codes[(size_t)i] = c;
        rc = check_query(gs[i], k[i]);
        if (rc != WTRI_OK) return rc;
        if (!outs[i].tris || !outs[i].weight || outs[i].capacity < k[i])
            return set_error(WTRI_EINVAL, "result " + std::to_string(i) + " arrays NULL or too small");
    }
    return topk_batch(gs, codes.data(), k, nq, outs, gs[0]->stream, 1);
}

WTRI_API int wtri_sample_edges(const wtri_graph* g, double p, int64_t nsamples, uint64_t seed,
                               uint32_t* mark_words, int64_t words_capacity) {
    if (!g) return set_error(WTRI_EINVAL, "graph is NULL");
    int code = 0;
    WTRI_TRY(p_to_code(p, &code));
    WTRI_TRY(need_integer_weights(g, "edge sampling"));
    if (code != P_ONE && code != P_TWO && code != P_GEO)
        return set_error(WTRI_EUNSUPPORTED, "edge sampling needs p = 0, 1 or 2 (exact integer w^p)");
    if (nsamples < 0) return set_error(WTRI_EINVAL, "nsamples must be non-negative");
    const int64_t words = (g->d.m + 31) / 32;
    if (!mark_words || words_capacity < words)
        return set_error(WTRI_EINVAL, "mark array smaller than ceil(m/32) words");
    if (words == 0) return WTRI_OK;
    cudaStream_t s = g->stream;
    void* d = nullptr;
    WTRI_CUDA(cudaMallocAsync(&d, 4 * (size_t)words, s));
    int rc = WTRI_OK;
    if (nsamples == 0) {
        if (cudaMemsetAsync(d, 0, 4 * (size_t)words, s) != cudaSuccess)
            rc = cuda_error(cudaGetLastError(), "memset", __FILE__, __LINE__);
    } else {
        rc = sample_edges_device(g, code, nsamples, seed, (uint32_t*)d, s);
    }
    if (rc == WTRI_OK) {
        cudaError_t e = cudaMemcpyAsync(mark_words, d, 4 * (size_t)words, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = cuda_error(e, "mark copy", __FILE__, __LINE__);
    }
    cudaFreeAsync(d, s);
    return rc;
}

WTRI_API int wtri_graph_copy_array(const wtri_graph* g, int which, void* dst,
                                   int64_t bytes_capacity, int64_t* bytes_out) {
    if (!g) return set_error(WTRI_EINVAL, "graph is NULL");
    const int64_t n = g->d.n, m = g->d.m;
    const void* src = nullptr;
    int64_t bytes = 0;
    switch (which) {
        case WTRI_ARR_DEGREE: bytes = 4 * n; break;  // from the row offsets
        case WTRI_ARR_ROWPTR: src = g->d.rowptr; bytes = 8 * (n + 1); break;
        case WTRI_ARR_ORDER_U: src = g->d.ord_u; bytes = 4 * m; break;
        case WTRI_ARR_ORDER_V: src = g->d.ord_v; bytes = 4 * m; break;
        case WTRI_ARR_ORDER_W: src = g->d.ord_w; bytes = 4 * m; break;
        case WTRI_ARR_WCOL: src = g->d.wcol; bytes = 8 * m; break;
        case WTRI_ARR_WWT: src = g->d.wwt; bytes = 8 * m; break;
        case WTRI_ARR_WRANK: src = g->d.wrk; bytes = 8 * m; break;
        case WTRI_ARR_OROWPTR: src = g->d.orowptr; bytes = 8 * (n + 1); break;
        case WTRI_ARR_OCOL: src = g->d.ocol; bytes = 4 * m; break;
        case WTRI_ARR_OWT: src = g->d.owt; bytes = 4 * m; break;
        case WTRI_ARR_ORANK: src = g->d.ork; bytes = 4 * m; break;
        default: return set_error(WTRI_EINVAL, "unknown array id");
    }
    if (bytes_out) *bytes_out = bytes;
    if (!dst) return WTRI_OK;
    if (bytes_capacity < bytes) return set_error(WTRI_EINVAL, "destination too small");
    if (bytes == 0) return WTRI_OK;
    if (src) {
        WTRI_CUDA(cudaMemcpyAsync(dst, src, (size_t)bytes, cudaMemcpyDeviceToHost, g->stream));
        WTRI_CUDA(cudaStreamSynchronize(g->stream));
        return WTRI_OK;
    }
    // degrees: differences of the row offsets
    std::vector<int64_t> rp((size_t)n + 1);
    WTRI_CUDA(cudaMemcpyAsync(rp.data(), g->d.rowptr, 8 * ((size_t)n + 1), cudaMemcpyDeviceToHost,
                              g->stream));
    WTRI_CUDA(cudaStreamSynchronize(g->stream));
    int32_t* o = (int32_t*)dst;
    for (int64_t x = 0; x < n; x++) o[x] = (int32_t)(rp[(size_t)x + 1] - rp[(size_t)x]);
    return WTRI_OK;
}

}  // extern "C"
