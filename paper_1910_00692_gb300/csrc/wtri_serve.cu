// Serving loop with continuous batching.
//
// Graphs stay resident; requests (graph, p, k) are queued by wtri_submit.  A
// scheduler thread repeatedly
//   1. retires finished micro-batches (cudaEventQuery, no device sync):
//      results go to host memory, their device scratch and slots are freed;
//   2. admits waiting requests, oldest first, into a new micro-batch while
//      request slots (max_slots in flight) and the HBM budget (resident
//      graphs + scratch of everything in flight) allow, and launches it on a
//      free worker stream with the batched kernels.
// Requests that arrive while others run are admitted as soon as slots and
// memory free up, and several micro-batches overlap on the device (one per
// worker stream).  wtri_poll only looks at host state.
//
// Within a micro-batch, requests on the same graph with the same p are
// answered by one query at their largest k: under the total order (weight
// desc, triple asc) the top-k is exactly the first k of the top-k' for any
// k' >= k, so each request gets the prefix it asked for, identical to the
// result of its own query.  wtri_server_set_option(WTRI_SERVER_COALESCE, 0)
// (or WTRI_SERVE_COALESCE=0 in the environment at creation) runs one query
// per request.
#include <atomic>
#include <chrono>
#include <cstdlib>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "wtri_internal.cuh"

namespace wtri {
namespace {

constexpr int WORKER_STREAMS = 4;
constexpr int MAX_BATCH = 256;
constexpr size_t BATCH_FIXED_BYTES = (size_t(1) << 18) * 40 + (1u << 16);  // deferred list + slack

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Request {
    uint64_t ticket = 0;
    int32_t graph_id = 0;
    int pcode = 0;
    int32_t k = 0;
    size_t bytes = 0;  // admission estimate of its device scratch
    int state = 0;     // 0 waiting, 1 running, 2 done, 3 failed
    int rc = WTRI_OK;
    std::vector<wtri_tri> tris;
    std::vector<double> w;
    double t_submit = 0, t_done = 0;
};

struct InFlight {
    BatchPlan* plan = nullptr;
    void* dbuf = nullptr;
    size_t bytes = 0;
    int stream = -1;
    cudaEvent_t done = nullptr;
    std::vector<std::shared_ptr<Request>> reqs;
    std::vector<int> query_of;  // request i is answered by query query_of[i] of the plan
};

// Default of a new server's coalescing option (environment, read once).
bool coalesce_default() {
    static const bool on = [] {
        const char* e = getenv("WTRI_SERVE_COALESCE");
        return !(e && e[0] == '0');
    }();
    return on;
}

size_t request_bytes(int32_t k, int64_t m) {
    const size_t cap = batch_query_cap(k, m);
    return 256 + cap * 24 + (size_t)k * 20 + 512;
}

}  // namespace
}  // namespace wtri

struct wtri_server {
    uint64_t budget = 0;
    int32_t max_slots = 0;
    int device = 0;
    std::vector<wtri_graph*> graphs;
    uint64_t graph_bytes = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<std::shared_ptr<wtri::Request>> waiting;
    std::unordered_map<uint64_t, std::shared_ptr<wtri::Request>> by_ticket;
    uint64_t next_ticket = 1;
    uint64_t scratch_in_use = 0;
    int running_requests = 0;
    bool stop = false;
    std::thread worker;
    cudaStream_t streams[wtri::WORKER_STREAMS] = {};
    bool stream_busy[wtri::WORKER_STREAMS] = {};
    std::vector<wtri::InFlight> inflight;  // touched by the worker only
    uint64_t batches = 0, admitted = 0, retries = 0;
    std::atomic<bool> coalesce{true};  // same-(graph, p) requests of a micro-batch share a query
};

namespace wtri {
namespace {

void finish_batch(wtri_server* S, InFlight& f) {
    cudaStream_t s = S->streams[f.stream];
    int rc = batch_plan_collect(f.plan, f.dbuf, s);
    const double t = now_s();
    for (size_t i = 0; i < f.reqs.size(); i++) {
        auto& r = f.reqs[i];
        const int qi = f.query_of[i];
        int32_t c = rc == WTRI_OK ? batch_plan_status(f.plan, qi) : rc;
        if (c > r->k) c = r->k;  // the prefix this request asked for
        r->tris.assign((size_t)std::max(r->k, 1), wtri_tri{0, 0, 0});
        r->w.assign((size_t)std::max(r->k, 1), 0.0);
        int rrc = WTRI_OK;
        if (c == WTRI_ENOMEM) {
            {
                std::lock_guard<std::mutex> lk(S->mu);
                S->retries++;
            }
            int32_t cnt = 0;
            rrc = topk_retry_host(S->graphs[(size_t)r->graph_id], r->pcode, r->k, s, r->tris.data(),
                                  r->w.data(), &cnt);
            c = rrc == WTRI_OK ? cnt : rrc;
        } else if (c >= 0) {
            std::copy(batch_plan_tris(f.plan, qi), batch_plan_tris(f.plan, qi) + c, r->tris.begin());
            std::copy(batch_plan_weights(f.plan, qi), batch_plan_weights(f.plan, qi) + c, r->w.begin());
        }
        std::lock_guard<std::mutex> lk(S->mu);
        if (c >= 0) {
            r->tris.resize((size_t)c);
            r->w.resize((size_t)c);
            r->state = 2;
            r->rc = WTRI_OK;
        } else {
            r->state = 3;
            r->rc = c;
        }
        r->t_done = t;
    }
    cudaFreeAsync(f.dbuf, s);
    cudaEventDestroy(f.done);
    batch_plan_destroy(f.plan);
    std::lock_guard<std::mutex> lk(S->mu);
    S->scratch_in_use -= f.bytes;
    S->running_requests -= (int)f.reqs.size();
    S->stream_busy[f.stream] = false;
    S->cv.notify_all();
}

// Launches one micro-batch; on failure marks its requests failed.
void launch_batch(wtri_server* S, std::vector<std::shared_ptr<Request>>& reqs, int si, size_t bytes) {
    InFlight f;
    f.stream = si;
    f.reqs = reqs;
    f.bytes = bytes;
    cudaStream_t s = S->streams[si];
    // one query per (graph, p) at the group's largest k, or one per request
    std::vector<const wtri_graph*> gs;
    std::vector<int32_t> pc, ks;
    std::unordered_map<int64_t, int> group;
    f.query_of.resize(reqs.size());
    const bool merge = S->coalesce.load(std::memory_order_relaxed);
    for (size_t i = 0; i < reqs.size(); i++) {
        const int64_t key = (int64_t)reqs[i]->graph_id * 8 + reqs[i]->pcode;
        auto it = merge ? group.find(key) : group.end();
        if (it == group.end()) {
            if (merge) group.emplace(key, (int)gs.size());
            f.query_of[i] = (int)gs.size();
            gs.push_back(S->graphs[(size_t)reqs[i]->graph_id]);
            pc.push_back(reqs[i]->pcode);
            ks.push_back(reqs[i]->k);
        } else {
            f.query_of[i] = it->second;
            ks[(size_t)it->second] = std::max(ks[(size_t)it->second], reqs[i]->k);
        }
    }
    int rc = WTRI_OK;
    // the plan's scratch is at most the sum of its requests' estimates
    // (one of them asked for the group's largest k), so admission holds
    f.plan = batch_plan_create(gs.data(), pc.data(), ks.data(), (int32_t)gs.size());
    if (!f.plan) rc = WTRI_ENOMEM;
    if (rc == WTRI_OK && cudaMallocAsync(&f.dbuf, batch_plan_bytes(f.plan), s) != cudaSuccess) {
        cudaGetLastError();
        rc = WTRI_ENOMEM;
    }
    if (rc == WTRI_OK) rc = batch_plan_launch(f.plan, f.dbuf, s, 0);
    if (rc == WTRI_OK && (cudaEventCreateWithFlags(&f.done, cudaEventDisableTiming) != cudaSuccess ||
                          cudaEventRecord(f.done, s) != cudaSuccess))
        rc = WTRI_ECUDA;
    if (rc != WTRI_OK) {
        if (f.dbuf) cudaFreeAsync(f.dbuf, s);
        if (f.plan) batch_plan_destroy(f.plan);
        if (f.done) cudaEventDestroy(f.done);
        std::lock_guard<std::mutex> lk(S->mu);
        for (auto& r : reqs) {
            r->state = 3;
            r->rc = rc;
            r->t_done = now_s();
        }
        S->scratch_in_use -= bytes;
        S->running_requests -= (int)reqs.size();
        S->stream_busy[si] = false;
        S->cv.notify_all();
        return;
    }
    S->inflight.push_back(f);
}

void worker_loop(wtri_server* S) {
    cudaSetDevice(S->device);
    for (;;) {
        // 1. retire finished micro-batches
        for (size_t i = 0; i < S->inflight.size();) {
            cudaError_t e = cudaEventQuery(S->inflight[i].done);
            if (e == cudaSuccess) {
                finish_batch(S, S->inflight[i]);
                S->inflight.erase(S->inflight.begin() + (long)i);
            } else {
                if (e != cudaErrorNotReady) cudaGetLastError();
                i++;
            }
        }
        // 2. admit waiting requests into a new micro-batch
        std::vector<std::shared_ptr<Request>> batch;
        int si = -1;
        size_t bytes = 0;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            if (S->stop && S->waiting.empty() && S->inflight.empty()) return;
            for (int k = 0; k < WORKER_STREAMS; k++)
                if (!S->stream_busy[k]) {
                    si = k;
                    break;
                }
            const uint64_t scratch_budget = S->budget - S->graph_bytes;
            if (si >= 0) {
                bytes = BATCH_FIXED_BYTES;
                while (!S->waiting.empty() && (int)batch.size() < MAX_BATCH &&
                       S->running_requests + (int)batch.size() < S->max_slots) {
                    auto& r = S->waiting.front();
                    if (S->scratch_in_use + bytes + r->bytes > scratch_budget) break;
                    bytes += r->bytes;
                    r->state = 1;
                    batch.push_back(r);
                    S->waiting.pop_front();
                }
                if (!batch.empty()) {
                    S->scratch_in_use += bytes;
                    S->running_requests += (int)batch.size();
                    S->stream_busy[si] = true;
                    S->batches++;
                    S->admitted += batch.size();
                }
            }
            if (batch.empty()) {
                // Nothing to launch: wait for a submission, or poll the
                // running micro-batches again shortly.
                if (S->inflight.empty())
                    S->cv.wait_for(lk, std::chrono::milliseconds(50));
                else
                    S->cv.wait_for(lk, std::chrono::microseconds(20));
                continue;
            }
        }
        launch_batch(S, batch, si, bytes);
    }
}

}  // namespace
}  // namespace wtri

using namespace wtri;

extern "C" {

WTRI_API int wtri_server_create(uint64_t hbm_budget_bytes, int32_t max_slots, wtri_server** out) {
    if (!out) return set_error(WTRI_EINVAL, "out is NULL");
    *out = nullptr;
    if (max_slots <= 0) return set_error(WTRI_EINVAL, "max_slots must be positive");
    if (hbm_budget_bytes == 0) return set_error(WTRI_EINVAL, "budget must be positive");
    wtri_server* S = new (std::nothrow) wtri_server();
    if (!S) return set_error(WTRI_ENOMEM, "host allocation failed");
    S->budget = hbm_budget_bytes;
    S->max_slots = max_slots;
    S->coalesce.store(coalesce_default());
    if (cudaGetDevice(&S->device) != cudaSuccess) {
        delete S;
        return set_error(WTRI_ECUDA, "no current device");
    }
    for (int i = 0; i < WORKER_STREAMS; i++) {
        if (cudaStreamCreateWithFlags(&S->streams[i], cudaStreamNonBlocking) != cudaSuccess) {
            for (int j = 0; j < i; j++) cudaStreamDestroy(S->streams[j]);
            delete S;
            return set_error(WTRI_ECUDA, "stream creation failed");
        }
    }
    try {
        S->worker = std::thread(worker_loop, S);
    } catch (...) {
        for (int i = 0; i < WORKER_STREAMS; i++) cudaStreamDestroy(S->streams[i]);
        delete S;
        return set_error(WTRI_ENOMEM, "could not start the scheduler thread");
    }
    *out = S;
    return WTRI_OK;
}

WTRI_API int wtri_server_add_graph(wtri_server* S, wtri_graph* g, int32_t* graph_id) {
    if (!S || !g || !graph_id) return set_error(WTRI_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    if (g->device != S->device) return set_error(WTRI_EINVAL, "graph on another device");
    WTRI_TRY(need_integer_weights(g, "the server"));
    if (S->graph_bytes + (uint64_t)g->bytes > S->budget)
        return set_error(WTRI_ENOMEM, "graph does not fit the server's HBM budget");
    S->graph_bytes += (uint64_t)g->bytes;
    S->graphs.push_back(g);
    *graph_id = (int32_t)S->graphs.size() - 1;
    return WTRI_OK;
}

WTRI_API int wtri_submit(wtri_server* S, int32_t graph_id, double p, int32_t k, uint64_t* ticket) {
    if (!S || !ticket) return set_error(WTRI_EINVAL, "NULL argument");
    int code = 0;
    WTRI_TRY(p_to_code(p, &code));
    if (code == P_GEN)
        return set_error(WTRI_EUNSUPPORTED,
                         "the server takes p in {-inf, 0, 1, 2, +inf}; other p through wtri_topk");
    if (k <= 0) return set_error(WTRI_EINVAL, "k must be positive");
    if (k > 65536) return set_error(WTRI_EUNSUPPORTED, "k above 65536");
    auto r = std::make_shared<Request>();
    r->pcode = code;
    r->k = k;
    r->t_submit = now_s();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (graph_id < 0 || graph_id >= (int32_t)S->graphs.size())
            return set_error(WTRI_ENOTFOUND, "unknown graph id");
        if (code == P_GEO && S->graphs[(size_t)graph_id]->d.wmax > GEO_WMAX)
            return set_error(WTRI_EUNSUPPORTED, "p = 0 needs weights below 2^21 (exact product key)");
        r->bytes = request_bytes(k, S->graphs[(size_t)graph_id]->d.m);
        if (S->stop) return set_error(WTRI_EINVAL, "server is shutting down");
        if (S->graph_bytes + BATCH_FIXED_BYTES + r->bytes > S->budget)
            return set_error(WTRI_ENOMEM, "request scratch can never fit the HBM budget");
        r->graph_id = graph_id;
        r->ticket = S->next_ticket++;
        S->waiting.push_back(r);
        S->by_ticket[r->ticket] = r;
        *ticket = r->ticket;
    }
    S->cv.notify_all();
    return WTRI_OK;
}

WTRI_API int wtri_poll_timed(wtri_server* S, uint64_t ticket, wtri_result* out, double* latency_s) {
    if (!S || !out) return set_error(WTRI_EINVAL, "NULL argument");
    std::shared_ptr<Request> r;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->by_ticket.find(ticket);
        if (it == S->by_ticket.end()) return set_error(WTRI_ENOTFOUND, "unknown ticket");
        r = it->second;
        if (r->state < 2) return WTRI_PENDING;
        if (r->state == 2 && (!out->tris || !out->weight || out->capacity < (int32_t)r->tris.size()))
            return set_error(WTRI_EINVAL, "result arrays NULL or too small");
        S->by_ticket.erase(it);
    }
    if (latency_s) *latency_s = r->t_done - r->t_submit;
    if (r->state == 3) {
        out->count = 0;
        return set_error(r->rc, "request failed");
    }
    std::copy(r->tris.begin(), r->tris.end(), out->tris);
    std::copy(r->w.begin(), r->w.end(), out->weight);
    out->count = (int32_t)r->tris.size();
    return WTRI_OK;
}

WTRI_API int wtri_poll(wtri_server* S, uint64_t ticket, wtri_result* out) {
    return wtri_poll_timed(S, ticket, out, nullptr);
}

WTRI_API int wtri_server_stats(wtri_server* S, uint64_t* batches, uint64_t* admitted, int32_t* waiting,
                               int32_t* running, uint64_t* scratch_bytes, uint64_t* retries) {
    if (!S) return set_error(WTRI_EINVAL, "server is NULL");
    std::lock_guard<std::mutex> lk(S->mu);
    if (retries) *retries = S->retries;
    if (batches) *batches = S->batches;
    if (admitted) *admitted = S->admitted;
    if (waiting) *waiting = (int32_t)S->waiting.size();
    if (running) *running = S->running_requests;
    if (scratch_bytes) *scratch_bytes = S->scratch_in_use;
    return WTRI_OK;
}

WTRI_API void wtri_server_free(wtri_server* S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv.notify_all();
    if (S->worker.joinable()) S->worker.join();
    for (int i = 0; i < WORKER_STREAMS; i++) {
        cudaStreamSynchronize(S->streams[i]);
        cudaStreamDestroy(S->streams[i]);
    }
    delete S;
}

}  // extern "C"

extern "C" WTRI_API int wtri_server_set_option(wtri_server* S, int option, int64_t value) {
    using namespace wtri;
    if (!S) return set_error(WTRI_EINVAL, "server is NULL");
    switch (option) {
        case WTRI_SERVER_COALESCE:
            S->coalesce.store(value != 0);
            return WTRI_OK;
        default:
            return set_error(WTRI_EINVAL, "unknown server option");
    }
}
