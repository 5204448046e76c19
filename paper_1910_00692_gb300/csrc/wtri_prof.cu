// Launch counting and CUDA-event phase timers.
//
// Every kernel launch of the library goes through prof_begin/prof_end with a
// phase name, the number of launches it covers and two byte figures: the
// phase's share of the path's algorithmic bytes (each input read once and
// each resident output written once; a sort counts one read and one write of
// its payload however many passes it takes, spread evenly over the passes,
// and helper kernels such as histograms count none), and the bytes the
// phase's own accesses move by its design (every pass of a sort reads and
// writes its records).  When timing is enabled the pair records CUDA events
// on the launching stream; wtri_prof_read / wtri_prof_read_ex resolve them
// and report per-phase calls, device time and bytes.  The launch counter is
// always on (one atomic add per phase).
#include <cuda_runtime.h>
#include <string.h>

#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "wtri_internal.cuh"

namespace wtri {
namespace {

std::atomic<long long> g_launches{0};
std::atomic<int> g_enabled{0};

struct Pending {
    std::string name;
    cudaEvent_t a, b;
    double bytes;
    double moved;
};

struct Agg {
    long long calls = 0;
    double ms = 0.0;
    double bytes = 0.0;
    double moved = 0.0;
};

std::mutex g_mu;
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_free_events;
std::map<std::string, Agg> g_agg;

thread_local std::vector<Pending> t_stack;

cudaEvent_t get_event() {
    cudaEvent_t e = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_free_events.empty()) {
            e = g_free_events.back();
            g_free_events.pop_back();
        }
    }
    if (!e) cudaEventCreate(&e);
    return e;
}

void resolve_locked() {
    for (auto& p : g_pending) {
        float ms = 0.f;
        cudaEventSynchronize(p.b);
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            Agg& a = g_agg[p.name];
            a.calls++;
            a.ms += ms;
            a.bytes += p.bytes;
            a.moved += p.moved;
        }
        g_free_events.push_back(p.a);
        g_free_events.push_back(p.b);
    }
    g_pending.clear();
}

}  // namespace

void prof_begin(const char* name, cudaStream_t s, double bytes, int launches, double moved) {
    g_launches.fetch_add(launches, std::memory_order_relaxed);
    if (!g_enabled.load(std::memory_order_relaxed)) return;
    Pending p;
    p.name = name;
    p.bytes = bytes;
    p.moved = moved < 0 ? bytes : moved;
    p.a = get_event();
    p.b = get_event();
    cudaEventRecord(p.a, s);
    t_stack.push_back(p);
}

void count_launches(int launches) { g_launches.fetch_add(launches, std::memory_order_relaxed); }

void prof_end(cudaStream_t s) {
    if (!g_enabled.load(std::memory_order_relaxed) || t_stack.empty()) return;
    Pending p = t_stack.back();
    t_stack.pop_back();
    cudaEventRecord(p.b, s);
    std::lock_guard<std::mutex> lk(g_mu);
    g_pending.push_back(p);
}

}  // namespace wtri

using namespace wtri;

extern "C" {

WTRI_API void wtri_prof_enable(int on) { g_enabled.store(on ? 1 : 0); }

WTRI_API void wtri_prof_reset(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    resolve_locked();
    g_agg.clear();
}

WTRI_API long long wtri_launch_count(void) { return g_launches.load(); }

WTRI_API int wtri_prof_read_ex(int idx, char* name, int name_cap, long long* calls, double* ms,
                               double* bytes, double* moved) {
    std::lock_guard<std::mutex> lk(g_mu);
    resolve_locked();
    if (idx < 0 || idx >= (int)g_agg.size()) return WTRI_ENOTFOUND;
    auto it = g_agg.begin();
    std::advance(it, idx);
    if (name && name_cap > 0) {
        strncpy(name, it->first.c_str(), (size_t)name_cap - 1);
        name[name_cap - 1] = 0;
    }
    if (calls) *calls = it->second.calls;
    if (ms) *ms = it->second.ms;
    if (bytes) *bytes = it->second.bytes;
    if (moved) *moved = it->second.moved;
    return WTRI_OK;
}

WTRI_API int wtri_prof_read(int idx, char* name, int name_cap, long long* calls, double* ms,
                            double* bytes) {
    return wtri_prof_read_ex(idx, name, name_cap, calls, ms, bytes, nullptr);
}

}  // extern "C"
