// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>

#include "../../include/wtri.h"

namespace wtri {

// ---------------------------------------------------------------------------
// Errors: every host function returns a WTRI_* code; the message goes to the
// thread-local last-error slot.
// ---------------------------------------------------------------------------
int set_error(int code, const std::string& msg);
int cuda_error(cudaError_t e, const char* what, const char* file, int line);

#define WTRI_CUDA(call)                                                        \
    do {                                                                       \
        cudaError_t e_ = (call);                                               \
        if (e_ != cudaSuccess) return ::wtri::cuda_error(e_, #call, __FILE__, __LINE__); \
    } while (0)

#define WTRI_TRY(call)                     \
    do {                                   \
        int rc_ = (call);                  \
        if (rc_ != WTRI_OK) return rc_;    \
    } while (0)

// Device-side error bits (written to a status word; read by the host).
enum : uint32_t {
    DEV_ERR_SELF_LOOP = 1u << 0,
    DEV_ERR_RANGE = 1u << 1,
    DEV_ERR_WEIGHT = 1u << 2,
    DEV_ERR_DUPLICATE = 1u << 3,
    DEV_ERR_INTERNAL = 1u << 4,   // an invariant of the path failed
    DEV_ERR_OVERFLOW = 1u << 5,   // a bounded device buffer filled up
    DEV_ERR_TIMEOUT = 1u << 6,    // a bounded wait ran out
};

// p codes (template parameter of the scoring kernels).  P_GEO is p = 0, the
// geometric mean (Eq. 1's limit), ranked by the exact product of the weights.
// P_GEN is any other finite p (p = -1, the harmonic mean; p = 3; ...): no
// exact 64-bit integer key exists there, so the key is the fp64 mean itself
// (its bit pattern, which orders positive doubles like their values).
enum PCode : int { P_MIN = 0, P_ONE = 1, P_TWO = 2, P_MAX = 3, P_GEO = 4, P_GEN = 5 };
constexpr int P_COUNT = 6;
// Phase-timer name of a query at p code P ("query_p=...").
const char* query_name(int pcode);
// Largest weight for which the product key of p = 0 fits 63 bits.
constexpr int32_t GEO_WMAX = (1 << 21) - 1;

int p_to_code(double p, int* code);  // any finite p (general p -> P_GEN)
// p_to_code, and p = 0 only for graphs whose weights keep the product key exact.
int p_to_code_for(double p, const wtri_graph* g, int* code);
// WTRI_EUNSUPPORTED for a float-weight graph: `what` needs integer weights.
int need_integer_weights(const wtri_graph* g, const char* what);

// ---------------------------------------------------------------------------
// Device-resident graph (all arrays library-owned device memory).
// Layouts (r is an edge's position in the edge order: weight desc, input
// index asc):
//   ord_u/v/w[r]          edge order
//   rowptr[n+1]           offsets of the weight-sorted lists (degree d_x =
//                         rowptr[x+1] - rowptr[x])
//   wcol/wwt/wrk[2m]      per-vertex lists in edge order (weight-sorted)
//   orowptr[n+1]          offsets of the oriented lists
//   ocol/owt/ork[m]       oriented lists by neighbour id: each edge once, at
//                         its endpoint of lower (degree, id) rank; the
//                         lookup of edge {a, b} searches the one list that
//                         can hold it
// 48 bytes per edge and 16 per vertex.
// ---------------------------------------------------------------------------
struct DevGraph {
    int32_t n;
    int64_t m;
    int32_t wmax;
    int32_t maxdeg;
    int32_t fw;  // weights are positive fp32 bit patterns (1) or integers (0)
    const int64_t* rowptr;
    const int64_t* orowptr;
    const int32_t* ord_u;
    const int32_t* ord_v;
    const int32_t* ord_w;
    const int32_t* wcol;
    const int32_t* wwt;
    const int32_t* wrk;
    const int32_t* ocol;
    const int32_t* owt;
    const int32_t* ork;
};

}  // namespace wtri

struct wtri_batch_plan;  // defined in wtri_batch.cu

namespace wtri {
// Query schedule: rounds over [0, first_round), then ranges growing by
// `growth`; threads scan t_short wedges inline before deferring.
struct Tune {
    int64_t first_round = 64;
    int32_t growth = 8;
    int32_t t_short = 32;
};
}  // namespace wtri

struct wtri_graph {
    wtri::DevGraph d;
    cudaStream_t stream;
    int device;
    void* base;        // one allocation holding every array
    int64_t bytes;
    wtri::Tune tune;   // set by wtri_autotune; read by every later query
};

namespace wtri {

// Build (wtri_build.cu).
// fw: w holds positive fp32 values (their bit patterns), else integers.
int build_graph(int32_t n, int64_t m, const int32_t* u, const int32_t* v, const int32_t* w,
                int on_device, cudaStream_t stream, wtri_graph** out, int fw = 0);

// Exact top-k (wtri_topk.cu).  Writes device outputs; status (count or a
// negative code) to d_count.  'retry_scale' enlarges the scratch buffers.
// gp: the value of p for P_GEN (ignored otherwise).
int topk_device(const wtri_graph* g, int pcode, int32_t k, wtri_tri* d_tris, double* d_weight,
                int32_t* d_count, cudaStream_t stream, int retry_scale, int shard = 0,
                int nshards = 1, unsigned long long* d_keys = nullptr, double gp = 0.0);

// Edge sampling (wtri_topk.cu).
int sample_topk_device(const wtri_graph* g, int pcode, int32_t k, int64_t nsamples,
                       uint64_t seed, wtri_tri* d_tris, double* d_weight, int32_t* d_count,
                       cudaStream_t stream, int retry_scale);
// Only the draws: bitmap over edge-order positions (ceil(m/32) words).
int sample_edges_device(const wtri_graph* g, int pcode, int64_t nsamples, uint64_t seed,
                        uint32_t* d_mark, cudaStream_t stream);

// Weighted wedge sampling (wtri_wedge.cu), p codes P_GEO, P_ONE, P_TWO.
int wedge_topk_device(const wtri_graph* g, int pcode, int32_t k, int64_t nsamples, uint64_t seed,
                      wtri_tri* d_tris, double* d_weight, int32_t* d_count, cudaStream_t s);
// Top-k q-cliques (q = 4, 5) on the edges drawn at p (every edge when
// nsamples < 0); host outputs.
int clique_topk_host(const wtri_graph* g, int q, int pcode, int32_t k, int64_t nsamples, uint64_t seed,
                     int32_t* h_ids, double* h_w, uint64_t* h_keys, int32_t* h_count);
int wedge_draws_host(const wtri_graph* g, int pcode, int64_t nsamples, uint64_t seed, int32_t* center,
                     int32_t* jb, int32_t* jc, int32_t* tri);

// Batched top-k (wtri_batch.cu): host results, optional CUDA-graph capture.
int topk_batch(const wtri_graph* const* gs, const int32_t* pcodes, const int32_t* ks, int32_t nq,
               wtri_result* outs, cudaStream_t s, int use_graph);
// Pieces of a batch for the serving loop: plan (host), launch into one device
// scratch block (bytes from batch_plan_bytes), collect (synchronizes).
typedef ::wtri_batch_plan BatchPlan;
uint32_t batch_query_cap(int32_t k, int64_t m);
BatchPlan* batch_plan_create(const wtri_graph* const* gs, const int32_t* pcodes, const int32_t* ks,
                             int32_t nq);
size_t batch_plan_bytes(const BatchPlan* P);
int batch_plan_launch(BatchPlan* P, void* dbuf, cudaStream_t s, int use_graph);
int batch_plan_collect(BatchPlan* P, void* dbuf, cudaStream_t s);
int32_t batch_plan_status(const BatchPlan* P, int i);
const wtri_tri* batch_plan_tris(const BatchPlan* P, int i);
const double* batch_plan_weights(const BatchPlan* P, int i);
void batch_plan_destroy(BatchPlan* P);
int topk_retry_host(const wtri_graph* g, int pcode, int32_t k, cudaStream_t s, wtri_tri* htri,
                    double* hw, int32_t* count);

// Phase timers / launch counter (wtri_prof.cu).  'bytes' is the phase's
// share of the algorithmic bytes; 'moved' the bytes its accesses move by
// design (negative: the same as 'bytes'); 'launches' the number of kernels
// it launches.
void prof_begin(const char* name, cudaStream_t s, double bytes, int launches, double moved = -1.0);
void prof_end(cudaStream_t s);
void count_launches(int launches);  // launch counter only, no events

struct ProfScope {
    cudaStream_t s;
    ProfScope(const char* name, cudaStream_t st, double bytes, int launches, double moved = -1.0)
        : s(st) {
        prof_begin(name, st, bytes, launches, moved);
    }
    ~ProfScope() { prof_end(s); }
};

// Instrumented query byte counting (wtri_topk.cu): when on, the query
// kernels add the bytes of every global load they issue on the adjacency
// structures to a per-device counter.
bool query_bytes_on();
unsigned long long* query_bytes_counter();  // device address for the current device

// Shared launch helpers.
inline unsigned int ceil_div_u(int64_t a, int64_t b) { return (unsigned int)((a + b - 1) / b); }
int sm_count();  // of the current device

// Raises a kernel's dynamic shared-memory limit to 'bytes' on the current
// device.  The attribute belongs to the device that is current when it is
// set, so 'done' keeps one bit per device (ordinals 0..63; higher ordinals
// set the attribute on every call).  Two threads may both set it the first
// time: the call is idempotent.
int smem_optin(const void* fn, int bytes, std::atomic<uint64_t>& done);

// Device-wide exclusive scan of int32 counts into int64 offsets (n+1
// outputs; out[n] = total).  Scratch is stream-ordered.
int exclusive_scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, cudaStream_t s);

}  // namespace wtri
