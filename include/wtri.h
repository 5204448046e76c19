/*
 * wtri — exact top-k weighted triangles on one GPU (sm_103a).
 *
 * C ABI of libwtri.so.  Plain pointers and sizes only; no exceptions cross
 * this boundary and the library never aborts, traps or exits.  Every entry
 * point returns one of the WTRI_* codes below; wtri_last_error() gives a
 * thread-local message for the last failing call on the calling thread.
 *
 * Problem (Kumar, Liu, Charikar, Benson, "Retrieving Top Weighted Triangles
 * in Graphs", WSDM 2020, Section 1): G = (V, E, w) is a simple undirected
 * graph with positive integer edge weights.  A triangle {a, b, c} weighs the
 * generalized p-mean of its three edge weights (Eq. 1):
 *     m_p = ((w_ab^p + w_bc^p + w_ac^p) / 3)^(1/p),
 * with p = +inf the max, p = -inf the min and p = 0 the geometric mean
 * (abc)^(1/3), the limit of Eq. 1 as p -> 0.  p = 0 is refused
 * (WTRI_EUNSUPPORTED) on a graph with a weight of 2^21 or more (its exact
 * product key would not fit 63 bits).
 *
 * Results are ranked by a total order: weight descending, then the sorted
 * vertex triple (a < b < c) ascending.  The paper notes that ties may make
 * several answers valid (Section 3.2); the triple order makes the answer
 * unique.  For p in {-inf, 0, 1, 2, +inf} ranking uses exact integer keys
 * (a+b+c for p=1, a^2+b^2+c^2 for p=2, a*b*c for p=0, max, min), never the
 * floating value; the reported fp64 weight is (a+b+c)/3.0,
 * sqrt((a^2+b^2+c^2)/3.0), cbrt(a*b*c), max or min.
 *
 * Any other finite p (the harmonic mean p = -1, p = -2, p = 0.5, p = 3, ...)
 * has no exact 64-bit integer key.  wtri_topk, wtri_topk_device,
 * wtri_topk_device_noalloc and wtri_topk_shard then rank by the fp64 mean
 * itself, computed from Eq. 1 with the weights in ascending order and the
 * largest (p > 0) or smallest (p < 0) factored out so that no power
 * overflows: m_p = s * (((a/s)^p + (b/s)^p + (c/s)^p)/3)^(1/p).  Means that
 * differ by less than fp64 rounding may rank either way; the set returned
 * is exact except for triangles within that rounding of the k-th mean.  The
 * batched and serving calls and the samplers take only the five exact p.
 *
 * A graph with fewer than k triangles returns all of them: count < k
 * (Section 3.2, "provided the graph has at least k triangles").
 *
 * Device memory behind a wtri_graph is owned by the library and freed by
 * wtri_graph_free.  A graph is immutable after wtri_build_csr; queries on
 * one graph from several host threads are safe (each query uses its own
 * stream-ordered scratch).
 */
#ifndef WTRI_H
#define WTRI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define WTRI_API __attribute__((visibility("default")))

/* Return codes. */
enum {
    WTRI_OK = 0,
    WTRI_PENDING = 1,         /* wtri_poll: the request is not finished yet */
    WTRI_EINVAL = -1,         /* bad argument or invalid graph */
    WTRI_ENOMEM = -2,         /* device or host allocation failed, or over budget */
    WTRI_ECUDA = -3,          /* a CUDA runtime call failed */
    WTRI_ETIMEOUT = -4,       /* a bounded device-side wait ran out */
    WTRI_EUNSUPPORTED = -5,   /* valid request outside what this build supports */
    WTRI_ENOTFOUND = -6       /* unknown ticket or graph id */
};

typedef struct wtri_graph wtri_graph;
typedef struct wtri_server wtri_server;

/* One triangle, vertex ids ascending (a < b < c). */
typedef struct {
    int32_t a, b, c;
} wtri_tri;

/* Caller-owned HOST result arrays.  capacity >= k entries in tris and weight.
 * On success count = min(k, #triangles); entries are in rank order.  On
 * error count = 0 and nothing else is written. */
typedef struct {
    wtri_tri* tris;
    double* weight;
    int32_t capacity;
    int32_t count;
} wtri_result;

/*
 * Builds the device-resident graph (the preprocessing of Algorithm 2 and of
 * the edge sampler of Section 4.1):
 *   - validation: ids in [0, n), no self-loops, weights > 0, no repeated
 *     undirected pair (Section 1: simple graph, positive weights);
 *   - the edge order: edges sorted by weight descending (Algorithm 2, first
 *     step), ties by input index ascending, so the order is total;
 *   - per-vertex neighbour lists N(a) in that edge order (weight-sorted);
 *   - the symmetric adjacency with rows ascending by neighbour id;
 *   - the degree orientation of NodeIterator++ (Section 5.2): vertices ranked
 *     by (degree, id), each edge stored once from its lower-ranked endpoint,
 *     rows ascending by id.
 *
 * n        number of vertices (ids 0..n-1), 1 <= n <= 2^31-1.
 * m        number of undirected edges, 0 <= m <= 2^30.
 * u, v, w  m int32 each: edge i joins u[i] and v[i] with weight w[i].  Each
 *          undirected pair appears once, in either orientation.
 * on_device 0: u, v, w are host pointers (copied in on the stream);
 *          1: device pointers (read in place, not retained after return).
 * cuda_stream a cudaStream_t to order the build on (NULL = legacy default);
 *          the graph remembers it for wtri_topk / wtri_sample_topk.
 * out      receives the new graph.  The call returns after the build has
 *          completed on the device.
 *
 * Errors: WTRI_EINVAL (n <= 0, m < 0, NULL pointers, an invalid edge or a
 * repeated pair; the message names the first offending edge index when it
 * is known), WTRI_ENOMEM, WTRI_ECUDA.  *out is NULL on error.
 */
WTRI_API int wtri_build_csr(int32_t n, int64_t m, const int32_t* u, const int32_t* v,
                            const int32_t* w, int on_device, void* cuda_stream,
                            wtri_graph** out);

/*
 * The same build for real weights (Eq. 1 over positive reals): w holds m
 * positive finite fp32 values (WTRI_EINVAL for zero, negative, infinite or
 * NaN weights).  Positive floats order like their bit patterns, so the
 * graph keeps the bits and the edge order is weight descending as above.
 * Queries on such a graph rank p = -inf and +inf by the exact min / max and
 * every other finite p (0 included: the geometric mean) by the fp64 mean,
 * with the set-equality rule of the fp64 keys (two means closer than fp64
 * rounding may rank either way).  wtri_graph_info's max_weight is then the
 * largest weight's bit pattern.  The samplers, the batched call and the
 * server take integer weights only (WTRI_EUNSUPPORTED).
 */
WTRI_API int wtri_build_csr_f32(int32_t n, int64_t m, const int32_t* u, const int32_t* v,
                                const float* w, int on_device, void* cuda_stream,
                                wtri_graph** out);

/* Frees the graph's device memory.  NULL is a no-op. */
WTRI_API void wtri_graph_free(wtri_graph* g);

/* Basic facts about a built graph (any pointer may be NULL). */
WTRI_API int wtri_graph_info(const wtri_graph* g, int32_t* n, int64_t* m, int32_t* max_degree,
                             int32_t* max_weight, int64_t* device_bytes);

/*
 * Exact top-k triangles by generalized p-mean (Eq. 1), the problem that
 * Algorithm 2 solves.  Runs on the graph's stream, then copies the k results
 * to the caller's host arrays and returns when they are there.
 *
 * p   any non-NaN value (NaN -> WTRI_EINVAL): -INFINITY, 0.0, 1.0, 2.0 and
 *     +INFINITY rank by exact keys, any other finite p by the fp64 mean
 *     (see above); 0.0 on a graph with a weight of 2^21 or more ->
 *     WTRI_EUNSUPPORTED.
 * k   1 <= k <= out->capacity and k <= 65536 (WTRI_EUNSUPPORTED above).
 */
WTRI_API int wtri_topk(const wtri_graph* g, double p, int32_t k, wtri_result* out);

/*
 * Same query, fully stream-ordered and with DEVICE outputs: nothing is
 * copied to the host and the call does not synchronize (it may be captured
 * in a CUDA graph after one warm-up call with the same g, p, k).
 *
 * d_tris    device array of k wtri_tri.
 * d_weight  device array of k doubles.
 * d_count   device int32: min(k, #triangles) on completion, or a negative
 *           WTRI_* code if the device detected an error (e.g. an internal
 *           buffer overflowed: the host-result wtri_topk retries such a
 *           query with larger buffers; this variant reports it).
 * stream    cudaStream_t to run on (NULL = the graph's stream).
 */
WTRI_API int wtri_topk_device(const wtri_graph* g, double p, int32_t k, wtri_tri* d_tris,
                              double* d_weight, int32_t* d_count, void* stream);

/*
 * wtri_topk_device without any allocation.  The paper has no counterpart:
 * this exists for callers that cannot allocate device memory while they
 * run, such as a server that hands all device memory to its own caching
 * allocator at start-up, or a latency-critical loop that must never block
 * on cudaMalloc/cudaMallocAsync.  Arguments, outputs and results are those
 * of wtri_topk_device.
 *
 * Scratch comes from one fixed array inside the library: about 26 MB
 * (1,048,576 candidate triangles and 65,536 deferred scans) that every GPU
 * loading the library keeps until the process exits.  k above 16384 is
 * rejected with WTRI_EINVAL.  If a query produces more candidates than the
 * array holds, d_count receives WTRI_ENOMEM; use wtri_topk_device then.
 * All calls share the array (its status word is cleared at the start of
 * each call), so calls that overlap on the GPU, on different streams or
 * from different host threads, race: serialize them.  The first call on a
 * device looks up the array's device address with that device current;
 * make that first call before any stream capture.
 */
WTRI_API int wtri_topk_device_noalloc(const wtri_graph* g, double p, int32_t k, wtri_tri* d_tris,
                                      double* d_weight, int32_t* d_count, void* stream);

/*
 * One shard of a query split across GPUs (Section 2 of the paper discusses
 * partitioned triangle enumeration; the split here is this library's).
 * Every triangle belongs to its first edge in the edge order; the edges are
 * dealt to nshards shards in chunks of 1024 consecutive positions,
 * round-robin.  Returns the exact top-k of the triangles whose first edge
 * belongs to `shard` (results as wtri_topk) and their ranking keys
 * (a+b+c, a^2+b^2+c^2, max, min or a*b*c; for other p the fp64 mean's bit
 * pattern) in keys[0..count).  The union of all
 * shards' results holds the global top-k: merge them with wtri_merge_topk.
 * 0 <= shard < nshards; keys has room for k entries.
 */
WTRI_API int wtri_topk_shard(const wtri_graph* g, double p, int32_t k, int32_t shard,
                             int32_t nshards, wtri_result* out, uint64_t* keys);

/*
 * Host-side merge of per-shard results: the k best of all parts under the
 * total order (key desc, triple asc), with their weights and (if out_keys
 * is not NULL) keys.  Part i has counts[i] entries in tris[i], weights[i],
 * keys[i].  Parts must be disjoint (WTRI_EINVAL if a triangle repeats).
 * Pure host code: no device needed.
 */
WTRI_API int wtri_merge_topk(int32_t nparts, const int32_t* counts, const wtri_tri* const* tris,
                             const double* const* weights, const uint64_t* const* keys, int32_t k,
                             wtri_result* out, uint64_t* out_keys);

/*
 * Batched exact top-k: query i asks for the top-k[i] triangles of gs[i] at
 * p[i] (same problem and result format as wtri_topk, results in outs[i]).
 * All queries run in one launch sequence captured in a CUDA graph on the
 * first graph's stream: each phase kernel covers every query at once, and
 * each query keeps its own threshold and candidate buffer.  Graphs must be
 * on one device.  Returns after all results are in the host arrays.  No
 * counterpart in the paper (whose algorithms answer one query at a time).
 */
WTRI_API int wtri_topk_batch(const wtri_graph* const* gs, const double* p, const int32_t* k,
                             int32_t nq, wtri_result* outs);

/*
 * Serving with continuous batching (no counterpart in the paper).
 *
 * wtri_server_create: a server with an HBM budget (bytes: resident graphs
 *   plus the scratch of every request in flight) and at most max_slots
 *   requests running at once.  A scheduler thread admits waiting requests,
 *   oldest first, as slots and budget free up, and launches them as
 *   micro-batches on its own worker streams (several overlap on the
 *   device).  Requests of one micro-batch on the same graph with the same p
 *   share one query at their largest k; each still receives exactly its own
 *   top-k (the first k of that answer under the total order), the same as
 *   wtri_topk would return.  The environment variable WTRI_SERVE_COALESCE=0
 *   runs one query per request instead.  The server uses the device current
 *   at creation.
 * wtri_server_add_graph: registers a built graph (borrowed: it must outlive
 *   the server); its device bytes count against the budget (WTRI_ENOMEM if
 *   it does not fit).  *graph_id receives its id.
 * wtri_submit: queues the query (graph_id, p, k) and returns at once with a
 *   ticket.  WTRI_ENOTFOUND for an unknown graph, WTRI_ENOMEM if the
 *   request could never fit the budget, p and k as in wtri_topk.
 * wtri_poll: WTRI_PENDING while the request waits or runs; otherwise copies
 *   the result (as wtri_topk would return it) to out and retires the ticket
 *   (WTRI_OK), or returns the request's error.  Reads host state only.
 *   WTRI_ENOTFOUND for an unknown or retired ticket.
 * wtri_poll_timed: wtri_poll that also returns the seconds from submission
 *   to completion.
 * wtri_server_stats: micro-batches launched, requests admitted, requests
 *   waiting and running, scratch bytes in flight, requests re-run alone
 *   after overflowing their batched buffers (any pointer may be NULL).
 * wtri_server_free: finishes every queued request, stops the scheduler and
 *   frees the server (not the graphs).
 */
WTRI_API int wtri_server_create(uint64_t hbm_budget_bytes, int32_t max_slots, wtri_server** out);
WTRI_API int wtri_server_add_graph(wtri_server* s, wtri_graph* g, int32_t* graph_id);
WTRI_API int wtri_submit(wtri_server* s, int32_t graph_id, double p, int32_t k, uint64_t* ticket);
WTRI_API int wtri_poll(wtri_server* s, uint64_t ticket, wtri_result* out);
WTRI_API int wtri_poll_timed(wtri_server* s, uint64_t ticket, wtri_result* out, double* latency_s);
WTRI_API int wtri_server_stats(wtri_server* s, uint64_t* batches, uint64_t* admitted, int32_t* waiting,
                               int32_t* running, uint64_t* scratch_bytes, uint64_t* retries);
WTRI_API void wtri_server_free(wtri_server* s);

/*
 * Server options (no counterpart in the paper).
 * WTRI_SERVER_COALESCE (default 1, or 0 when the environment has
 * WTRI_SERVE_COALESCE=0 at creation): requests of one micro-batch that ask
 * the same graph at the same p share one query at their largest k (each
 * gets the prefix it asked for: under the total order the top-k is the
 * first k of any top-k' with k' >= k).  0 runs one query per request.
 * Takes effect for micro-batches launched after the call.
 */
enum { WTRI_SERVER_COALESCE = 1 };
WTRI_API int wtri_server_set_option(wtri_server* s, int option, int64_t value);

/*
 * Query schedule tuning (no counterpart in the paper).  A query sweeps the
 * edge order in rounds over [0, first_round), then ranges growing by
 * `growth`; a thread scans up to t_short wedges of an edge itself and hands
 * longer scans to a block that stages the closing vertex's list in shared
 * memory, so t_short is the boundary between the short-list and long-list
 * strategies.  Defaults: 64, 8, 32.
 *
 * wtri_autotune times a grid of settings (first_round in {32, 64, 256,
 * 1024}, growth in {4, 8, 16}, t_short in {8, 16, 32, 64, 128}) on the
 * graph itself with CUDA events — one exact top-k query at each of
 * p = -inf, 1, 2, +inf, median of `reps` — and keeps the fastest for every
 * later query on that graph (single, device and sampled queries read it;
 * a batched query reads its t_short, the batch keeping one round schedule,
 * the defaults, for all its queries; results do not depend on it).  Not thread-safe against queries
 * running on the same graph.  wtri_set_tune sets the values directly.
 */
typedef struct {
    int64_t first_round;
    int32_t growth;
    int32_t t_short;
    double default_ms;   /* the four queries with the defaults */
    double tuned_ms;     /* ... with the chosen setting */
    int32_t configs_tried;
} wtri_tune_info;

WTRI_API int wtri_autotune(wtri_graph* g, int32_t k, int32_t reps, wtri_tune_info* info);

/*
 * Tuning for a collection of graphs (e.g. the graphs of a batch): graphs
 * are grouped by size (the bit length of their edge count); the largest
 * graph of each group is tuned with wtri_autotune and its setting applied
 * to every graph of the group.  In a batched call each query takes its
 * own graph's t_short (the short/long scan boundary), so one batch mixes
 * the boundaries of all its groups; the rounds are the batch's own.
 * *buckets_tuned (may be NULL) receives the number of groups.
 */
WTRI_API int wtri_autotune_buckets(wtri_graph* const* gs, int32_t ngraphs, int32_t k, int32_t reps,
                                   int32_t* buckets_tuned);
WTRI_API int wtri_set_tune(wtri_graph* g, int64_t first_round, int32_t growth, int32_t t_short);

/*
 * Weighted edge sampling (Algorithm 3, Section 4.1): draws nsamples edges
 * with probability w_e^p / Z (Proposition 4.1), adds every triangle on each
 * sampled edge (the common neighbours N(a) ∩ N(b)) to a set, and returns the
 * top-k of that set in the same order and format as wtri_topk.  The edge
 * draw is an integer inverse CDF over the weight-sorted edge order
 * (Section 4.1's weight classes are contiguous in that order) driven by
 * Philox4x64-10 (Salmon et al., SC'11) with key = seed and counter = the
 * sample index, so a seed gives the same samples on any device.
 *
 * p in {0, 1, 2}: w^p is an exact integer (p = 0 draws every edge with the
 * same probability); +-inf -> WTRI_EUNSUPPORTED (w^p has no meaning there),
 * and so does any other p (no exact integer cumulative mass).
 * nsamples >= 0 (0 returns count 0).
 */
WTRI_API int wtri_sample_topk(const wtri_graph* g, double p, int32_t k, int64_t nsamples,
                              uint64_t seed, wtri_result* out);

/*
 * Only the draws of wtri_sample_topk (the first step of Algorithm 3): bit r
 * of mark_words (word r/32, bit r%32) is set iff the r-th edge of the edge
 * order (weight desc, input index asc) was drawn at least once.  Host
 * output of ceil(m/32) words (words_capacity at least that).  Exists so
 * that the draws can be compared bit for bit with another implementation.
 */
WTRI_API int wtri_sample_edges(const wtri_graph* g, double p, int64_t nsamples, uint64_t seed,
                               uint32_t* mark_words, int64_t words_capacity);

/*
 * Weighted wedge sampling (Algorithm 4, Eqs. 6-8, Section 4.2).  Each of
 * nsamples iterations draws a center a with probability 2 d_a D(a) / Z1
 * (D(a) = sum over N(a) of w^p), then b in N(a) with weight
 * d_a w_ab^p + D(a), then c in N(a) with weight w_ac^p + w_ab^p; when c is
 * not b and {b, c} is an edge, the triangle joins the set T.  Returns the
 * top-k of T in the order and format of wtri_topk.  Each iteration closes a
 * given triangle with probability 2 w_p(a,b,c) / sum_v d_v D(v): b and c
 * are drawn in order, so every unordered wedge arises twice (the paper's
 * Proposition 4.2 prints w_p / sum_v d_v D(v)).  The draws are exact
 * integer inverse CDFs (the vertices in id order, a's neighbours in the
 * edge order) driven by Philox4x64-10 (Salmon et al., SC'11) words 0, 1, 2
 * of counter (sample index, 0, 0, 0) and key (seed, 1), so a seed gives the
 * same draws on any device.
 *
 * p in {0, 1, 2}; any other p -> WTRI_EUNSUPPORTED, and so does a graph
 * with a vertex whose sum of w^p reaches 2^64.  0 <= nsamples < 2^31.
 */
WTRI_API int wtri_wedge_topk(const wtri_graph* g, double p, int32_t k, int64_t nsamples,
                             uint64_t seed, wtri_result* out);

/*
 * Only the draws of wtri_wedge_topk, to host arrays of nsamples entries:
 * center[s] = a, jb[s] and jc[s] = the positions of b and c in a's
 * neighbour list in the edge order (weight desc, input index asc), and
 * tri[3s..3s+2] = the closed triangle (ascending ids) or -1, -1, -1.
 * Exists so that the draws can be compared with another implementation.
 */
WTRI_API int wtri_sample_wedges(const wtri_graph* g, double p, int64_t nsamples, uint64_t seed,
                                int32_t* center, int32_t* jb, int32_t* jc, int32_t* tri);

/*
 * Top weighted q-cliques by edge sampling (Section 4.5: sample an edge and
 * enumerate the cliques incident on it; Appendix A: a clique weighs the
 * generalized p-mean of its edge weights, Eq. 1 over q(q-1)/2 weights).
 * q = 4 or 5.  Edges are drawn exactly as wtri_sample_edges draws them
 * (nsamples draws of Algorithm 3 at p, seed): p = 1 or 2.  nsamples < 0
 * takes every edge instead: the exact top-k q-cliques, at any p in
 * {-inf, 1, 2, +inf}.  Cliques rank by (weight desc, sorted vertex tuple
 * asc) with exact integer keys (min, sum, sum of squares, max of the edge
 * weights; p = 2 needs weights up to 2^30, else WTRI_EUNSUPPORTED).
 * Outputs (host, caller-owned): cliques[q i .. q i + q-1] ascending ids,
 * weights[i] the fp64 mean (min, sum / E, sqrt(sum of squares / E), max with
 * E = q(q-1)/2), keys[i] the key (keys may be NULL), *count = min(k, number
 * of cliques found).  k in [1, 65536].  WTRI_EUNSUPPORTED if a drawn edge
 * has more than 1024 common neighbours; WTRI_ENOMEM past 2^23 cliques on
 * the drawn edges.  No counterpart for the exact mode in the paper (its
 * baseline enumerates cliques on the CPU).
 */
WTRI_API int wtri_sample_cliques(const wtri_graph* g, int32_t q, double p, int32_t k, int64_t nsamples,
                                 uint64_t seed, int32_t* cliques, double* weights, uint64_t* keys,
                                 int32_t* count);

/*
 * Copies one internal array of a built graph to host memory, for tests that
 * compare the device structures with an independent construction.
 * which: one of the WTRI_ARR_* values.  dst must hold bytes_capacity bytes;
 * *bytes_out receives the array's size (also when dst is NULL, which only
 * queries the size).
 */
enum {
    WTRI_ARR_DEGREE = 0,      /* int32[n]     degree d_a */
    WTRI_ARR_ROWPTR = 1,      /* int64[n+1]   row offsets of the weight-sorted rows */
    WTRI_ARR_ORDER_U = 2,     /* int32[m]     edge order: endpoint u of the r-th edge */
    WTRI_ARR_ORDER_V = 3,     /* int32[m]     edge order: endpoint v */
    WTRI_ARR_ORDER_W = 4,     /* int32[m]     edge order: weight (non-increasing) */
    WTRI_ARR_WCOL = 5,        /* int32[2m]    weight-sorted rows: neighbour */
    WTRI_ARR_WWT = 6,         /* int32[2m]    weight-sorted rows: weight */
    WTRI_ARR_WRANK = 7,       /* int32[2m]    weight-sorted rows: edge rank r */
    /* 8..10: unused (no symmetric id-sorted rows are kept: every lookup
       searches the one oriented row that can hold the edge) */
    WTRI_ARR_OROWPTR = 11,    /* int64[n+1]   oriented row offsets */
    WTRI_ARR_OCOL = 12,       /* int32[m]     oriented rows: higher-ranked endpoint */
    WTRI_ARR_OWT = 13,        /* int32[m]     oriented rows: weight */
    WTRI_ARR_ORANK = 14       /* int32[m]     oriented rows: edge rank r */
};
WTRI_API int wtri_graph_copy_array(const wtri_graph* g, int which, void* dst,
                                   int64_t bytes_capacity, int64_t* bytes_out);

/*
 * Profiling (no counterpart in the paper; used to attribute device time).
 * wtri_launch_count: kernels launched by this library since load (always on).
 * wtri_prof_enable(1): every library phase is bracketed by CUDA events on its
 * stream; wtri_prof_read(i, ...) returns phase i (sorted by name) with its
 * number of calls, summed device milliseconds and summed algorithmic bytes,
 * WTRI_ENOTFOUND past the last phase.  wtri_prof_reset clears the totals.
 *
 * Algorithmic bytes: the COO input read once (12 per edge); each resident
 * output written once (the oriented rows 12 per edge, each row-offset
 * array 8 per vertex); each
 * sort one read and one write of its payload (the edge order 8 + 8 per
 * edge, the weight-sorted rows 24 + 24 per edge) whatever its number of
 * passes, spread evenly over the passes; histogram, scan and other helper
 * kernels none.  wtri_prof_read_ex also returns the bytes each phase moves
 * by design (`moved`: every pass of a sort reads and writes its records),
 * so moved / bytes shows what the design spends beyond the algorithmic
 * bytes.  Query phases count bytes only while wtri_query_bytes is on.
 */
WTRI_API void wtri_prof_enable(int on);
WTRI_API void wtri_prof_reset(void);
WTRI_API long long wtri_launch_count(void);
WTRI_API int wtri_prof_read(int idx, char* name, int name_cap, long long* calls, double* ms,
                            double* bytes);
WTRI_API int wtri_prof_read_ex(int idx, char* name, int name_cap, long long* calls, double* ms,
                               double* bytes, double* moved);

/*
 * Instrumented query (no counterpart in the paper): while on != 0, the
 * exact top-k kernels (single and device queries) count the bytes of every
 * global load they issue on the graph's adjacency structures (edge order,
 * weight-sorted and oriented rows, offsets, degrees) into a
 * counter of the current device.  The counting costs time: time queries
 * with it off.  *bytes receives the counter after the device is idle
 * (cudaDeviceSynchronize); reset != 0 zeroes it afterwards.  bytes may be
 * NULL (only set or reset).
 */
WTRI_API int wtri_query_bytes(int on, int reset, unsigned long long* bytes);

/*
 * Fault injection for tests (no counterpart in the paper).  The long-scan
 * kernel of the exact query stages a vertex's neighbour list in shared
 * memory with a bulk copy and waits for it with a bounded number of polls
 * of an mbarrier; when the polls run out the query reports WTRI_ETIMEOUT
 * (the copy in flight is still waited for, with the full bound, before the
 * block moves on).  This sets the bound of that first wait for queries
 * started afterwards in this process: polls = 0 makes every staged wait
 * report a timeout at once; polls < 0 restores the default.  Nothing else
 * changes; a query after restoring the default is unaffected.
 */
WTRI_API int wtri_debug_set_wait_limit(int64_t polls);

/* Thread-local message for the last failing call on this thread ("" if none). */
WTRI_API const char* wtri_last_error(void);

/* Library version string. */
WTRI_API const char* wtri_version(void);

#ifdef __cplusplus
}
#endif

#endif /* WTRI_H */
