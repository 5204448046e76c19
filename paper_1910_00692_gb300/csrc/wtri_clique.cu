// Top weighted 4- and 5-cliques by edge sampling (Section 4.5, Appendix A).
//
// A q-clique weighs the p-mean of its q(q-1)/2 edge weights (Appendix A).
// Its key, exact and monotone in that mean, is the minimum, sum, sum of
// squares or maximum of the edge weights (p = -inf, 1, 2, +inf).  Edge
// sampling draws edges with probability proportional to w^p (Algorithm 3:
// the draws of wtri_sample_edges) and enumerates every q-clique on a drawn
// edge (Section 4.5); with every edge taken instead of draws the answer is
// the exact top-k.
//
// Per drawn edge {u, v} (one block): the common neighbours c of u and v,
// with the weights and edge ranks of {u, c} and {v, c}, go to shared memory
// (the shorter weight-sorted row is scanned, the other endpoint looked up
// in the oriented rows).  q = 4: each pair of common neighbours joined by an
// edge closes a 4-clique.  q = 5: the adjacency among the common neighbours
// becomes a bit matrix in shared memory; an adjacent pair (i, j) and each
// l above j adjacent to both close a 5-clique.  A clique is reported by its
// first drawn edge in the edge order (no other of its edges is drawn and
// earlier), so the candidates hold each clique once.  One block then keeps
// exactly the k best under (key desc, sorted vertex tuple asc) by an
// MSB-first radix select over the tuple, and a rank pass orders them.
#include "wtri_query.cuh"

#include <algorithm>

namespace wtri {
namespace {

constexpr int CB = 256;              // threads of a clique block
constexpr int CNB = 1024;            // most common neighbours of one drawn edge
constexpr int CNW = CNB / 32;        // words of a row of the q = 5 bit matrix
constexpr int QMAX = 5;
constexpr int CSB = 1024;            // threads of the select block
constexpr uint32_t CERR_CAND = 1u;   // the candidate buffer filled up
constexpr uint32_t CERR_NBR = 2u;    // a common neighbourhood above CNB
constexpr uint32_t CLIQUE_CAP = 1u << 23;

struct CliqueRun {
    const uint32_t* mark;  // drawn edges: bit r = the r-th edge of the edge order
    int32_t words;
    int32_t q, pcode;
    unsigned long long* ckey;
    int32_t* cids;         // QMAX ids per candidate, ascending
    uint32_t* count;
    uint32_t cap;
    uint32_t* err;
    int32_t* cursor;       // next bitmap word
};

// Shared memory of a clique block; the q = 5 bit matrix (CNB rows of CNW
// words, upper triangle) follows it.
struct CliqueSmem {
    int32_t cid[CNB], cdg[CNB], cwu[CNB], cwv[CNB], cru[CNB], crv[CNB];
    int32_t n;
    int32_t word;
};

__device__ __forceinline__ bool drawn(const uint32_t* mark, int32_t r) {
    return (__ldg(mark + (r >> 5)) >> (r & 31)) & 1u;
}

__device__ __forceinline__ unsigned long long clique_key(int pcode, const uint32_t* w, int ne) {
    unsigned long long acc = pcode == P_MIN ? ~0ull : 0ull;
    for (int e = 0; e < ne; e++) {
        const unsigned long long x = w[e];
        if (pcode == P_MIN) acc = x < acc ? x : acc;
        else if (pcode == P_ONE) acc += x;
        else if (pcode == P_TWO) acc += x * x;
        else acc = x > acc ? x : acc;
    }
    return acc;
}

// Appends the clique (ids[0..q), edge weights w[0..ne), ranks rk[0..ne),
// rk[0] = r the drawn edge) unless another edge of it is drawn and earlier.
__device__ void emit(const CliqueRun& C, int32_t r, int32_t* ids, const uint32_t* w, const int32_t* rk,
                     int ne) {
    for (int e = 1; e < ne; e++)
        if (rk[e] < r && drawn(C.mark, rk[e])) return;
    const unsigned long long key = clique_key(C.pcode, w, ne);
    for (int a = 1; a < C.q; a++)
        for (int b = a; b > 0 && ids[b - 1] > ids[b]; b--) {
            const int32_t t = ids[b];
            ids[b] = ids[b - 1];
            ids[b - 1] = t;
        }
    const uint32_t idx = atomicAdd(C.count, 1u);
    if (idx >= C.cap) {
        atomicOr(C.err, CERR_CAND);
        return;
    }
    C.ckey[idx] = key;
    for (int a = 0; a < QMAX; a++) C.cids[(size_t)idx * QMAX + a] = a < C.q ? ids[a] : 0;
}

__device__ void clique_edge(const DevGraph& G, const CliqueRun& C, CliqueSmem& S, uint32_t* bits, int32_t r,
                            Tally& tb) {
    const int32_t u = __ldg(G.ord_u + r), v = __ldg(G.ord_v + r);
    const uint32_t wuv = (uint32_t)__ldg(G.ord_w + r);
    const int64_t bu = __ldg(G.rowptr + u), eu = __ldg(G.rowptr + u + 1);
    const int64_t bv = __ldg(G.rowptr + v), ev = __ldg(G.rowptr + v + 1);
    const bool xu = (eu - bu) <= (ev - bv);  // scan the shorter row
    const int32_t y = xu ? v : u;
    const int64_t bx = xu ? bu : bv, ex = xu ? eu : ev;
    const int64_t dy = xu ? ev - bv : eu - bu;
    if (threadIdx.x == 0) S.n = 0;
    __syncthreads();
    for (int64_t j = bx + threadIdx.x; j < ex; j += CB) {
        const int32_t c = __ldg(G.wcol + j);
        if (c == y) continue;
        int32_t wyc, ryc;
        if (!probe_oriented(G, y, dy, c, wyc, ryc, tb)) continue;
        const int idx = atomicAdd(&S.n, 1);
        if (idx >= CNB) {
            atomicOr(C.err, CERR_NBR);
            continue;
        }
        const int32_t wxc = __ldg(G.wwt + j), rxc = __ldg(G.wrk + j);
        S.cid[idx] = c;
        S.cdg[idx] = (int32_t)(__ldg(G.rowptr + c + 1) - __ldg(G.rowptr + c));
        S.cwu[idx] = xu ? wxc : wyc;
        S.cwv[idx] = xu ? wyc : wxc;
        S.cru[idx] = xu ? rxc : ryc;
        S.crv[idx] = xu ? ryc : rxc;
    }
    __syncthreads();
    const int nc = S.n;
    if (nc > CNB) {  // recorded as an error; the call fails
        __syncthreads();
        return;
    }
    if (C.q == 4) {
        for (int i = 0; i < nc; i++)
            for (int j = i + 1 + threadIdx.x; j < nc; j += CB) {
                int32_t wij, rij;
                if (!probe_oriented(G, S.cid[i], S.cdg[i], S.cid[j], wij, rij, tb)) continue;
                int32_t ids[QMAX] = {u, v, S.cid[i], S.cid[j], 0};
                const uint32_t w[6] = {wuv, (uint32_t)S.cwu[i], (uint32_t)S.cwv[i],
                                       (uint32_t)S.cwu[j], (uint32_t)S.cwv[j], (uint32_t)wij};
                const int32_t rk[6] = {r, S.cru[i], S.crv[i], S.cru[j], S.crv[j], rij};
                emit(C, r, ids, w, rk, 6);
            }
    } else {
        const int nw = (nc + 31) >> 5;
        for (int t = threadIdx.x; t < nc * nw; t += CB) bits[(t / nw) * CNW + t % nw] = 0u;
        __syncthreads();
        for (int i = 0; i < nc; i++)
            for (int j = i + 1 + threadIdx.x; j < nc; j += CB) {
                int32_t wij, rij;
                if (probe_oriented(G, S.cid[i], S.cdg[i], S.cid[j], wij, rij, tb))
                    atomicOr(&bits[i * CNW + (j >> 5)], 1u << (j & 31));
            }
        __syncthreads();
        for (int i = 0; i < nc; i++)
            for (int j = i + 1 + threadIdx.x; j < nc; j += CB) {
                if (!((bits[i * CNW + (j >> 5)] >> (j & 31)) & 1u)) continue;
                int32_t wij = 0, rij = 0;
                probe_oriented(G, S.cid[i], S.cdg[i], S.cid[j], wij, rij, tb);
                for (int wd = (j + 1) >> 5; wd < nw; wd++) {
                    uint32_t both = bits[i * CNW + wd] & bits[j * CNW + wd];
                    if (wd == ((j + 1) >> 5)) both &= ~0u << ((j + 1) & 31);  // l > j
                    while (both) {
                        const int l = wd * 32 + __ffs(both) - 1;
                        both &= both - 1;
                        int32_t wil = 0, ril = 0, wjl = 0, rjl = 0;
                        probe_oriented(G, S.cid[i], S.cdg[i], S.cid[l], wil, ril, tb);
                        probe_oriented(G, S.cid[j], S.cdg[j], S.cid[l], wjl, rjl, tb);
                        int32_t ids[QMAX] = {u, v, S.cid[i], S.cid[j], S.cid[l]};
                        const uint32_t w[10] = {wuv,
                                                (uint32_t)S.cwu[i], (uint32_t)S.cwv[i],
                                                (uint32_t)S.cwu[j], (uint32_t)S.cwv[j],
                                                (uint32_t)S.cwu[l], (uint32_t)S.cwv[l],
                                                (uint32_t)wij, (uint32_t)wil, (uint32_t)wjl};
                        const int32_t rk[10] = {r, S.cru[i], S.crv[i], S.cru[j], S.crv[j],
                                                S.cru[l], S.crv[l], rij, ril, rjl};
                        emit(C, r, ids, w, rk, 10);
                    }
                }
            }
    }
    __syncthreads();  // the shared lists are reused by the next edge
}

// Blocks take words of the drawn-edge bitmap and handle their edges in turn.
__global__ void __launch_bounds__(CB) k_cliques(DevGraph G, CliqueRun C) {
    extern __shared__ __align__(16) unsigned char csm[];
    CliqueSmem& S = *reinterpret_cast<CliqueSmem*>(csm);
    uint32_t* bits = reinterpret_cast<uint32_t*>(csm + sizeof(CliqueSmem));
    Tally tb;
    for (;;) {
        if (threadIdx.x == 0) S.word = atomicAdd(C.cursor, 1);
        __syncthreads();
        const int32_t wi = S.word;
        __syncthreads();
        if (wi >= C.words) break;
        uint32_t mw = __ldg(C.mark + wi);
        while (mw) {
            const int32_t r = wi * 32 + __ffs(mw) - 1;
            mw &= mw - 1;
            clique_edge(G, C, S, bits, r, tb);
        }
    }
}

// Every edge drawn: all bits of the first m positions.
__global__ void k_mark_all(int64_t m, uint32_t* mark) {
    const int64_t words = (m + 31) / 32;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t left = m - 32 * i;
        mark[i] = left >= 32 ? ~0u : ((1u << left) - 1u);
    }
}

// ---- selection of the k best candidates ------------------------------------
// Tuple of a candidate, smaller is better: (~key_hi, ~key_lo, id_0 .. id_{q-1}).
__device__ __forceinline__ uint32_t cword(const unsigned long long* ckey, const int32_t* cids, uint32_t i,
                                          int wi) {
    if (wi == 0) return ~(uint32_t)(ckey[i] >> 32);
    if (wi == 1) return ~(uint32_t)ckey[i];
    return (uint32_t)cids[(size_t)i * QMAX + (wi - 2)];
}

struct CSelSmem {
    uint32_t hist[256];
    uint32_t pw[2 + QMAX];
    uint32_t below, eq, done, kept;
    uint32_t warp_cnt[CSB / 32];
};

// <0, 0, >0: the first `depth` bytes of candidate i's tuple against pw.
__device__ __forceinline__ int cmp_cprefix(const unsigned long long* ckey, const int32_t* cids, uint32_t i,
                                           const uint32_t* pw, int depth) {
    const int full = depth >> 2, rem = depth & 3;
    for (int wi = 0; wi < full; wi++) {
        const uint32_t a = cword(ckey, cids, i, wi);
        if (a != pw[wi]) return a < pw[wi] ? -1 : 1;
    }
    if (rem) {
        const uint32_t mask = 0xffffffffu << (32 - 8 * rem);
        const uint32_t a = cword(ckey, cids, i, full) & mask, b = pw[full] & mask;
        if (a != b) return a < b ? -1 : 1;
    }
    return 0;
}

// Keeps exactly min(K, n) best candidates at the front (tuples are unique:
// every clique appears once), n = *count; *kept receives their number.
__global__ void __launch_bounds__(CSB) k_clique_select(unsigned long long* ckey, int32_t* cids,
                                                       const uint32_t* count, uint32_t cap, int q, uint32_t K,
                                                       const uint32_t* err, uint32_t* kept) {
    __shared__ CSelSmem S;
    if (*(volatile const uint32_t*)err) return;
    const uint32_t n = min(*(volatile const uint32_t*)count, cap);
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int nbytes = 4 * (2 + q);
    if (tid < 2 + QMAX) S.pw[tid] = 0;
    if (tid == 0) {
        S.below = 0;
        S.eq = n;
        S.done = n <= K ? 1u : 0u;
    }
    __syncthreads();
    int depth = 0;
    while (!S.done && depth < nbytes) {
        for (int i = tid; i < 256; i += CSB) S.hist[i] = 0;
        __syncthreads();
        const int wi = depth >> 2, sh = 24 - 8 * (depth & 3);
        for (uint32_t i = tid; i < n; i += CSB)
            if (cmp_cprefix(ckey, cids, i, S.pw, depth) == 0)
                atomicAdd(&S.hist[(cword(ckey, cids, i, wi) >> sh) & 255u], 1u);
        __syncthreads();
        if (tid == 0) {
            const uint32_t need = K - S.below;
            uint32_t acc = 0, dsel = 0;
            for (uint32_t d = 0; d < 256; d++) {
                if (acc + S.hist[d] >= need) {
                    dsel = d;
                    break;
                }
                acc += S.hist[d];
            }
            S.below += acc;
            S.eq = S.hist[dsel];
            S.pw[wi] |= dsel << sh;
            if (S.below + S.eq == K) S.done = 1;
        }
        __syncthreads();
        depth++;
    }
    const bool keep_all = n <= K;
    uint32_t out = 0;
    for (uint32_t base = 0; base < n; base += CSB) {
        const uint32_t i = base + tid;
        bool keep = false;
        unsigned long long kk = 0;
        int32_t t[QMAX] = {0, 0, 0, 0, 0};
        if (i < n) {
            keep = keep_all || cmp_cprefix(ckey, cids, i, S.pw, depth) <= 0;
            kk = ckey[i];
            for (int a = 0; a < QMAX; a++) t[a] = cids[(size_t)i * QMAX + a];
        }
        const uint32_t b = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) S.warp_cnt[wid] = __popc(b);
        __syncthreads();
        if (tid == 0) {
            uint32_t acc = 0;
            for (int wv = 0; wv < CSB / 32; wv++) {
                const uint32_t c = S.warp_cnt[wv];
                S.warp_cnt[wv] = acc;
                acc += c;
            }
            S.kept = acc;
        }
        __syncthreads();
        if (keep) {
            const uint32_t p = out + S.warp_cnt[wid] + __popc(b & ((1u << lane) - 1u));
            ckey[p] = kk;  // p <= i: this chunk was read before the barrier
            for (int a = 0; a < QMAX; a++) cids[(size_t)p * QMAX + a] = t[a];
        }
        out += S.kept;
        __syncthreads();
    }
    if (tid == 0) *kept = out;
}

// Whether candidate a ranks before candidate b.
__device__ __forceinline__ bool cbefore(const unsigned long long* ckey, const int32_t* cids, uint32_t a,
                                        uint32_t b, int q) {
    if (ckey[a] != ckey[b]) return ckey[a] > ckey[b];
    for (int i = 0; i < q; i++) {
        const int32_t x = cids[(size_t)a * QMAX + i], y = cids[(size_t)b * QMAX + i];
        if (x != y) return x < y;
    }
    return false;
}

// One warp per kept candidate: its rank among the kept ones, then the
// outputs at that rank (ids, fp64 mean, key).
__global__ void k_clique_rank(const unsigned long long* ckey, const int32_t* cids, const uint32_t* kept,
                              const uint32_t* err, int q, int pcode, uint32_t kmax, int32_t* ids_out,
                              double* w_out, unsigned long long* key_out) {
    if (*(volatile const uint32_t*)err) return;
    const uint32_t K = *kept;
    const uint32_t i = (uint32_t)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= K) return;
    uint32_t rank = 0;
    for (uint32_t j = lane; j < K; j += 32) rank += cbefore(ckey, cids, j, i, q) ? 1u : 0u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rank += __shfl_xor_sync(0xffffffffu, rank, o);
    if (lane == 0 && rank < kmax) {
        const unsigned long long key = ckey[i];
        const double ne = (double)(q * (q - 1) / 2);
        for (int a = 0; a < q; a++) ids_out[(size_t)rank * q + a] = cids[(size_t)i * QMAX + a];
        w_out[rank] = pcode == P_ONE ? (double)key / ne : (pcode == P_TWO ? sqrt((double)key / ne) : (double)key);
        key_out[rank] = key;
    }
}

}  // namespace

int clique_topk_host(const wtri_graph* g, int q, int pcode, int32_t k, int64_t nsamples, uint64_t seed,
                     int32_t* h_ids, double* h_w, uint64_t* h_keys, int32_t* h_count) {
    const DevGraph& G = g->d;
    const int64_t m = G.m;
    const int64_t words = (m + 31) / 32;
    const uint32_t cap = CLIQUE_CAP;
    cudaStream_t s = g->stream;
    const size_t bytes = 4 * (size_t)words + 256 + (size_t)cap * 8 + (size_t)cap * 4 * QMAX + 256 +
                         (size_t)k * (4 * q + 16) + 256 + 64;
    void* buf = nullptr;
    if (cudaMallocAsync(&buf, bytes, s) != cudaSuccess) {
        cudaGetLastError();
        return set_error(WTRI_ENOMEM, "clique scratch allocation failed");
    }
    char* p = (char*)buf;
    uint32_t* mark = (uint32_t*)p;
    p += (4 * (size_t)words + 255) & ~(size_t)255;
    unsigned long long* ckey = (unsigned long long*)p;
    p += (size_t)cap * 8;
    int32_t* cids = (int32_t*)p;
    p += ((size_t)cap * 4 * QMAX + 255) & ~(size_t)255;
    unsigned long long* okey = (unsigned long long*)p;
    double* ow = (double*)(okey + k);
    int32_t* oids = (int32_t*)(ow + k);
    p += ((size_t)k * (4 * q + 16) + 255) & ~(size_t)255;
    uint32_t* small = (uint32_t*)p;  // count, err, cursor, kept
    auto done = [&](int rc) {
        cudaFreeAsync(buf, s);
        cudaStreamSynchronize(s);
        return rc;
    };
    if (cudaMemsetAsync(small, 0, 64, s) != cudaSuccess)
        return done(cuda_error(cudaGetLastError(), "memset", __FILE__, __LINE__));
    if (nsamples >= 0) {
        int rc = sample_edges_device(g, pcode, nsamples, seed, mark, s);
        if (rc != WTRI_OK) return done(rc);
    } else {
        k_mark_all<<<std::max<int64_t>(1, std::min<int64_t>((words + 255) / 256, sm_count() * 8)), 256, 0, s>>>(
            m, mark);
    }
    CliqueRun C;
    C.mark = mark;
    C.words = (int32_t)words;
    C.q = q;
    C.pcode = pcode;
    C.ckey = ckey;
    C.cids = cids;
    C.count = small;
    C.cap = cap;
    C.err = small + 1;
    C.cursor = (int32_t*)(small + 2);
    const int smem = (int)sizeof(CliqueSmem) + (q == 5 ? CNB * CNW * 4 : 0);
    static std::atomic<uint64_t> optin{0};
    {
        int rc = smem_optin((const void*)k_cliques, (int)sizeof(CliqueSmem) + CNB * CNW * 4, optin);
        if (rc != WTRI_OK) return done(rc);
    }
    {
        ProfScope ps("cliques_enumerate", s, 0.0, 1);
        k_cliques<<<sm_count() * (q == 5 ? 1 : 4), CB, smem, s>>>(G, C);
    }
    {
        ProfScope ps("cliques_select", s, 0.0, 2);
        k_clique_select<<<1, CSB, 0, s>>>(ckey, cids, small, cap, q, (uint32_t)k, small + 1, small + 3);
        k_clique_rank<<<ceil_div_u(k, 8), 256, 0, s>>>(ckey, cids, small + 3, small + 1, q, pcode,
                                                        (uint32_t)k, oids, ow, okey);
    }
    if (cudaGetLastError() != cudaSuccess)
        return done(set_error(WTRI_ECUDA, "clique kernel launch failed"));
    uint32_t hs[4] = {0, 0, 0, 0};
    cudaError_t e = cudaMemcpyAsync(hs, small, sizeof(hs), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return done(cuda_error(e, "clique results", __FILE__, __LINE__));
    if (hs[1] & CERR_NBR)
        return done(set_error(WTRI_EUNSUPPORTED, "a drawn edge has more than " + std::to_string(CNB) +
                                                     " common neighbours"));
    if (hs[1] & CERR_CAND)
        return done(set_error(WTRI_ENOMEM, "more than " + std::to_string(cap) + " cliques on the drawn edges"));
    const uint32_t kept = std::min(hs[3], (uint32_t)k);
    e = cudaMemcpyAsync(h_ids, oids, 4 * (size_t)kept * q, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_w, ow, 8 * (size_t)kept, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && h_keys) e = cudaMemcpyAsync(h_keys, okey, 8 * (size_t)kept, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return done(cuda_error(e, "clique results", __FILE__, __LINE__));
    *h_count = (int32_t)kept;
    return done(WTRI_OK);
}

}  // namespace wtri
