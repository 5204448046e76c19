/*
 * CPU oracle for exact top-k weighted triangles.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file; only the test suite, the smoke check and the bench's CPU
 * baseline leg use it.  It shares no code, header or constant with the CUDA
 * library.
 *
 * What it computes (Kumar, Liu, Charikar, Benson, "Retrieving Top Weighted
 * Triangles in Graphs", WSDM 2020):
 *
 *  - the triangle weight is the generalized p-mean of its three edge weights
 *    (Eq. 1, Section 1), for p in {-inf, 0, 1, 2, +inf}: min, geometric mean
 *    (Eq. 1's limit as p -> 0), arithmetic mean, quadratic mean, max;
 *  - the top-k triangles are the k of largest weight (Section 1); ties are
 *    broken by the sorted vertex triple ascending, which makes the answer
 *    unique (the paper notes ties may exist, Section 3.2);
 *  - enumeration is the paper's brute-force baseline (Section 3, Section 5.2):
 *    NodeIterator++ over a degree ordering, keeping a heap of the k heaviest.
 *
 * For p in {-inf, 0, 1, 2, +inf} ranking never uses the floating value.
 * Each triangle gets an exact integer key that is monotone in m_p: a+b+c
 * (p=1), a^2+b^2+c^2 (p=2), max (p=+inf), min (p=-inf), a*b*c (p=0; exact
 * for weights below 2^21).  Eq. 4 (Section 4) ranks by the sum of p-th
 * powers, which is only order-preserving for p>0; these keys are the
 * order-preserving choice for every supported p.  The reported value is
 * fp64: (a+b+c)/3, sqrt((a^2+b^2+c^2)/3), max, min, cbrt(a*b*c).
 *
 * Any other finite p (code 5: the harmonic mean p = -1, p = -2, p = 3, ...)
 * has no exact 64-bit integer key; there the key is m_p itself in fp64
 * (its bit pattern, which orders positive doubles like their values),
 * computed from Eq. 1 with the largest weight factored out for p > 0 (the
 * smallest for p < 0) so that no power overflows:
 *     m_p = s * ((( a/s)^p + (b/s)^p + (c/s)^p) / 3)^(1/p).
 * Two triangles whose means differ by less than fp64 rounding may then rank
 * either way; the tests allow exactly that and nothing more.
 *
 * Input hygiene (Section 1: "simple, undirected graph with positive edge
 * weights"): self-loops, ids outside [0,n), weights <= 0 and repeated
 * undirected pairs are rejected, never silently repaired.
 *
 * Parity pins live in tests/: closed forms on complete graphs, an independent
 * triangle count (trace(A^3)/6), hand-enumerated graphs under tests/golden/,
 * and a Python itertools brute force on small random graphs.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_EINVAL -1
#define OR_ENOMEM -2

/* p codes: 0 -> -inf, 1 -> 1, 2 -> 2, 3 -> +inf, 4 -> 0, 5 -> any other
 * finite p (passed beside the code as a double) */
#define OR_PCODE_MAX 5

/* ------------------------------------------------------------------------ */
/* Validation and the symmetric adjacency (N(a), d_a of Section 4).          */
/* ------------------------------------------------------------------------ */

typedef struct {
    int32_t c;
    int32_t w;
    int64_t eid;
} or_ent;

static int cmp_ent_by_col(const void* a, const void* b) {
    const or_ent* x = (const or_ent*)a;
    const or_ent* y = (const or_ent*)b;
    return (x->c > y->c) - (x->c < y->c);
}

/* Checks the edge list.  Returns OR_OK or OR_EINVAL.  err_edge receives the
 * first offending edge index (or -1). */
int or_validate(int32_t n, int64_t m, const int32_t* u, const int32_t* v,
                const int32_t* w, int64_t* err_edge) {
    *err_edge = -1;
    if (n <= 0 || m < 0) return OR_EINVAL;
    for (int64_t i = 0; i < m; i++) {
        if (u[i] < 0 || u[i] >= n || v[i] < 0 || v[i] >= n || u[i] == v[i] || w[i] <= 0) {
            *err_edge = i;
            return OR_EINVAL;
        }
    }
    return OR_OK;
}

/* Symmetric CSR with each row ascending by neighbour id.  rowptr has n+1
 * entries; col, wt, eid have 2m.  Returns OR_EINVAL on invalid input,
 * including a repeated undirected pair (found as equal neighbours in a
 * sorted row). */
int or_sym_csr(int32_t n, int64_t m, const int32_t* u, const int32_t* v,
               const int32_t* w, int64_t* rowptr, int32_t* col, int32_t* wt,
               int64_t* eid) {
    int64_t bad;
    if (or_validate(n, m, u, v, w, &bad) != OR_OK) return OR_EINVAL;
    int64_t* fill = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    or_ent* ent = (or_ent*)malloc(sizeof(or_ent) * (size_t)(2 * m + 1));
    if (!fill || !ent) {
        free(fill);
        free(ent);
        return OR_ENOMEM;
    }
    memset(rowptr, 0, sizeof(int64_t) * ((size_t)n + 1));
    for (int64_t i = 0; i < m; i++) {
        rowptr[u[i] + 1]++;
        rowptr[v[i] + 1]++;
    }
    for (int32_t a = 0; a < n; a++) rowptr[a + 1] += rowptr[a];
    for (int64_t i = 0; i < m; i++) {
        int64_t pu = rowptr[u[i]] + fill[u[i]]++;
        ent[pu].c = v[i];
        ent[pu].w = w[i];
        ent[pu].eid = i;
        int64_t pv = rowptr[v[i]] + fill[v[i]]++;
        ent[pv].c = u[i];
        ent[pv].w = w[i];
        ent[pv].eid = i;
    }
    int rc = OR_OK;
    for (int32_t a = 0; a < n; a++) {
        int64_t s = rowptr[a], e = rowptr[a + 1];
        qsort(ent + s, (size_t)(e - s), sizeof(or_ent), cmp_ent_by_col);
        for (int64_t j = s + 1; j < e; j++)
            if (ent[j].c == ent[j - 1].c) rc = OR_EINVAL;
    }
    for (int64_t j = 0; j < 2 * m; j++) {
        col[j] = ent[j].c;
        wt[j] = ent[j].w;
        eid[j] = ent[j].eid;
    }
    free(fill);
    free(ent);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Edge order: E sorted in decreasing order of weight (Algorithm 2, first   */
/* step), ties by ascending edge index so that the order is total.          */
/* ------------------------------------------------------------------------ */

static const int32_t* g_sort_w;

static int cmp_eid_by_weight(const void* a, const void* b) {
    int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
    int32_t wx = g_sort_w[x], wy = g_sort_w[y];
    if (wx != wy) return wx > wy ? -1 : 1;
    return (x > y) - (x < y);
}

/* perm[r] = edge index of the r-th edge in the order. */
int or_edge_order(int64_t m, const int32_t* w, int64_t* perm) {
    for (int64_t i = 0; i < m; i++) perm[i] = i;
    g_sort_w = w;
    qsort(perm, (size_t)m, sizeof(int64_t), cmp_eid_by_weight);
    g_sort_w = NULL;
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Degree orientation used by NodeIterator++ (Section 5.2): vertices ranked */
/* by (degree, id); each edge is kept once, from its lower-ranked endpoint  */
/* to its higher-ranked one.  Rows ascending by id.                         */
/* ------------------------------------------------------------------------ */

static int rank_less(const int64_t* deg, int32_t a, int32_t b) {
    if (deg[a] != deg[b]) return deg[a] < deg[b];
    return a < b;
}

int or_oriented_csr(int32_t n, int64_t m, const int32_t* u, const int32_t* v,
                    const int32_t* w, int64_t* orowptr, int32_t* ocol, int32_t* owt,
                    int64_t* oeid) {
    int64_t bad;
    if (or_validate(n, m, u, v, w, &bad) != OR_OK) return OR_EINVAL;
    int64_t* deg = (int64_t*)calloc((size_t)n, sizeof(int64_t));
    int64_t* fill = (int64_t*)calloc((size_t)n, sizeof(int64_t));
    or_ent* ent = (or_ent*)malloc(sizeof(or_ent) * (size_t)(m + 1));
    if (!deg || !fill || !ent) {
        free(deg);
        free(fill);
        free(ent);
        return OR_ENOMEM;
    }
    for (int64_t i = 0; i < m; i++) {
        deg[u[i]]++;
        deg[v[i]]++;
    }
    memset(orowptr, 0, sizeof(int64_t) * ((size_t)n + 1));
    for (int64_t i = 0; i < m; i++) {
        int32_t lo = rank_less(deg, u[i], v[i]) ? u[i] : v[i];
        orowptr[lo + 1]++;
    }
    for (int32_t a = 0; a < n; a++) orowptr[a + 1] += orowptr[a];
    for (int64_t i = 0; i < m; i++) {
        int up = rank_less(deg, u[i], v[i]);
        int32_t lo = up ? u[i] : v[i];
        int32_t hi = up ? v[i] : u[i];
        int64_t p = orowptr[lo] + fill[lo]++;
        ent[p].c = hi;
        ent[p].w = w[i];
        ent[p].eid = i;
    }
    int rc = OR_OK;
    for (int32_t a = 0; a < n; a++) {
        int64_t s = orowptr[a], e = orowptr[a + 1];
        qsort(ent + s, (size_t)(e - s), sizeof(or_ent), cmp_ent_by_col);
        for (int64_t j = s + 1; j < e; j++)
            if (ent[j].c == ent[j - 1].c) rc = OR_EINVAL;
    }
    for (int64_t j = 0; j < m; j++) {
        ocol[j] = ent[j].c;
        owt[j] = ent[j].w;
        oeid[j] = ent[j].eid;
    }
    free(deg);
    free(fill);
    free(ent);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Scoring: exact key and fp64 value of m_p (Eq. 1).                        */
/* ------------------------------------------------------------------------ */

/* m_p of Eq. 1 for a finite p other than 0, in fp64, scaled so that no power
 * overflows: s = max(a,b,c) for p > 0, min(a,b,c) for p < 0.  The weights
 * are summed in ascending order, so equal multisets give equal bits. */
static double general_mean(double p, int32_t a, int32_t b, int32_t c) {
    int32_t t3[3] = {a, b, c}, x;
    if (t3[0] > t3[1]) { x = t3[0]; t3[0] = t3[1]; t3[1] = x; }
    if (t3[1] > t3[2]) { x = t3[1]; t3[1] = t3[2]; t3[2] = x; }
    if (t3[0] > t3[1]) { x = t3[0]; t3[0] = t3[1]; t3[1] = x; }
    const double s = p > 0 ? (double)t3[2] : (double)t3[0];
    const double t = (pow((double)t3[0] / s, p) + pow((double)t3[1] / s, p) +
                      pow((double)t3[2] / s, p)) / 3.0;
    return s * pow(t, 1.0 / p);
}

static uint64_t tri_key(int pcode, double p, int32_t a, int32_t b, int32_t c) {
    switch (pcode) {
        case 0: {
            int32_t x = a < b ? a : b;
            return (uint64_t)(x < c ? x : c);
        }
        case 1:
            return (uint64_t)a + (uint64_t)b + (uint64_t)c;
        case 2:
            return (uint64_t)a * (uint64_t)a + (uint64_t)b * (uint64_t)b + (uint64_t)c * (uint64_t)c;
        case 4: /* p = 0: the geometric mean ranks as the product (weights < 2^21) */
            return (uint64_t)a * (uint64_t)b * (uint64_t)c;
        case 5: { /* the positive fp64 mean's bit pattern orders like its value */
            const double m = general_mean(p, a, b, c);
            uint64_t k;
            memcpy(&k, &m, sizeof k);
            return k;
        }
        default: {
            int32_t x = a > b ? a : b;
            return (uint64_t)(x > c ? x : c);
        }
    }
}

static double tri_value(int pcode, uint64_t key) {
    switch (pcode) {
        case 1:
            return (double)key / 3.0;
        case 2:
            return sqrt((double)key / 3.0);
        case 4:
            return cbrt((double)key);
        case 5: {
            double m;
            memcpy(&m, &key, sizeof m);
            return m;
        }
        default:
            return (double)key;
    }
}

/* Checks a (code, p) pair: code 5 needs a finite p outside {0, 1, 2}. */
static int pcode_ok(int pcode, double p) {
    if (pcode < 0 || pcode > OR_PCODE_MAX) return 0;
    if (pcode == 5) return isfinite(p) && p != 0.0 && p != 1.0 && p != 2.0;
    return 1;
}

/* Public scorer, so that tests can pin it against hand-computed means. */
int or_score(int pcode, double p, int32_t a, int32_t b, int32_t c, uint64_t* key, double* value) {
    if (!pcode_ok(pcode, p)) return OR_EINVAL;
    *key = tri_key(pcode, p, a, b, c);
    *value = tri_value(pcode, *key);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Top-k under the total order (key desc, sorted triple asc).               */
/* ------------------------------------------------------------------------ */

typedef struct {
    uint64_t key;
    int32_t t[3]; /* ascending vertex ids */
} or_tri;

/* 1 if x ranks strictly before y. */
static int tri_before(const or_tri* x, const or_tri* y) {
    if (x->key != y->key) return x->key > y->key;
    for (int i = 0; i < 3; i++)
        if (x->t[i] != y->t[i]) return x->t[i] < y->t[i];
    return 0;
}

static int cmp_tri(const void* a, const void* b) {
    const or_tri* x = (const or_tri*)a;
    const or_tri* y = (const or_tri*)b;
    if (tri_before(x, y)) return -1;
    if (tri_before(y, x)) return 1;
    return 0;
}

/* Bounded heap holding the k best triangles seen; the root is the worst. */
typedef struct {
    or_tri* h;
    int64_t size, cap;
} or_heap;

static void heap_sift_down(or_heap* hp, int64_t i) {
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, worst = i;
        if (l < hp->size && tri_before(&hp->h[worst], &hp->h[l])) worst = l;
        if (r < hp->size && tri_before(&hp->h[worst], &hp->h[r])) worst = r;
        if (worst == i) return;
        or_tri t = hp->h[i];
        hp->h[i] = hp->h[worst];
        hp->h[worst] = t;
        i = worst;
    }
}

static void heap_sift_up(or_heap* hp, int64_t i) {
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (!tri_before(&hp->h[p], &hp->h[i])) return; /* parent already worse */
        or_tri t = hp->h[i];
        hp->h[i] = hp->h[p];
        hp->h[p] = t;
        i = p;
    }
}

static void heap_offer(or_heap* hp, const or_tri* x) {
    if (hp->size < hp->cap) {
        hp->h[hp->size] = *x;
        heap_sift_up(hp, hp->size);
        hp->size++;
    } else if (tri_before(x, &hp->h[0])) {
        hp->h[0] = *x;
        heap_sift_down(hp, 0);
    }
}

static void sort3(int32_t* t) {
    int32_t x;
    if (t[0] > t[1]) { x = t[0]; t[0] = t[1]; t[1] = x; }
    if (t[1] > t[2]) { x = t[1]; t[1] = t[2]; t[2] = x; }
    if (t[0] > t[1]) { x = t[0]; t[0] = t[1]; t[1] = x; }
}

/*
 * Brute-force exact top-k (the paper's BF baseline: NodeIterator++ with a
 * heap, Sections 3 and 5.2).  Every triangle {a,b,c} is found exactly once,
 * from its lowest-ranked vertex, as the intersection of two oriented rows.
 *
 * Outputs the first min(k, #triangles) triangles in rank order: tri[3*i..],
 * key[i], value[i].  *count receives that number and *ntri the total number
 * of triangles in the graph.  nthreads <= 0 means all available threads.
 */
int or_topk(int32_t n, int64_t m, const int32_t* u, const int32_t* v, const int32_t* w,
            int pcode, double preal, int64_t k, int nthreads, int32_t* tri, uint64_t* key,
            double* value, int64_t* count, int64_t* ntri) {
    *count = 0;
    *ntri = 0;
    if (!pcode_ok(pcode, preal) || k <= 0) return OR_EINVAL;
    int64_t* orow = (int64_t*)malloc(sizeof(int64_t) * ((size_t)n + 1));
    int32_t* ocol = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m + 1));
    int32_t* owt = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m + 1));
    int64_t* oeid = (int64_t*)malloc(sizeof(int64_t) * (size_t)(m + 1));
    if (!orow || !ocol || !owt || !oeid) {
        free(orow); free(ocol); free(owt); free(oeid);
        return OR_ENOMEM;
    }
    int rc = or_oriented_csr(n, m, u, v, w, orow, ocol, owt, oeid);
    free(oeid);
    if (rc != OR_OK) {
        free(orow); free(ocol); free(owt);
        return rc;
    }
    int nt = 1;
#ifdef _OPENMP
    nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#endif
    or_heap* heaps = (or_heap*)calloc((size_t)nt, sizeof(or_heap));
    int64_t* counts = (int64_t*)calloc((size_t)nt, sizeof(int64_t));
    int alloc_fail = 0;
    for (int t = 0; t < nt; t++) {
        heaps[t].cap = k;
        heaps[t].h = (or_tri*)malloc(sizeof(or_tri) * (size_t)k);
        if (!heaps[t].h) alloc_fail = 1;
    }
    if (!alloc_fail) {
#ifdef _OPENMP
#pragma omp parallel num_threads(nt)
#endif
        {
            int tid = 0;
#ifdef _OPENMP
            tid = omp_get_thread_num();
#endif
            or_heap* hp = &heaps[tid];
            int64_t local = 0;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 64)
#endif
            for (int32_t a = 0; a < n; a++) {
                for (int64_t i = orow[a]; i < orow[a + 1]; i++) {
                    int32_t b = ocol[i];
                    int32_t wab = owt[i];
                    /* N+(a) intersect N+(b), both ascending by id. */
                    int64_t p = orow[a], pe = orow[a + 1];
                    int64_t q = orow[b], qe = orow[b + 1];
                    while (p < pe && q < qe) {
                        if (ocol[p] < ocol[q]) {
                            p++;
                        } else if (ocol[p] > ocol[q]) {
                            q++;
                        } else {
                            or_tri x;
                            x.key = tri_key(pcode, preal, wab, owt[p], owt[q]);
                            x.t[0] = a;
                            x.t[1] = b;
                            x.t[2] = ocol[p];
                            sort3(x.t);
                            heap_offer(hp, &x);
                            local++;
                            p++;
                            q++;
                        }
                    }
                }
            }
            counts[tid] = local;
        }
        int64_t total = 0, pooled = 0;
        for (int t = 0; t < nt; t++) {
            total += counts[t];
            pooled += heaps[t].size;
        }
        or_tri* all = (or_tri*)malloc(sizeof(or_tri) * (size_t)(pooled + 1));
        if (!all) {
            rc = OR_ENOMEM;
        } else {
            int64_t at = 0;
            for (int t = 0; t < nt; t++) {
                memcpy(all + at, heaps[t].h, sizeof(or_tri) * (size_t)heaps[t].size);
                at += heaps[t].size;
            }
            qsort(all, (size_t)pooled, sizeof(or_tri), cmp_tri);
            int64_t out = pooled < k ? pooled : k;
            for (int64_t i = 0; i < out; i++) {
                tri[3 * i + 0] = all[i].t[0];
                tri[3 * i + 1] = all[i].t[1];
                tri[3 * i + 2] = all[i].t[2];
                key[i] = all[i].key;
                value[i] = tri_value(pcode, all[i].key);
            }
            *count = out;
            *ntri = total;
            free(all);
        }
    } else {
        rc = OR_ENOMEM;
    }
    for (int t = 0; t < nt; t++) free(heaps[t].h);
    free(heaps);
    free(counts);
    free(orow);
    free(ocol);
    free(owt);
    return rc;
}

/* Triangle count by a different route: for every edge {a,b} with a<b, count
 * common neighbours c>b by merging the id-sorted symmetric rows.  Used to
 * cross-check the enumeration count. */
int or_count_triangles(int32_t n, int64_t m, const int32_t* u, const int32_t* v,
                       const int32_t* w, int64_t* ntri) {
    *ntri = 0;
    int64_t* rowptr = (int64_t*)malloc(sizeof(int64_t) * ((size_t)n + 1));
    int32_t* col = (int32_t*)malloc(sizeof(int32_t) * (size_t)(2 * m + 1));
    int32_t* wt = (int32_t*)malloc(sizeof(int32_t) * (size_t)(2 * m + 1));
    int64_t* eid = (int64_t*)malloc(sizeof(int64_t) * (size_t)(2 * m + 1));
    if (!rowptr || !col || !wt || !eid) {
        free(rowptr); free(col); free(wt); free(eid);
        return OR_ENOMEM;
    }
    int rc = or_sym_csr(n, m, u, v, w, rowptr, col, wt, eid);
    if (rc == OR_OK) {
        int64_t total = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : total)
#endif
        for (int32_t a = 0; a < n; a++) {
            for (int64_t i = rowptr[a]; i < rowptr[a + 1]; i++) {
                int32_t b = col[i];
                if (b <= a) continue;
                int64_t p = rowptr[a], pe = rowptr[a + 1];
                int64_t q = rowptr[b], qe = rowptr[b + 1];
                while (p < pe && q < qe) {
                    if (col[p] < col[q]) p++;
                    else if (col[p] > col[q]) q++;
                    else {
                        if (col[p] > b) total++;
                        p++;
                        q++;
                    }
                }
            }
        }
        *ntri = total;
    }
    free(rowptr);
    free(col);
    free(wt);
    free(eid);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Weighted edge sampling (Algorithm 3, Section 4.1).                       */
/* ------------------------------------------------------------------------ */

/* Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel Random Numbers: As
 * Easy as 1, 2, 3", SC'11): ten rounds of two 64x64->128 multiplies with
 * the published multipliers and Weyl key increments.  Written from that
 * description; pinned against numpy's Philox bit generator in the tests. */
void or_philox4x64_10(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4]) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
    uint64_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint64_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; r++) {
        unsigned __int128 p0 = (unsigned __int128)M0 * c0;
        unsigned __int128 p1 = (unsigned __int128)M1 * c2;
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        uint64_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0;
        k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/*
 * Draws nsamples edges with probability w_e^p / Z, Z = sum_e w_e^p (the
 * first step of Algorithm 3; Proposition 4.1), p in {1, 2}.
 *
 * Definition used on both sides: with the edges in the edge order
 * perm[0..m) (weight desc, index asc) and C[r] = sum_{j<=r} w_{perm[j]}^p
 * (exact, 128-bit), sample s takes x = word 0 of
 * Philox4x64-10(counter = (s, 0, 0, 0), key = (seed, 0)), t = floor(x * Z /
 * 2^64), and returns the first r with C[r] > t.
 *
 * hits[r] receives how many times the r-th edge of the order was drawn.
 */
int or_sample_edges(int64_t m, const int32_t* w, const int64_t* perm, int pcode, int64_t nsamples,
                    uint64_t seed, int64_t* hits) {
    if (pcode != 1 && pcode != 2 && pcode != 4) return OR_EINVAL;
    unsigned __int128* C = (unsigned __int128*)malloc(sizeof(unsigned __int128) * (size_t)(m + 1));
    if (!C) return OR_ENOMEM;
    unsigned __int128 acc = 0;
    for (int64_t r = 0; r < m; r++) {
        unsigned __int128 x = (unsigned __int128)(uint64_t)w[perm[r]];
        acc += pcode == 4 ? 1 : (pcode == 1 ? x : x * x); /* w^p, p = 0 -> 1 */
        C[r] = acc;
        hits[r] = 0;
    }
    const unsigned __int128 Z = acc;
    const uint64_t key[2] = {seed, 0};
    for (int64_t s = 0; s < nsamples && m > 0; s++) {
        uint64_t ctr[4] = {(uint64_t)s, 0, 0, 0}, out[4];
        or_philox4x64_10(ctr, key, out);
        /* t = floor(x * Z / 2^64), with Z < 2^128 split in two halves */
        const uint64_t zl = (uint64_t)Z, zh = (uint64_t)(Z >> 64);
        unsigned __int128 t = (unsigned __int128)out[0] * zh +
                              (((unsigned __int128)out[0] * zl) >> 64);
        int64_t lo = 0, hi = m;  /* first r with C[r] > t */
        while (lo < hi) {
            int64_t mid = lo + (hi - lo) / 2;
            if (C[mid] > t) hi = mid;
            else lo = mid + 1;
        }
        hits[lo]++;
    }
    free(C);
    return OR_OK;
}

/*
 * Top-k of the triangle set T of Algorithm 3: T holds every triangle that
 * has at least one sampled edge (a triangle is added when any of its edges
 * is drawn).  Enumerated by brute force over all triangles (NodeIterator++),
 * keeping those with a sampled edge; ranked like or_topk.
 * edge_sampled[i] != 0 marks input edge i.
 */
int or_topk_of_sampled(int32_t n, int64_t m, const int32_t* u, const int32_t* v, const int32_t* w,
                       const uint8_t* edge_sampled, int pcode, double preal, int64_t k,
                       int nthreads, int32_t* tri, uint64_t* key, double* value, int64_t* count,
                       int64_t* ntri) {
    *count = 0;
    *ntri = 0;
    if (!pcode_ok(pcode, preal) || k <= 0) return OR_EINVAL;
    int64_t* orow = (int64_t*)malloc(sizeof(int64_t) * ((size_t)n + 1));
    int32_t* ocol = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m + 1));
    int32_t* owt = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m + 1));
    int64_t* oeid = (int64_t*)malloc(sizeof(int64_t) * (size_t)(m + 1));
    if (!orow || !ocol || !owt || !oeid) {
        free(orow); free(ocol); free(owt); free(oeid);
        return OR_ENOMEM;
    }
    int rc = or_oriented_csr(n, m, u, v, w, orow, ocol, owt, oeid);
    if (rc != OR_OK) {
        free(orow); free(ocol); free(owt); free(oeid);
        return rc;
    }
    int nt = 1;
#ifdef _OPENMP
    nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#endif
    or_heap* heaps = (or_heap*)calloc((size_t)nt, sizeof(or_heap));
    int64_t* counts = (int64_t*)calloc((size_t)nt, sizeof(int64_t));
    int alloc_fail = 0;
    for (int t = 0; t < nt; t++) {
        heaps[t].cap = k;
        heaps[t].h = (or_tri*)malloc(sizeof(or_tri) * (size_t)k);
        if (!heaps[t].h) alloc_fail = 1;
    }
    if (!alloc_fail) {
#ifdef _OPENMP
#pragma omp parallel num_threads(nt)
#endif
        {
            int tid = 0;
#ifdef _OPENMP
            tid = omp_get_thread_num();
#endif
            or_heap* hp = &heaps[tid];
            int64_t local = 0;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 64)
#endif
            for (int32_t a = 0; a < n; a++) {
                for (int64_t i = orow[a]; i < orow[a + 1]; i++) {
                    int32_t b = ocol[i];
                    int64_t p = orow[a], pe = orow[a + 1];
                    int64_t q = orow[b], qe = orow[b + 1];
                    while (p < pe && q < qe) {
                        if (ocol[p] < ocol[q]) {
                            p++;
                        } else if (ocol[p] > ocol[q]) {
                            q++;
                        } else {
                            if (edge_sampled[oeid[i]] || edge_sampled[oeid[p]] || edge_sampled[oeid[q]]) {
                                or_tri x;
                                x.key = tri_key(pcode, preal, owt[i], owt[p], owt[q]);
                                x.t[0] = a;
                                x.t[1] = b;
                                x.t[2] = ocol[p];
                                sort3(x.t);
                                heap_offer(hp, &x);
                                local++;
                            }
                            p++;
                            q++;
                        }
                    }
                }
            }
            counts[tid] = local;
        }
        int64_t total = 0, pooled = 0;
        for (int t = 0; t < nt; t++) {
            total += counts[t];
            pooled += heaps[t].size;
        }
        or_tri* all = (or_tri*)malloc(sizeof(or_tri) * (size_t)(pooled + 1));
        if (!all) {
            rc = OR_ENOMEM;
        } else {
            int64_t at = 0;
            for (int t = 0; t < nt; t++) {
                memcpy(all + at, heaps[t].h, sizeof(or_tri) * (size_t)heaps[t].size);
                at += heaps[t].size;
            }
            qsort(all, (size_t)pooled, sizeof(or_tri), cmp_tri);
            int64_t out = pooled < k ? pooled : k;
            for (int64_t i = 0; i < out; i++) {
                tri[3 * i + 0] = all[i].t[0];
                tri[3 * i + 1] = all[i].t[1];
                tri[3 * i + 2] = all[i].t[2];
                key[i] = all[i].key;
                value[i] = tri_value(pcode, all[i].key);
            }
            *count = out;
            *ntri = total;
            free(all);
        }
    } else {
        rc = OR_ENOMEM;
    }
    for (int t = 0; t < nt; t++) free(heaps[t].h);
    free(heaps);
    free(counts);
    free(orow);
    free(ocol);
    free(owt);
    free(oeid);
    return rc;
}

/*
 * Top-k of the triangles whose first edge in the edge order (weight desc,
 * index asc) lies in shard `shard` of `nshards`, the edges being dealt to
 * shards in chunks of 2^chunk_shift consecutive positions, round-robin.
 * rank[i] is input edge i's position in the edge order.  Brute force over
 * every triangle (NodeIterator++), like or_topk.
 */
int or_topk_shard(int32_t n, int64_t m, const int32_t* u, const int32_t* v, const int32_t* w,
                  const int64_t* rank, int pcode, double preal, int64_t k, int32_t shard,
                  int32_t nshards, int chunk_shift, int32_t* tri, uint64_t* key, double* value,
                  int64_t* count, int64_t* ntri) {
    *count = 0;
    *ntri = 0;
    if (!pcode_ok(pcode, preal) || k <= 0 || nshards < 1 || shard < 0 || shard >= nshards)
        return OR_EINVAL;
    int64_t* orow = (int64_t*)malloc(sizeof(int64_t) * ((size_t)n + 1));
    int32_t* ocol = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m + 1));
    int32_t* owt = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m + 1));
    int64_t* oeid = (int64_t*)malloc(sizeof(int64_t) * (size_t)(m + 1));
    if (!orow || !ocol || !owt || !oeid) {
        free(orow); free(ocol); free(owt); free(oeid);
        return OR_ENOMEM;
    }
    int rc = or_oriented_csr(n, m, u, v, w, orow, ocol, owt, oeid);
    if (rc != OR_OK) {
        free(orow); free(ocol); free(owt); free(oeid);
        return rc;
    }
    or_heap hp;
    hp.cap = k;
    hp.size = 0;
    hp.h = (or_tri*)malloc(sizeof(or_tri) * (size_t)k);
    int64_t total = 0;
    if (!hp.h) rc = OR_ENOMEM;
    for (int32_t a = 0; a < n && rc == OR_OK; a++) {
        for (int64_t i = orow[a]; i < orow[a + 1]; i++) {
            int32_t b = ocol[i];
            int64_t p = orow[a], pe = orow[a + 1];
            int64_t q = orow[b], qe = orow[b + 1];
            while (p < pe && q < qe) {
                if (ocol[p] < ocol[q]) {
                    p++;
                } else if (ocol[p] > ocol[q]) {
                    q++;
                } else {
                    int64_t r0 = rank[oeid[i]], r1 = rank[oeid[p]], r2 = rank[oeid[q]];
                    int64_t own = r0 < r1 ? r0 : r1;
                    own = own < r2 ? own : r2;
                    if ((int32_t)((own >> chunk_shift) % nshards) == shard) {
                        or_tri x;
                        x.key = tri_key(pcode, preal, owt[i], owt[p], owt[q]);
                        x.t[0] = a;
                        x.t[1] = b;
                        x.t[2] = ocol[p];
                        sort3(x.t);
                        heap_offer(&hp, &x);
                        total++;
                    }
                    p++;
                    q++;
                }
            }
        }
    }
    if (rc == OR_OK) {
        qsort(hp.h, (size_t)hp.size, sizeof(or_tri), cmp_tri);
        for (int64_t i = 0; i < hp.size; i++) {
            tri[3 * i + 0] = hp.h[i].t[0];
            tri[3 * i + 1] = hp.h[i].t[1];
            tri[3 * i + 2] = hp.h[i].t[2];
            key[i] = hp.h[i].key;
            value[i] = tri_value(pcode, hp.h[i].key);
        }
        *count = hp.size;
        *ntri = total;
    }
    free(hp.h);
    free(orow);
    free(ocol);
    free(owt);
    free(oeid);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Weighted wedge sampling (Algorithm 4, Proposition 4.2, Section 4.2).     */
/* ------------------------------------------------------------------------ */

typedef unsigned __int128 or_u128;

/* floor(x * Z / 2^64) for a 64-bit x and Z < 2^128 (Z's high half < 2^64). */
static or_u128 mulhi_z(uint64_t x, or_u128 Z) {
    const uint64_t zl = (uint64_t)Z, zh = (uint64_t)(Z >> 64);
    return (or_u128)x * zh + (((or_u128)x * zl) >> 64);
}

static or_u128 wpow(int pcode, int32_t w) {
    const or_u128 x = (or_u128)(uint64_t)w;
    return pcode == 4 ? (or_u128)1 : (pcode == 1 ? x : x * x);
}

/*
 * Draws of Algorithm 4.  D(a) = sum over b in N(a) of w_ab^p.  Sample s uses
 * the words (x0, x1, x2) of Philox4x64-10(counter (s, 0, 0, 0), key
 * (seed, 1)):
 *   a: t = floor(x0 * Z1 / 2^64), Z1 = sum_v 2 d_v D(v); a = first vertex
 *      (by id) whose cumulative 2 d_v D(v) exceeds t (Eq. 6);
 *   b: a's neighbours in the edge order (the weight-sorted row), entry j with
 *      weight d_a w_j^p + D(a) (Eq. 7): t = floor(x1 * 2 d_a D(a) / 2^64);
 *      t < d_a D(a) picks j with the cumulative w^p first above t / d_a, else
 *      j = (t - d_a D(a)) / D(a) (the uniform part);
 *   c: entry j with weight w_j^p + w_ab^p (Eq. 8): t = floor(x2 * (D(a) +
 *      d_a w_ab^p) / 2^64); t < D(a) picks the cumulative w^p first above t,
 *      else j = (t - D(a)) / w_ab^p.
 * The wedge closes when c differs from b and {b, c} is an edge.  Outputs per
 * sample: center[s] = a, jb[s], jc[s] (positions in a's weight-sorted row)
 * and tri[3s..3s+2] = the sorted triangle or -1, -1, -1.  p codes 4 (p = 0),
 * 1 and 2 (w^p is an exact integer).
 */
int or_wedge_samples(int32_t n, int64_t m, const int32_t* u, const int32_t* v, const int32_t* w,
                     int pcode, int64_t nsamples, uint64_t seed, int32_t* center, int32_t* jb_out,
                     int32_t* jc_out, int32_t* tri) {
    if (pcode != 1 && pcode != 2 && pcode != 4) return OR_EINVAL;
    if (m <= 0) {
        for (int64_t s = 0; s < nsamples; s++) {
            center[s] = jb_out[s] = jc_out[s] = -1;
            tri[3 * s] = tri[3 * s + 1] = tri[3 * s + 2] = -1;
        }
        return OR_OK;
    }
    int rc = OR_OK;
    int64_t* perm = (int64_t*)malloc(sizeof(int64_t) * (size_t)m);
    int64_t* deg = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    int64_t* wrow = (int64_t*)malloc(sizeof(int64_t) * ((size_t)n + 1));
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * ((size_t)n + 1));
    int32_t* wc = (int32_t*)malloc(sizeof(int32_t) * (size_t)(2 * m));
    int32_t* ww = (int32_t*)malloc(sizeof(int32_t) * (size_t)(2 * m));
    or_u128* P = (or_u128*)malloc(sizeof(or_u128) * (size_t)(2 * m));
    or_u128* D = (or_u128*)calloc((size_t)n, sizeof(or_u128));
    or_u128* C1 = (or_u128*)malloc(sizeof(or_u128) * (size_t)n);
    int64_t* srow = (int64_t*)malloc(sizeof(int64_t) * ((size_t)n + 1));
    int32_t* scl = (int32_t*)malloc(sizeof(int32_t) * (size_t)(2 * m));
    int32_t* swt = (int32_t*)malloc(sizeof(int32_t) * (size_t)(2 * m));
    int64_t* seid = (int64_t*)malloc(sizeof(int64_t) * (size_t)(2 * m));
    if (!perm || !deg || !wrow || !fill || !wc || !ww || !P || !D || !C1 || !srow || !scl || !swt || !seid) {
        rc = OR_ENOMEM;
        goto done;
    }
    rc = or_edge_order(m, w, perm);
    if (rc != OR_OK) goto done;
    rc = or_sym_csr(n, m, u, v, w, srow, scl, swt, seid); /* validates too */
    if (rc != OR_OK) goto done;
    /* weight-sorted rows: append every edge, in edge order, to both rows */
    for (int64_t i = 0; i < m; i++) {
        deg[u[i]]++;
        deg[v[i]]++;
    }
    wrow[0] = 0;
    for (int32_t x = 0; x < n; x++) wrow[x + 1] = wrow[x] + deg[x];
    for (int32_t x = 0; x <= n; x++) fill[x] = wrow[x];
    for (int64_t r = 0; r < m; r++) {
        const int64_t e = perm[r];
        wc[fill[u[e]]] = v[e];
        ww[fill[u[e]]++] = w[e];
        wc[fill[v[e]]] = u[e];
        ww[fill[v[e]]++] = w[e];
    }
    {
        or_u128 acc = 0;
        for (int32_t x = 0; x < n; x++) {
            or_u128 rs = 0;
            for (int64_t j = wrow[x]; j < wrow[x + 1]; j++) {
                rs += wpow(pcode, ww[j]);
                P[j] = rs; /* cumulative w^p within the row */
            }
            D[x] = rs;
            acc += (or_u128)2 * (or_u128)(uint64_t)deg[x] * rs;
            C1[x] = acc;
        }
    }
    {
        const or_u128 Z1 = C1[n - 1];
        const uint64_t key[2] = {seed, 1};
        for (int64_t s = 0; s < nsamples; s++) {
            uint64_t ctr[4] = {(uint64_t)s, 0, 0, 0}, x[4];
            or_philox4x64_10(ctr, key, x);
            const or_u128 t1 = mulhi_z(x[0], Z1);
            int32_t lo = 0, hi = n - 1; /* first vertex with C1 > t1 */
            while (lo < hi) {
                const int32_t mid = lo + (hi - lo) / 2;
                if (C1[mid] > t1) hi = mid;
                else lo = mid + 1;
            }
            const int32_t a = lo;
            const int64_t b0 = wrow[a], da = deg[a];
            const or_u128 Da = D[a];
            /* b: d_a w^p + D(a) */
            const or_u128 dD = (or_u128)(uint64_t)da * Da;
            const or_u128 t2 = mulhi_z(x[1], 2 * dD);
            int64_t jb;
            if (t2 < dD) {
                const or_u128 tp = t2 / (or_u128)(uint64_t)da;
                int64_t l2 = 0, h2 = da - 1;
                while (l2 < h2) {
                    const int64_t mid = l2 + (h2 - l2) / 2;
                    if (P[b0 + mid] > tp) h2 = mid;
                    else l2 = mid + 1;
                }
                jb = l2;
            } else {
                jb = (int64_t)((t2 - dD) / Da);
            }
            /* c: w_c^p + w_ab^p */
            const or_u128 wab = wpow(pcode, ww[b0 + jb]);
            const or_u128 t3 = mulhi_z(x[2], Da + (or_u128)(uint64_t)da * wab);
            int64_t jc;
            if (t3 < Da) {
                int64_t l2 = 0, h2 = da - 1;
                while (l2 < h2) {
                    const int64_t mid = l2 + (h2 - l2) / 2;
                    if (P[b0 + mid] > t3) h2 = mid;
                    else l2 = mid + 1;
                }
                jc = l2;
            } else {
                jc = (int64_t)((t3 - Da) / wab);
            }
            center[s] = a;
            jb_out[s] = (int32_t)jb;
            jc_out[s] = (int32_t)jc;
            tri[3 * s] = tri[3 * s + 1] = tri[3 * s + 2] = -1;
            if (jb != jc) {
                const int32_t b = wc[b0 + jb], c = wc[b0 + jc];
                /* closure: is c in N(b)?  (id-sorted row of b) */
                int64_t l2 = srow[b], h2 = srow[b + 1];
                while (l2 < h2) {
                    const int64_t mid = l2 + (h2 - l2) / 2;
                    if (scl[mid] < c) l2 = mid + 1;
                    else h2 = mid;
                }
                if (l2 < srow[b + 1] && scl[l2] == c) {
                    int32_t t3v[3] = {a, b, c};
                    sort3(t3v);
                    tri[3 * s] = t3v[0];
                    tri[3 * s + 1] = t3v[1];
                    tri[3 * s + 2] = t3v[2];
                }
            }
        }
    }
done:
    free(perm); free(deg); free(wrow); free(fill); free(wc); free(ww); free(P); free(D); free(C1);
    free(srow); free(scl); free(swt); free(seid);
    return rc;
}

static int cmp_triple(const void* pa, const void* pb) {
    const int32_t* x = (const int32_t*)pa;
    const int32_t* y = (const int32_t*)pb;
    for (int i = 0; i < 3; i++)
        if (x[i] != y[i]) return x[i] < y[i] ? -1 : 1;
    return 0;
}

/*
 * Top-k of Algorithm 4's triangle set T (every distinct triangle some sample
 * closed), scored like or_topk.  *ntri receives |T|.
 */
int or_wedge_topk(int32_t n, int64_t m, const int32_t* u, const int32_t* v, const int32_t* w,
                  int pcode, int64_t k, int64_t nsamples, uint64_t seed, int32_t* tri, uint64_t* key,
                  double* value, int64_t* count, int64_t* ntri) {
    *count = 0;
    *ntri = 0;
    if ((pcode != 1 && pcode != 2 && pcode != 4) || k <= 0 || nsamples < 0) return OR_EINVAL;
    if (nsamples == 0 || m == 0) return OR_OK;
    int32_t* ctr = (int32_t*)malloc(sizeof(int32_t) * (size_t)nsamples * 3);
    int32_t* st = (int32_t*)malloc(sizeof(int32_t) * (size_t)nsamples * 3);
    int64_t* rowp = (int64_t*)malloc(sizeof(int64_t) * ((size_t)n + 1));
    int32_t* col = (int32_t*)malloc(sizeof(int32_t) * (size_t)(2 * m));
    int32_t* wt = (int32_t*)malloc(sizeof(int32_t) * (size_t)(2 * m));
    int64_t* eid = (int64_t*)malloc(sizeof(int64_t) * (size_t)(2 * m));
    int rc = OR_ENOMEM;
    if (ctr && st && rowp && col && wt && eid) {
        rc = or_wedge_samples(n, m, u, v, w, pcode, nsamples, seed, ctr, ctr + nsamples,
                              ctr + 2 * nsamples, st);
        if (rc == OR_OK) rc = or_sym_csr(n, m, u, v, w, rowp, col, wt, eid);
    }
    if (rc == OR_OK) {
        /* the distinct closed triangles */
        int64_t nt = 0;
        for (int64_t s = 0; s < nsamples; s++)
            if (st[3 * s] >= 0) {
                st[3 * nt] = st[3 * s];
                st[3 * nt + 1] = st[3 * s + 1];
                st[3 * nt + 2] = st[3 * s + 2];
                nt++;
            }
        qsort(st, (size_t)nt, 3 * sizeof(int32_t), cmp_triple);
        int64_t nu = 0;
        for (int64_t i = 0; i < nt; i++)
            if (nu == 0 || cmp_triple(st + 3 * i, st + 3 * (nu - 1)) != 0) {
                memmove(st + 3 * nu, st + 3 * i, 3 * sizeof(int32_t));
                nu++;
            }
        or_tri* all = (or_tri*)malloc(sizeof(or_tri) * (size_t)(nu + 1));
        if (!all) {
            rc = OR_ENOMEM;
        } else {
            for (int64_t i = 0; i < nu; i++) {
                int32_t ws[3];
                const int32_t a = st[3 * i], b = st[3 * i + 1], c = st[3 * i + 2];
                const int32_t pr[3][2] = {{a, b}, {b, c}, {a, c}};
                for (int e = 0; e < 3; e++) {
                    const int32_t x = pr[e][0], y = pr[e][1];
                    int64_t l2 = rowp[x], h2 = rowp[x + 1];
                    while (l2 < h2) {
                        const int64_t mid = l2 + (h2 - l2) / 2;
                        if (col[mid] < y) l2 = mid + 1;
                        else h2 = mid;
                    }
                    ws[e] = wt[l2];
                }
                all[i].key = tri_key(pcode, 0.0, ws[0], ws[1], ws[2]);
                all[i].t[0] = a;
                all[i].t[1] = b;
                all[i].t[2] = c;
            }
            qsort(all, (size_t)nu, sizeof(or_tri), cmp_tri);
            const int64_t out = nu < k ? nu : k;
            for (int64_t i = 0; i < out; i++) {
                tri[3 * i] = all[i].t[0];
                tri[3 * i + 1] = all[i].t[1];
                tri[3 * i + 2] = all[i].t[2];
                key[i] = all[i].key;
                value[i] = tri_value(pcode, all[i].key);
            }
            *count = out;
            *ntri = nu;
            free(all);
        }
    }
    free(ctr); free(st); free(rowp); free(col); free(wt); free(eid);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Top weighted cliques (Section 4.5, Appendix A).                          */
/* ------------------------------------------------------------------------ */

/*
 * The weight of a q-clique is the generalized p-mean of the weights of its
 * q(q-1)/2 edges (Appendix A).  Keys, exact and monotone in that mean, for
 * p in {-inf, 1, 2, +inf} (codes 0..3): the minimum, the sum, the sum of
 * squares (weights at most 2^30, so that ten squares fit 64 bits) and the
 * maximum of the edge weights.  p = 0 and other finite p are not taken (the
 * product of ten weights has no 64-bit key).  Value: min, sum / E,
 * sqrt(sum of squares / E), max with E = q(q-1)/2.
 */
#define OR_CLIQUE_P2_WMAX (1 << 30)

typedef struct {
    uint64_t key;
    int32_t t[5];
} or_clq;

static int g_clq_q;

static int cmp_clq(const void* a, const void* b) {
    const or_clq* x = (const or_clq*)a;
    const or_clq* y = (const or_clq*)b;
    if (x->key != y->key) return x->key > y->key ? -1 : 1;
    for (int i = 0; i < g_clq_q; i++)
        if (x->t[i] != y->t[i]) return x->t[i] < y->t[i] ? -1 : 1;
    return 0;
}

/* Position of b in a's id-sorted row, or -1. */
static int64_t row_find(const int64_t* rowptr, const int32_t* col, int32_t a, int32_t b) {
    int64_t lo = rowptr[a], hi = rowptr[a + 1];
    while (lo < hi) {
        int64_t mid = (lo + hi) / 2;
        if (col[mid] < b) lo = mid + 1;
        else hi = mid;
    }
    return (lo < rowptr[a + 1] && col[lo] == b) ? lo : -1;
}

static uint64_t clique_key(int pcode, const int32_t* wts, int ne) {
    uint64_t acc = (pcode == 0) ? UINT64_MAX : 0;
    for (int i = 0; i < ne; i++) {
        uint64_t x = (uint64_t)wts[i];
        if (pcode == 0) acc = x < acc ? x : acc;
        else if (pcode == 1) acc += x;
        else if (pcode == 2) acc += x * x;
        else acc = x > acc ? x : acc;
    }
    return acc;
}

static double clique_value(int pcode, uint64_t key, int ne) {
    if (pcode == 1) return (double)key / (double)ne;
    if (pcode == 2) return sqrt((double)key / (double)ne);
    return (double)key;
}

/*
 * Top-k q-cliques (q = 4 or 5) under (weight desc, sorted vertex tuple asc).
 * edge_sampled == NULL: every clique of the graph; else only the cliques
 * with at least one edge i with edge_sampled[i] != 0 -- the set that edge
 * sampling enumerates (Section 4.5: sample edges, enumerate the cliques on
 * them).  Every clique is listed once, as vertices a < b < c < d (< e) with
 * every pair adjacent, then all of them are sorted.  ids receives q ids
 * per clique, ascending; *nclq the number of cliques in the set.
 */
int or_clique_topk(int32_t n, int64_t m, const int32_t* u, const int32_t* v, const int32_t* w,
                   int q, int pcode, const uint8_t* edge_sampled, int64_t k, int32_t* ids,
                   uint64_t* key, double* value, int64_t* count, int64_t* nclq) {
    *count = 0;
    *nclq = 0;
    if ((q != 4 && q != 5) || pcode < 0 || pcode > 3 || k <= 0) return OR_EINVAL;
    if (pcode == 2)
        for (int64_t i = 0; i < m; i++)
            if (w[i] > OR_CLIQUE_P2_WMAX) return OR_EINVAL;
    int64_t* rowptr = (int64_t*)malloc(sizeof(int64_t) * ((size_t)n + 1));
    int32_t* col = (int32_t*)malloc(sizeof(int32_t) * (size_t)(2 * m + 1));
    int32_t* wt = (int32_t*)malloc(sizeof(int32_t) * (size_t)(2 * m + 1));
    int64_t* eid = (int64_t*)malloc(sizeof(int64_t) * (size_t)(2 * m + 1));
    if (!rowptr || !col || !wt || !eid) {
        free(rowptr); free(col); free(wt); free(eid);
        return OR_ENOMEM;
    }
    int rc = or_sym_csr(n, m, u, v, w, rowptr, col, wt, eid);
    const int ne = q * (q - 1) / 2;
    int64_t cap = 1024, len = 0;
    or_clq* all = (or_clq*)malloc(sizeof(or_clq) * (size_t)cap);
    if (!all) rc = OR_ENOMEM;
    int32_t t[5];
    for (int32_t a = 0; a < n && rc == OR_OK; a++) {
        t[0] = a;
        /* extend t[0..depth) by neighbours of a above t[depth-1], adjacent to all */
        int64_t pos[5];
        int depth = 1;
        pos[1] = rowptr[a];
        while (depth > 0 && rc == OR_OK) {
            if (depth == q) {
                int32_t wts[10];
                int sampled = edge_sampled == NULL;
                int e = 0;
                for (int i = 0; i < q; i++)
                    for (int j = i + 1; j < q; j++) {
                        int64_t p_ = row_find(rowptr, col, t[i], t[j]);
                        wts[e++] = wt[p_];
                        if (edge_sampled && edge_sampled[eid[p_]]) sampled = 1;
                    }
                if (sampled) {
                    if (len == cap) {
                        or_clq* grown = (or_clq*)realloc(all, sizeof(or_clq) * (size_t)(2 * cap));
                        if (!grown) {
                            rc = OR_ENOMEM;
                            break;
                        }
                        all = grown;
                        cap *= 2;
                    }
                    all[len].key = clique_key(pcode, wts, ne);
                    for (int i = 0; i < 5; i++) all[len].t[i] = i < q ? t[i] : 0;
                    len++;
                }
                depth--;
                continue;
            }
            /* next candidate for slot `depth`: a neighbour of a above t[depth-1] */
            int found = 0;
            while (pos[depth] < rowptr[a + 1]) {
                int32_t c = col[pos[depth]++];
                if (c <= t[depth - 1]) continue;
                int adj = 1;
                for (int i = 1; i < depth && adj; i++) adj = row_find(rowptr, col, t[i], c) >= 0;
                if (adj) {
                    t[depth] = c;
                    found = 1;
                    break;
                }
            }
            if (found) {
                depth++;
                if (depth < q) pos[depth] = pos[depth - 1];  /* the row is id-sorted */
            } else {
                depth--;
            }
        }
    }
    if (rc == OR_OK) {
        g_clq_q = q;
        qsort(all, (size_t)len, sizeof(or_clq), cmp_clq);
        int64_t out = len < k ? len : k;
        for (int64_t i = 0; i < out; i++) {
            for (int j = 0; j < q; j++) ids[q * i + j] = all[i].t[j];
            key[i] = all[i].key;
            value[i] = clique_value(pcode, all[i].key, ne);
        }
        *count = out;
        *nclq = len;
    }
    free(all);
    free(rowptr);
    free(col);
    free(wt);
    free(eid);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Real (fp32) edge weights: Eq. 1 over positive reals.                       */
/* ------------------------------------------------------------------------ */

/*
 * m_p of three positive fp32 weights, in fp64: min, max (p = -inf, +inf),
 * (a+b+c)/3 (p = 1), sqrt((a^2+b^2+c^2)/3) (p = 2), cbrt(a*b*c) (p = 0), and
 * Eq. 1 with the largest (p > 0) or smallest (p < 0) weight factored out for
 * any other finite p.  The weights are taken in ascending order.
 */
static double real_mean(int pcode, double p, float fa, float fb, float fc) {
    double t3[3] = {fa, fb, fc}, x;
    if (t3[0] > t3[1]) { x = t3[0]; t3[0] = t3[1]; t3[1] = x; }
    if (t3[1] > t3[2]) { x = t3[1]; t3[1] = t3[2]; t3[2] = x; }
    if (t3[0] > t3[1]) { x = t3[0]; t3[0] = t3[1]; t3[1] = x; }
    switch (pcode) {
        case 0: return t3[0];
        case 3: return t3[2];
        case 1: return (t3[0] + t3[1] + t3[2]) / 3.0;
        case 2: return sqrt((t3[0] * t3[0] + t3[1] * t3[1] + t3[2] * t3[2]) / 3.0);
        case 4: return cbrt(t3[0] * t3[1] * t3[2]);
        default: {
            const double s = p > 0 ? t3[2] : t3[0];
            const double t = (pow(t3[0] / s, p) + pow(t3[1] / s, p) + pow(t3[2] / s, p)) / 3.0;
            return s * pow(t, 1.0 / p);
        }
    }
}

/*
 * Top-k triangles of a graph with positive finite fp32 weights (Eq. 1 over
 * reals), p code as or_topk (general p: preal).  The key is the fp64 mean's
 * bit pattern (positive doubles order like their values).  Every triangle
 * {a < b < c} is enumerated once from the id-sorted rows, then all are
 * sorted by (key desc, triple asc).  Weights are checked: a non-finite or
 * non-positive weight is OR_EINVAL.
 */
int or_topk_real(int32_t n, int64_t m, const int32_t* u, const int32_t* v, const float* w, int pcode,
                 double preal, int64_t k, int32_t* tri, uint64_t* key, double* value, int64_t* count,
                 int64_t* ntri) {
    *count = 0;
    *ntri = 0;
    if (pcode < 0 || pcode > OR_PCODE_MAX || k <= 0) return OR_EINVAL;
    if (pcode == 5 && !(isfinite(preal) && preal != 0.0 && preal != 1.0 && preal != 2.0)) return OR_EINVAL;
    int32_t* bits = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m + 1));
    int64_t* rowptr = (int64_t*)malloc(sizeof(int64_t) * ((size_t)n + 1));
    int32_t* col = (int32_t*)malloc(sizeof(int32_t) * (size_t)(2 * m + 1));
    int32_t* wt = (int32_t*)malloc(sizeof(int32_t) * (size_t)(2 * m + 1));
    int64_t* eid = (int64_t*)malloc(sizeof(int64_t) * (size_t)(2 * m + 1));
    int rc = (bits && rowptr && col && wt && eid) ? OR_OK : OR_ENOMEM;
    for (int64_t i = 0; i < m && rc == OR_OK; i++) {
        if (!(isfinite(w[i]) && w[i] > 0.0f)) rc = OR_EINVAL;
        memcpy(&bits[i], &w[i], 4); /* positive: a positive int32 */
    }
    if (rc == OR_OK) rc = or_sym_csr(n, m, u, v, bits, rowptr, col, wt, eid);
    int64_t cap = 1024, len = 0;
    or_tri* all = rc == OR_OK ? (or_tri*)malloc(sizeof(or_tri) * (size_t)cap) : NULL;
    if (rc == OR_OK && !all) rc = OR_ENOMEM;
    for (int32_t a = 0; a < n && rc == OR_OK; a++)
        for (int64_t i = rowptr[a]; i < rowptr[a + 1] && rc == OR_OK; i++) {
            const int32_t b = col[i];
            if (b <= a) continue;
            for (int64_t j = i + 1; j < rowptr[a + 1]; j++) {
                const int32_t c = col[j];  /* c > b: the row is id-sorted */
                const int64_t pbc = row_find(rowptr, col, b, c);
                if (pbc < 0) continue;
                float fab, fac, fbc;
                memcpy(&fab, &wt[i], 4);
                memcpy(&fac, &wt[j], 4);
                memcpy(&fbc, &wt[pbc], 4);
                const double mp = real_mean(pcode, preal, fab, fac, fbc);
                if (len == cap) {
                    or_tri* grown = (or_tri*)realloc(all, sizeof(or_tri) * (size_t)(2 * cap));
                    if (!grown) {
                        rc = OR_ENOMEM;
                        break;
                    }
                    all = grown;
                    cap *= 2;
                }
                memcpy(&all[len].key, &mp, 8);
                all[len].t[0] = a;
                all[len].t[1] = b;
                all[len].t[2] = c;
                len++;
            }
        }
    if (rc == OR_OK) {
        qsort(all, (size_t)len, sizeof(or_tri), cmp_tri);
        const int64_t out = len < k ? len : k;
        for (int64_t i = 0; i < out; i++) {
            for (int t = 0; t < 3; t++) tri[3 * i + t] = all[i].t[t];
            key[i] = all[i].key;
            memcpy(&value[i], &all[i].key, 8);
        }
        *count = out;
        *ntri = len;
    }
    free(all);
    free(bits);
    free(rowptr);
    free(col);
    free(wt);
    free(eid);
    return rc;
}
