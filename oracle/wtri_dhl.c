/*
 * The paper's own exact CPU algorithm: dynamic heavy-light (Algorithm 2,
 * Section 3.2) and its distribution-oblivious form (Auto-HL, the end of
 * Section 3.3), single-threaded like the paper's main loop (Section 5.3).
 *
 * TEST INFRASTRUCTURE and prior-art CPU baseline: only the test suite and
 * the CPU-baseline leg of bench.py call this.  It shares no code with the
 * CUDA path nor with the brute-force oracle in wtri_oracle.c (its own
 * scoring, ordering and adjacency structures), so the two CPU programs check
 * each other.
 *
 * The edges are sorted by (weight desc, index asc); e_r is the r-th.  Three
 * classes: S = e_0..e_h (super-heavy), H = e_{h+1}..e_l (heavy), L = the
 * rest (light).  Each step moves one edge up a class and lists triangles:
 *   L -> H (e = e_{l+1}): triangles of e with at least one more edge in S u H;
 *   H -> S (e = e_{h+1}): triangles of e whose other two edges are in L.
 * Invariant after every step: every triangle with an edge in S or two edges
 * in H is listed, so a triangle not yet listed has at most one edge in H and
 * at least two in L, and its key is at most K(w_{h+1}, w_{l+1}, w_{l+2})
 * (the tight bound of Section 3.2, taken in the exact key space of Eq. 1's
 * p-mean, which is monotone in each weight).  The loop stops once the k-th
 * best key listed exceeds that bound (strictly, so that unlisted triangles
 * tied with the k-th can still win the tie-break on the vertex triple), or
 * once L is empty.
 *
 * Readings (the printed algorithm is garbled in places):
 *  - promotion rule: the paper keeps w_h ~ w_l^alpha_p (Section 3.3); the
 *    condition as printed can never hold for weights > 1 and alpha > 1, so
 *    the L -> H move is taken when w_{l+1}^alpha > w_{h+1}, and always when H
 *    is empty (h == l);
 *  - the H -> S branch lists the triangles of the edge it moves, e_{h+1};
 *  - alpha_p = 2 - p / (p - 1 + beta) for power-law weights with exponent
 *    beta (Section 3.3); it tends to 1 as p -> +-inf;
 *  - Auto-HL estimates both pointers' "threshold decrease per unit of work"
 *    on the fly: the average weight drop over the run of equal weights at
 *    the pointer, turned into a decrease of tau = w_h^p + 2 w_l^p, divided by
 *    the degree sum of the moved edge's endpoints in G_L (h) or G_{S u H} (l).
 *    The paper gives it for finite p; at p = +-inf it takes the alpha = 1 rule.
 *
 * The answer is exact whatever the promotion rule: only speed depends on it.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define DHL_OK 0
#define DHL_EINVAL (-1)
#define DHL_ENOMEM (-2)

/* exact key of the p-mean (pcode 0: -inf, 1: p=1, 2: p=2, 3: +inf, 4: p=0,
 * the geometric mean, ranked by the product of the weights) */
static uint64_t dhl_key(int pcode, uint64_t a, uint64_t b, uint64_t c) {
    switch (pcode) {
        case 0: return a < b ? (a < c ? a : c) : (b < c ? b : c);
        case 1: return a + b + c;
        case 2: return a * a + b * b + c * c;
        case 4: return a * b * c;
        default: return a > b ? (a > c ? a : c) : (b > c ? b : c);
    }
}

static double dhl_value(int pcode, uint64_t key) {
    if (pcode == 1) return (double)key / 3.0;
    if (pcode == 2) return sqrt((double)key / 3.0);
    if (pcode == 4) return cbrt((double)key);
    return (double)key;
}

/* ---- listed triangles: open-addressing set ------------------------------ */
typedef struct {
    uint64_t key;
    int32_t t[3]; /* ascending; t[0] = -1 marks an empty slot */
} dhl_tri;

typedef struct {
    dhl_tri* slot;
    uint64_t cap, size;
} dhl_set;

static uint64_t tri_hash(const int32_t* t) {
    uint64_t x = ((uint64_t)(uint32_t)t[0] << 32) ^ (uint64_t)(uint32_t)t[1];
    x ^= (uint64_t)(uint32_t)t[2] * 0x9E3779B97F4A7C15ull;
    x ^= x >> 31;
    x *= 0xBF58476D1CE4E5B9ull;
    x ^= x >> 29;
    return x;
}

static int set_init(dhl_set* s, uint64_t cap) {
    s->cap = cap;
    s->size = 0;
    s->slot = (dhl_tri*)malloc(sizeof(dhl_tri) * cap);
    if (!s->slot) return DHL_ENOMEM;
    for (uint64_t i = 0; i < cap; i++) s->slot[i].t[0] = -1;
    return DHL_OK;
}

/* 1 if inserted, 0 if already present, <0 on allocation failure */
static int set_insert(dhl_set* s, const dhl_tri* x);

static int set_grow(dhl_set* s) {
    dhl_set b;
    if (set_init(&b, s->cap * 2) != DHL_OK) return DHL_ENOMEM;
    for (uint64_t i = 0; i < s->cap; i++)
        if (s->slot[i].t[0] >= 0) set_insert(&b, &s->slot[i]);
    free(s->slot);
    *s = b;
    return DHL_OK;
}

static int set_insert(dhl_set* s, const dhl_tri* x) {
    if (2 * (s->size + 1) > s->cap && set_grow(s) != DHL_OK) return DHL_ENOMEM;
    uint64_t i = tri_hash(x->t) & (s->cap - 1);
    for (;;) {
        dhl_tri* y = &s->slot[i];
        if (y->t[0] < 0) {
            *y = *x;
            s->size++;
            return 1;
        }
        if (y->t[0] == x->t[0] && y->t[1] == x->t[1] && y->t[2] == x->t[2]) return 0;
        i = (i + 1) & (s->cap - 1);
    }
}

/* ---- k largest keys: min-heap ------------------------------------------- */
typedef struct {
    uint64_t* h;
    int64_t size, cap;
} dhl_heap;

static void kheap_offer(dhl_heap* q, uint64_t key) {
    if (q->size < q->cap) {
        int64_t i = q->size++;
        q->h[i] = key;
        while (i > 0 && q->h[(i - 1) / 2] > q->h[i]) {
            uint64_t t = q->h[i];
            q->h[i] = q->h[(i - 1) / 2];
            q->h[(i - 1) / 2] = t;
            i = (i - 1) / 2;
        }
    } else if (key > q->h[0]) {
        q->h[0] = key;
        int64_t i = 0;
        for (;;) {
            int64_t l = 2 * i + 1, r = l + 1, s = i;
            if (l < q->size && q->h[l] < q->h[s]) s = l;
            if (r < q->size && q->h[r] < q->h[s]) s = r;
            if (s == i) break;
            uint64_t t = q->h[i];
            q->h[i] = q->h[s];
            q->h[s] = t;
            i = s;
        }
    }
}

/* ---- graph structures ----------------------------------------------------- */
typedef struct {
    int32_t nbr;
    uint32_t rank;
} dhl_ent;

typedef struct {
    int32_t n;
    int64_t m;
    int pcode;
    uint32_t* ew;       /* weight of e_r */
    int32_t* ea;        /* endpoints of e_r */
    int32_t* eb;
    int64_t* ptr;       /* row offsets, n + 1 */
    dhl_ent* by_rank;   /* row x: neighbours in edge order (rank ascending) */
    dhl_ent* by_id;     /* row x: neighbours by id ascending */
    dhl_set set;
    dhl_heap heap;
    int64_t probes;
} dhl_ctx;

/* rank of edge {x, y}, or -1: binary search in the shorter id-sorted row */
static int64_t find_edge(dhl_ctx* g, int32_t x, int32_t y) {
    if (g->ptr[x + 1] - g->ptr[x] > g->ptr[y + 1] - g->ptr[y]) {
        int32_t t = x;
        x = y;
        y = t;
    }
    int64_t lo = g->ptr[x], hi = g->ptr[x + 1];
    g->probes++;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (g->by_id[mid].nbr < y) lo = mid + 1;
        else hi = mid;
    }
    if (lo < g->ptr[x + 1] && g->by_id[lo].nbr == y) return (int64_t)g->by_id[lo].rank;
    return -1;
}

/* number of entries of x's edge-ordered row with rank <= r */
static int64_t rank_prefix(const dhl_ctx* g, int32_t x, int64_t r) {
    int64_t lo = g->ptr[x], hi = g->ptr[x + 1];
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if ((int64_t)g->by_rank[mid].rank <= r) lo = mid + 1;
        else hi = mid;
    }
    return lo - g->ptr[x];
}

static int offer(dhl_ctx* g, int32_t a, int32_t b, int32_t c, uint64_t wab, uint64_t wac,
                 uint64_t wbc) {
    dhl_tri x;
    x.key = dhl_key(g->pcode, wab, wac, wbc);
    if (g->heap.size == g->heap.cap && x.key < g->heap.h[0]) return DHL_OK; /* can never rank */
    int32_t t;
    if (a > b) { t = a; a = b; b = t; }
    if (b > c) { t = b; b = c; c = t; }
    if (a > b) { t = a; a = b; b = t; }
    x.t[0] = a;
    x.t[1] = b;
    x.t[2] = c;
    int ins = set_insert(&g->set, &x);
    if (ins < 0) return DHL_ENOMEM;
    if (ins) kheap_offer(&g->heap, x.key);
    return DHL_OK;
}

static uint64_t W(const dhl_ctx* g, int64_t r) { return r < g->m ? g->ew[r] : 0u; }

static int cmp_out(const void* pa, const void* pb) {
    const dhl_tri* x = (const dhl_tri*)pa;
    const dhl_tri* y = (const dhl_tri*)pb;
    if (x->key != y->key) return x->key > y->key ? -1 : 1;
    for (int i = 0; i < 3; i++)
        if (x->t[i] != y->t[i]) return x->t[i] < y->t[i] ? -1 : 1;
    return 0;
}

/* Build the edge order and both row layouts.  Rejects self-loops, ids out of
 * range, weights <= 0 and repeated pairs. */
static int prepare(dhl_ctx* g, const int32_t* u, const int32_t* v, const int32_t* w) {
    const int64_t m = g->m;
    const int32_t n = g->n;
    int32_t wmax = 0;
    for (int64_t i = 0; i < m; i++) {
        if (u[i] < 0 || u[i] >= n || v[i] < 0 || v[i] >= n || u[i] == v[i] || w[i] <= 0)
            return DHL_EINVAL;
        if (w[i] > wmax) wmax = w[i];
    }
    /* stable LSD radix sort of the indices by wmax - w (two 16-bit digits):
       weight descending, index ascending among equal weights */
    uint32_t* idx = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(m ? m : 1));
    uint32_t* tmp = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(m ? m : 1));
    int64_t* cnt = (int64_t*)malloc(sizeof(int64_t) * 65537);
    if (!idx || !tmp || !cnt) {
        free(idx);
        free(tmp);
        free(cnt);
        return DHL_ENOMEM;
    }
    for (int64_t i = 0; i < m; i++) idx[i] = (uint32_t)i;
    for (int pass = 0; pass < 2; pass++) {
        const int sh = 16 * pass;
        memset(cnt, 0, sizeof(int64_t) * 65537);
        for (int64_t i = 0; i < m; i++) cnt[(((uint32_t)(wmax - w[idx[i]])) >> sh & 0xffffu) + 1]++;
        for (int d = 0; d < 65536; d++) cnt[d + 1] += cnt[d];
        for (int64_t i = 0; i < m; i++) tmp[cnt[((uint32_t)(wmax - w[idx[i]])) >> sh & 0xffffu]++] = idx[i];
        uint32_t* s = idx;
        idx = tmp;
        tmp = s;
    }
    free(tmp);
    free(cnt);
    g->ew = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(m ? m : 1));
    g->ea = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m ? m : 1));
    g->eb = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m ? m : 1));
    g->ptr = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    g->by_rank = (dhl_ent*)malloc(sizeof(dhl_ent) * (size_t)(2 * m ? 2 * m : 1));
    g->by_id = (dhl_ent*)malloc(sizeof(dhl_ent) * (size_t)(2 * m ? 2 * m : 1));
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * ((size_t)n + 1));
    if (!g->ew || !g->ea || !g->eb || !g->ptr || !g->by_rank || !g->by_id || !fill) {
        free(idx);
        free(fill);
        return DHL_ENOMEM;
    }
    for (int64_t r = 0; r < m; r++) {
        const uint32_t i = idx[r];
        g->ew[r] = (uint32_t)w[i];
        g->ea[r] = u[i];
        g->eb[r] = v[i];
        g->ptr[u[i] + 1]++;
        g->ptr[v[i] + 1]++;
    }
    free(idx);
    for (int32_t x = 0; x < n; x++) g->ptr[x + 1] += g->ptr[x];
    /* rows in edge order: append edges by rank */
    memcpy(fill, g->ptr, sizeof(int64_t) * ((size_t)n + 1));
    for (int64_t r = 0; r < m; r++) {
        g->by_rank[fill[g->ea[r]]++] = (dhl_ent){g->eb[r], (uint32_t)r};
        g->by_rank[fill[g->eb[r]]++] = (dhl_ent){g->ea[r], (uint32_t)r};
    }
    /* rows by id: walk rows in id order and append x to each neighbour's row */
    memcpy(fill, g->ptr, sizeof(int64_t) * ((size_t)n + 1));
    for (int32_t x = 0; x < n; x++)
        for (int64_t j = g->ptr[x]; j < g->ptr[x + 1]; j++) {
            const dhl_ent e = g->by_rank[j];
            g->by_id[fill[e.nbr]++] = (dhl_ent){x, e.rank};
        }
    free(fill);
    for (int32_t x = 0; x < n; x++)
        for (int64_t j = g->ptr[x] + 1; j < g->ptr[x + 1]; j++)
            if (g->by_id[j].nbr == g->by_id[j - 1].nbr) return DHL_EINVAL;
    return DHL_OK;
}

static void release(dhl_ctx* g) {
    free(g->ew);
    free(g->ea);
    free(g->eb);
    free(g->ptr);
    free(g->by_rank);
    free(g->by_id);
    free(g->set.slot);
    free(g->heap.h);
}

/* L -> H: triangles of e_r (r = l + 1) with another edge in S u H (ranks < r) */
static int move_light_up(dhl_ctx* g, int64_t r) {
    const int32_t a = g->ea[r], b = g->eb[r];
    const uint64_t we = g->ew[r];
    for (int64_t j = g->ptr[a]; j < g->ptr[a + 1] && (int64_t)g->by_rank[j].rank < r; j++) {
        const int32_t c = g->by_rank[j].nbr;
        const int64_t rb = find_edge(g, b, c);
        if (rb >= 0 && offer(g, a, b, c, we, g->ew[g->by_rank[j].rank], g->ew[rb]) != DHL_OK)
            return DHL_ENOMEM;
    }
    for (int64_t j = g->ptr[b]; j < g->ptr[b + 1] && (int64_t)g->by_rank[j].rank < r; j++) {
        const int32_t c = g->by_rank[j].nbr;
        const int64_t ra = find_edge(g, a, c);
        /* (a, c) in S u H was listed by the loop over a's row */
        if (ra > r && offer(g, a, b, c, we, g->ew[ra], g->ew[g->by_rank[j].rank]) != DHL_OK)
            return DHL_ENOMEM;
    }
    return DHL_OK;
}

/* H -> S: triangles of e_r (r = h + 1) whose other two edges are in L (ranks > l) */
static int move_heavy_up(dhl_ctx* g, int64_t r, int64_t l) {
    int32_t x = g->ea[r], y = g->eb[r];
    const uint64_t we = g->ew[r];
    int64_t sx = g->ptr[x] + rank_prefix(g, x, l), sy = g->ptr[y] + rank_prefix(g, y, l);
    if (g->ptr[x + 1] - sx > g->ptr[y + 1] - sy) {
        int32_t t = x;
        x = y;
        y = t;
        sx = sy;
    }
    for (int64_t j = sx; j < g->ptr[x + 1]; j++) {
        const int32_t c = g->by_rank[j].nbr;
        const int64_t ry = find_edge(g, y, c);
        if (ry > l && offer(g, x, y, c, we, g->ew[g->by_rank[j].rank], g->ew[ry]) != DHL_OK)
            return DHL_ENOMEM;
    }
    return DHL_OK;
}

/* end of the run of equal weights that contains rank r */
static int64_t run_end(const dhl_ctx* g, int64_t r) {
    int64_t lo = r, hi = g->m; /* first rank > r with a smaller weight */
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (g->ew[mid] >= g->ew[r]) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

/* tau-decrease per unit of work of moving a pointer at rank r (Auto-HL) */
static double auto_rate(const dhl_ctx* g, int64_t r, double pw, double mult, double cost) {
    const int64_t e = run_end(g, r);
    const double w0 = (double)g->ew[r];
    const double w1 = e < g->m ? (double)g->ew[e] : 0.0;
    const double step = (w0 - w1) / (double)(e - r); /* average drop per edge of the run */
    return mult * (pow(w0, pw) - pow(w0 - step, pw)) / cost;
}

/*
 * Exact top-k by dynamic heavy-light.  alpha > 0: the DHL promotion rule with
 * that alpha_p; alpha <= 0: Auto-HL.  Outputs like the brute-force oracle
 * (first min(k, #triangles) in rank order).  stats (may be null), 6 words:
 * L->H moves, H->S moves, distinct triangles listed, edge probes, final h,
 * final l.
 */
int dhl_topk(int32_t n, int64_t m, const int32_t* u, const int32_t* v, const int32_t* w, int pcode,
             int64_t k, double alpha, int32_t* tri, uint64_t* key, double* value, int64_t* count,
             int64_t* stats) {
    *count = 0;
    if (n <= 0 || m < 0 || k <= 0 || pcode < 0 || pcode > 4 || m > (int64_t)UINT32_MAX)
        return DHL_EINVAL;
    dhl_ctx g;
    memset(&g, 0, sizeof(g));
    g.n = n;
    g.m = m;
    g.pcode = pcode;
    int rc = prepare(&g, u, v, w);
    if (rc == DHL_OK) rc = set_init(&g.set, 1u << 12);
    if (rc == DHL_OK) {
        g.heap.cap = k;
        g.heap.h = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)k);
        if (!g.heap.h) rc = DHL_ENOMEM;
    }
    const double pw = pcode == 2 ? 2.0 : 1.0;
    const int auto_hl = alpha <= 0 && (pcode == 1 || pcode == 2);
    if (alpha <= 0 && !auto_hl) alpha = 1.0;
    int64_t h = -1, l = -1, up_l = 0, up_h = 0;
    while (rc == DHL_OK && l + 1 < m) {
        const uint64_t ub = dhl_key(pcode, W(&g, h + 1), W(&g, l + 1), W(&g, l + 2));
        if (g.heap.size == k && g.heap.h[0] > ub) break;
        int light;
        if (h == l) {
            light = 1;
        } else if (auto_hl) {
            const int32_t la = g.ea[l + 1], lb = g.eb[l + 1], ha = g.ea[h + 1], hb = g.eb[h + 1];
            const double cost_l = 1.0 + (double)(rank_prefix(&g, la, l) + rank_prefix(&g, lb, l));
            const double cost_h = 1.0 + (double)((g.ptr[ha + 1] - g.ptr[ha] - rank_prefix(&g, ha, l)) +
                                                 (g.ptr[hb + 1] - g.ptr[hb] - rank_prefix(&g, hb, l)));
            light = auto_rate(&g, l + 1, pw, 2.0, cost_l) >= auto_rate(&g, h + 1, pw, 1.0, cost_h);
        } else {
            light = pow((double)W(&g, l + 1), alpha) > (double)W(&g, h + 1);
        }
        if (light) {
            rc = move_light_up(&g, l + 1);
            l++;
            up_l++;
        } else {
            rc = move_heavy_up(&g, h + 1, l);
            h++;
            up_h++;
        }
    }
    if (rc == DHL_OK) {
        const uint64_t kth = g.heap.size == k ? g.heap.h[0] : 0u;
        int64_t nc = 0;
        for (uint64_t i = 0; i < g.set.cap; i++)
            if (g.set.slot[i].t[0] >= 0 && g.set.slot[i].key >= kth) nc++;
        dhl_tri* out = (dhl_tri*)malloc(sizeof(dhl_tri) * (size_t)(nc ? nc : 1));
        if (!out) {
            rc = DHL_ENOMEM;
        } else {
            int64_t j = 0;
            for (uint64_t i = 0; i < g.set.cap; i++)
                if (g.set.slot[i].t[0] >= 0 && g.set.slot[i].key >= kth) out[j++] = g.set.slot[i];
            qsort(out, (size_t)nc, sizeof(dhl_tri), cmp_out);
            const int64_t c = nc < k ? nc : k;
            for (int64_t i = 0; i < c; i++) {
                tri[3 * i] = out[i].t[0];
                tri[3 * i + 1] = out[i].t[1];
                tri[3 * i + 2] = out[i].t[2];
                key[i] = out[i].key;
                value[i] = dhl_value(pcode, out[i].key);
            }
            *count = c;
            free(out);
        }
    }
    if (stats) {
        stats[0] = up_l;
        stats[1] = up_h;
        stats[2] = (int64_t)g.set.size;
        stats[3] = g.probes;
        stats[4] = h;
        stats[5] = l;
    }
    release(&g);
    return rc;
}

/* alpha_p = 2 - p / (p - 1 + beta) for power-law weights of exponent beta
 * (Section 3.3); 1 at p = +-inf, 2 at p = 0. */
double dhl_alpha(int pcode, double beta) {
    if (pcode == 0 || pcode == 3) return 1.0;
    const double p = pcode == 2 ? 2.0 : (pcode == 4 ? 0.0 : 1.0);
    return 2.0 - p / (p - 1.0 + beta);
}
