/*
 * CPU oracle for subgraph-isomorphism enumeration (Delta-Motif, arXiv 2508.21287).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path may link, load or call this
 * file; the tests, the smoke check and the benchmark's CPU-baseline leg use it to check
 * the CUDA path. It shares no code, header, table or helper with the CUDA library.
 *
 * What it computes is the plain definition of the result, not the paper's method:
 *   Emb(G_p, G_d) = all injective maps f : V_p -> V_d such that every pattern edge
 *   {u, v} maps to a data edge {f(u), f(v)}                       (Sec. 3.1, Preliminaries)
 * Graphs are undirected, simple and connected (Sec. 3.1). The paper's method (Alg. 1 with
 * the overlap filter of Sec. 3.2) only enforces edges that the motif slices cover plus
 * distinctness of the mapped vertices, so the set it reaches is the non-induced one
 * (monomorphisms); `induced` = 1 adds the non-edge condition of the literal "iff" reading.
 *
 * Two independent enumerators:
 *   or_enumerate   - backtracking over a BFS order of the pattern, candidates from the
 *                    data-graph neighbour lists, edge tests by binary search in CSR.
 *   or_brute_force - every injective map by nested enumeration, edges tested at the leaf
 *                    against a dense adjacency matrix. Only for tiny inputs.
 * Rows are (f(0), ..., f(n_p - 1)) indexed by pattern vertex id, sorted ascending
 * lexicographically, without duplicates.
 *
 * Checksum of a row set: sum over rows of H(row) mod 2^64 where
 *   H(row) = mix64(n_p + sum_{j=0}^{n_p-1} mix64(((j + 1) << 32) | (uint32)f(j)))   (mod 2^64)
 * and mix64 is the SplitMix64 output finaliser (Steele, Lea, Flood 2014). Each term binds a
 * vertex id to its pattern position, so H depends on every position; neither H's inner sum
 * nor the outer sum depends on order. (The paper has no checksum; this is the library's own
 * definition.)
 *
 * Score of a row (layout fidelity, Sec. 5.4): sum over pattern edges {u, v} of the edge
 * error w_e(f(u), f(v)) plus sum over pattern vertices of the vertex error w_q(f(u)),
 * accumulated in FP64. This is the log-domain form of the paper's product of fidelities;
 * lower is better. or_scores_directed is the direction-aware form (per-direction device
 * costs, per-direction pattern weights) of the same sum.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t n;
    const int32_t *rp, *ci;
} csr_t;

/* ---------------------------------------------------------------- checksum -------- */

static uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

uint64_t or_mix64(uint64_t z) { return mix64(z); }

uint64_t or_row_hash(const int32_t *row, int32_t n) {
    uint64_t s = (uint64_t)(uint32_t)n;
    for (int32_t j = 0; j < n; j++) s += mix64(((uint64_t)(uint32_t)(j + 1) << 32) | (uint64_t)(uint32_t)row[j]);
    return mix64(s);
}

uint64_t or_checksum(const int32_t *rows, int64_t nrows, int32_t n) {
    uint64_t s = 0;
    for (int64_t r = 0; r < nrows; r++) s += or_row_hash(rows + r * n, n);
    return s;
}

/* ---------------------------------------------------------------- row buffer ------ */

typedef struct {
    int32_t *a;
    int64_t len, cap; /* in int32 elements */
    int64_t count;
    uint64_t checksum;
    int store;
    int oom;
} rowbuf_t;

static void rb_push(rowbuf_t *b, const int32_t *row, int32_t n) {
    b->count++;
    b->checksum += or_row_hash(row, n);
    if (!b->store || b->oom) return;
    if (b->len + n > b->cap) {
        int64_t nc = b->cap ? 2 * b->cap : 1024;
        while (nc < b->len + n) nc *= 2;
        int32_t *na = (int32_t *)realloc(b->a, (size_t)nc * sizeof(int32_t));
        if (!na) {
            b->oom = 1;
            return;
        }
        b->a = na;
        b->cap = nc;
    }
    memcpy(b->a + b->len, row, (size_t)n * sizeof(int32_t));
    b->len += n;
}

static int32_t g_sort_n; /* row width for the comparator (set before each qsort) */

static int cmp_rows(const void *x, const void *y) {
    const int32_t *a = (const int32_t *)x, *b = (const int32_t *)y;
    for (int32_t j = 0; j < g_sort_n; j++) {
        if (a[j] != b[j]) return a[j] < b[j] ? -1 : 1;
    }
    return 0;
}

static pthread_mutex_t g_sort_lock = PTHREAD_MUTEX_INITIALIZER;

static void sort_rows(int32_t *rows, int64_t nrows, int32_t n) {
    pthread_mutex_lock(&g_sort_lock);
    g_sort_n = n;
    qsort(rows, (size_t)nrows, (size_t)n * sizeof(int32_t), cmp_rows);
    pthread_mutex_unlock(&g_sort_lock);
}

/* ---------------------------------------------------------------- graph helpers --- */

static int csr_adjacent(const csr_t *g, int32_t u, int32_t v) {
    int32_t lo = g->rp[u], hi = g->rp[u + 1];
    while (lo < hi) {
        int32_t mid = lo + (hi - lo) / 2;
        int32_t x = g->ci[mid];
        if (x == v) return 1;
        if (x < v) lo = mid + 1;
        else hi = mid;
    }
    return 0;
}

/* ---------------------------------------------------------------- backtracking ---- */

#define OR_MAXP 128

typedef struct {
    const csr_t *d, *p;
    int induced;
    int32_t np;
    int32_t order[OR_MAXP];     /* pi: position -> pattern vertex */
    int32_t parent[OR_MAXP];    /* pattern vertex of the BFS parent, -1 for pi[0] */
    int32_t nbk[OR_MAXP];       /* number of earlier pattern neighbours of pi[i] */
    int32_t nb[OR_MAXP][OR_MAXP];
    int32_t nnk[OR_MAXP];       /* earlier non-neighbours (induced only) */
    int32_t nn[OR_MAXP][OR_MAXP];
} search_t;

typedef struct {
    const search_t *s;
    int32_t f[OR_MAXP];
    unsigned char *used;
    rowbuf_t out;
} worker_t;

static void bt(worker_t *w, int32_t i) {
    const search_t *s = w->s;
    if (i == s->np) {
        rb_push(&w->out, w->f, s->np);
        return;
    }
    int32_t u = s->order[i];
    int32_t pv = w->f[s->parent[u]];
    for (int32_t k = s->d->rp[pv]; k < s->d->rp[pv + 1]; k++) {
        int32_t v = s->d->ci[k];
        if (w->used[v]) continue;
        int ok = 1;
        for (int32_t t = 0; t < s->nbk[i] && ok; t++)
            ok = csr_adjacent(s->d, w->f[s->nb[i][t]], v);
        for (int32_t t = 0; t < s->nnk[i] && ok; t++)
            ok = !csr_adjacent(s->d, w->f[s->nn[i][t]], v);
        if (!ok) continue;
        w->used[v] = 1;
        w->f[u] = v;
        bt(w, i + 1);
        w->used[v] = 0;
    }
}

/* BFS order of the pattern from the lowest-id vertex of maximum degree; neighbours are
 * visited in increasing id. Returns 0, or -2 if the pattern is not connected. */
static int make_order(search_t *s) {
    const csr_t *p = s->p;
    int32_t np = p->n, best = 0;
    for (int32_t u = 1; u < np; u++)
        if (p->rp[u + 1] - p->rp[u] > p->rp[best + 1] - p->rp[best]) best = u;
    int32_t pos[OR_MAXP];
    for (int32_t u = 0; u < np; u++) pos[u] = -1;
    int32_t head = 0, tail = 0;
    s->order[tail++] = best;
    pos[best] = 0;
    s->parent[best] = -1;
    while (head < tail) {
        int32_t u = s->order[head++];
        for (int32_t k = p->rp[u]; k < p->rp[u + 1]; k++) {
            int32_t v = p->ci[k];
            if (pos[v] < 0) {
                pos[v] = tail;
                s->parent[v] = u;
                s->order[tail++] = v;
            }
        }
    }
    if (tail != np) return -2;
    for (int32_t i = 0; i < np; i++) {
        int32_t u = s->order[i];
        s->nbk[i] = 0;
        s->nnk[i] = 0;
        for (int32_t j = 0; j < i; j++) {
            int32_t q = s->order[j];
            int adj = 0;
            for (int32_t k = p->rp[u]; k < p->rp[u + 1]; k++) adj |= (p->ci[k] == q);
            if (adj) {
                if (q != s->parent[u]) s->nb[i][s->nbk[i]++] = q;
            } else if (s->induced) {
                s->nn[i][s->nnk[i]++] = q;
            }
        }
    }
    return 0;
}

typedef struct {
    worker_t w;
    int32_t tid, nthreads;
} thread_arg_t;

static void *thread_main(void *arg) {
    thread_arg_t *ta = (thread_arg_t *)arg;
    worker_t *w = &ta->w;
    const search_t *s = w->s;
    int32_t u0 = s->order[0];
    for (int32_t v = ta->tid; v < s->d->n; v += ta->nthreads) {
        w->f[u0] = v;
        w->used[v] = 1;
        if (s->np == 1) rb_push(&w->out, w->f, 1);
        else bt(w, 1);
        w->used[v] = 0;
    }
    return NULL;
}

/*
 * Enumerate Emb(G_p, G_d). Returns the count (>= 0), or -1 (bad argument), -2 (pattern
 * not connected), -3 (out of host memory). With out_rows non-NULL the sorted rows are
 * returned in a malloc'd buffer (free with or_free). n_threads > 1 splits the candidates
 * of the first pattern vertex over POSIX threads.
 */
int64_t or_enumerate(int32_t nd, const int32_t *rp_d, const int32_t *ci_d, int32_t np,
                     const int32_t *rp_p, const int32_t *ci_p, int32_t induced,
                     int32_t n_threads, int32_t **out_rows, uint64_t *out_checksum) {
    if (np < 1 || np > OR_MAXP || nd < 0) return -1;
    csr_t d = {nd, rp_d, ci_d}, p = {np, rp_p, ci_p};
    search_t *s = (search_t *)calloc(1, sizeof(search_t));
    if (!s) return -3;
    s->d = &d;
    s->p = &p;
    s->np = np;
    s->induced = induced;
    if (make_order(s) != 0) {
        free(s);
        return -2;
    }
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    thread_arg_t *ta = (thread_arg_t *)calloc((size_t)n_threads, sizeof(thread_arg_t));
    pthread_t *th = (pthread_t *)calloc((size_t)n_threads, sizeof(pthread_t));
    int64_t rc = 0;
    if (!ta || !th) rc = -3;
    for (int32_t t = 0; t < n_threads && rc == 0; t++) {
        ta[t].tid = t;
        ta[t].nthreads = n_threads;
        ta[t].w.s = s;
        ta[t].w.used = (unsigned char *)calloc((size_t)(nd > 0 ? nd : 1), 1);
        ta[t].w.out.store = out_rows != NULL;
        if (!ta[t].w.used) rc = -3;
    }
    if (rc == 0) {
        if (n_threads == 1) {
            thread_main(&ta[0]);
        } else {
            for (int32_t t = 0; t < n_threads; t++) pthread_create(&th[t], NULL, thread_main, &ta[t]);
            for (int32_t t = 0; t < n_threads; t++) pthread_join(th[t], NULL);
        }
        int64_t count = 0;
        uint64_t cs = 0;
        int64_t total_len = 0;
        for (int32_t t = 0; t < n_threads; t++) {
            count += ta[t].w.out.count;
            cs += ta[t].w.out.checksum;
            total_len += ta[t].w.out.len;
            if (ta[t].w.out.oom) rc = -3;
        }
        if (rc == 0 && out_rows) {
            int32_t *all = (int32_t *)malloc((size_t)(total_len > 0 ? total_len : 1) * sizeof(int32_t));
            if (!all) {
                rc = -3;
            } else {
                int64_t off = 0;
                for (int32_t t = 0; t < n_threads; t++) {
                    if (ta[t].w.out.len)
                        memcpy(all + off, ta[t].w.out.a, (size_t)ta[t].w.out.len * sizeof(int32_t));
                    off += ta[t].w.out.len;
                }
                sort_rows(all, count, np);
                *out_rows = all;
            }
        }
        if (out_checksum) *out_checksum = cs;
        if (rc == 0) rc = count;
    }
    for (int32_t t = 0; ta && t < n_threads; t++) {
        free(ta[t].w.used);
        free(ta[t].w.out.a);
    }
    free(ta);
    free(th);
    free(s);
    return rc;
}

void or_free(void *p) { free(p); }

/* ---------------------------------------------------------------- brute force ----- */

typedef struct {
    int32_t nd, np;
    const unsigned char *dadj; /* nd x nd dense adjacency */
    const unsigned char *padj; /* np x np dense adjacency */
    int induced;
    int32_t f[OR_MAXP];
    unsigned char *used;
    rowbuf_t out;
} brute_t;

static void brute_rec(brute_t *b, int32_t i) {
    if (i == b->np) {
        for (int32_t u = 0; u < b->np; u++)
            for (int32_t v = u + 1; v < b->np; v++) {
                int pe = b->padj[u * b->np + v];
                int de = b->dadj[(int64_t)b->f[u] * b->nd + b->f[v]];
                if (pe && !de) return;
                if (b->induced && !pe && de) return;
            }
        rb_push(&b->out, b->f, b->np);
        return;
    }
    for (int32_t v = 0; v < b->nd; v++) {
        if (b->used[v]) continue;
        b->used[v] = 1;
        b->f[i] = v;
        brute_rec(b, i + 1);
        b->used[v] = 0;
    }
}

/* Every injective map V_p -> V_d, kept when it preserves all pattern edges. Leaves are
 * visited in lexicographic order, so the rows come out sorted. Same return convention as
 * or_enumerate. Cost nd!/(nd-np)! leaves: tiny inputs only. */
int64_t or_brute_force(int32_t nd, const int32_t *rp_d, const int32_t *ci_d, int32_t np,
                       const int32_t *rp_p, const int32_t *ci_p, int32_t induced,
                       int32_t **out_rows, uint64_t *out_checksum) {
    if (np < 1 || np > OR_MAXP || nd < 0) return -1;
    brute_t b;
    memset(&b, 0, sizeof(b));
    b.nd = nd;
    b.np = np;
    b.induced = induced;
    unsigned char *dadj = (unsigned char *)calloc((size_t)(nd > 0 ? nd : 1) * (size_t)(nd > 0 ? nd : 1), 1);
    unsigned char *padj = (unsigned char *)calloc((size_t)np * (size_t)np, 1);
    b.used = (unsigned char *)calloc((size_t)(nd > 0 ? nd : 1), 1);
    if (!dadj || !padj || !b.used) {
        free(dadj);
        free(padj);
        free(b.used);
        return -3;
    }
    for (int32_t u = 0; u < nd; u++)
        for (int32_t k = rp_d[u]; k < rp_d[u + 1]; k++) dadj[(int64_t)u * nd + ci_d[k]] = 1;
    for (int32_t u = 0; u < np; u++)
        for (int32_t k = rp_p[u]; k < rp_p[u + 1]; k++) padj[u * np + ci_p[k]] = 1;
    b.dadj = dadj;
    b.padj = padj;
    b.out.store = out_rows != NULL;
    brute_rec(&b, 0);
    int64_t rc = b.out.oom ? -3 : b.out.count;
    if (rc >= 0 && out_rows) *out_rows = b.out.a;
    else free(b.out.a);
    if (out_checksum) *out_checksum = b.out.checksum;
    free(dadj);
    free(padj);
    free(b.used);
    return rc;
}

/* ---------------------------------------------------------------- scores, top-k --- */

static double edge_weight(const csr_t *d, const float *edge_err, int32_t u, int32_t v, int *found) {
    int32_t lo = d->rp[u], hi = d->rp[u + 1];
    while (lo < hi) {
        int32_t mid = lo + (hi - lo) / 2;
        if (d->ci[mid] == v) {
            *found = 1;
            return (double)edge_err[mid];
        }
        if (d->ci[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    *found = 0;
    return 0.0;
}

/* FP64 layout score of each row: sum of w_e over pattern edges {u < v} in CSR order of the
 * pattern, then sum of w_q over pattern vertices 0..n_p-1 (w_q = 0 when qubit_err is
 * NULL). Returns 0, or -1 if some row maps a pattern edge to a non-edge. */
/* Per-row layout score. form 0: sum of the error rates e; form 1: sum of -log(1 - e), the
 * negative log of the product of the fidelities 1 - e (Sec. 5.4 ranks layouts by that product). */
static double score_term(double e, int32_t form) { return form ? -log1p(-e) : e; }

int32_t or_scores(int32_t nd, const int32_t *rp_d, const int32_t *ci_d, const float *edge_err,
                  const float *qubit_err, int32_t np, const int32_t *rp_p, const int32_t *ci_p,
                  const int32_t *rows, int64_t nrows, int32_t form, double *out) {
    csr_t d = {nd, rp_d, ci_d};
    for (int64_t r = 0; r < nrows; r++) {
        const int32_t *f = rows + r * np;
        double s = 0.0;
        for (int32_t u = 0; u < np; u++)
            for (int32_t k = rp_p[u]; k < rp_p[u + 1]; k++) {
                int32_t v = ci_p[k];
                if (u < v) {
                    int found;
                    double e = edge_weight(&d, edge_err, f[u], f[v], &found);
                    if (!found) return -1;
                    s += score_term(e, form);
                }
            }
        if (qubit_err)
            for (int32_t u = 0; u < np; u++) s += score_term((double)qubit_err[f[u]], form);
        out[r] = s;
    }
    return 0;
}

/* Direction-aware score of each row (the post-processing of Sec. 5.4's footnote: layouts are
 * enumerated on the undirected coupling graph, and a two-qubit gate whose control and target
 * land on a device edge is costed in the direction it runs there):
 *   score(f) = sum over pattern slots p -> q (every ordered pair with {p, q} in E_p) of
 *              w_dir[slot] * e_dir(f(p) -> f(q))
 *            + sum over pattern vertices u of qubit_err[f(u)]   (when given)
 * where w_dir is aligned with the pattern's col_idx (the number of gates run from p to q, or
 * any weight) and e_dir with the data graph's col_idx (the cost of a gate from the row's
 * vertex to the column's vertex; not symmetric in general). FP64. Returns -1 when a row maps
 * a pattern edge onto a non-edge. */
int32_t or_scores_directed(int32_t nd, const int32_t *rp_d, const int32_t *ci_d, const float *e_dir,
                           const float *qubit_err, int32_t np, const int32_t *rp_p, const int32_t *ci_p,
                           const float *w_dir, const int32_t *rows, int64_t nrows, double *out) {
    csr_t d = {nd, rp_d, ci_d};
    for (int64_t r = 0; r < nrows; r++) {
        const int32_t *f = rows + r * np;
        double s = 0.0;
        for (int32_t p = 0; p < np; p++)
            for (int32_t k = rp_p[p]; k < rp_p[p + 1]; k++) {
                int found;
                double e = edge_weight(&d, e_dir, f[p], f[ci_p[k]], &found);
                if (!found) return -1;
                s += (double)w_dir[k] * e;
            }
        if (qubit_err)
            for (int32_t u = 0; u < np; u++) s += (double)qubit_err[f[u]];
        out[r] = s;
    }
    return 0;
}

static const double *g_tk_scores;
static const int32_t *g_tk_rows;
static int32_t g_tk_n;
static pthread_mutex_t g_tk_lock = PTHREAD_MUTEX_INITIALIZER;

static int cmp_score_row(const void *x, const void *y) {
    int64_t a = *(const int64_t *)x, b = *(const int64_t *)y;
    double sa = g_tk_scores[a], sb = g_tk_scores[b];
    if (sa != sb) return sa < sb ? -1 : 1;
    const int32_t *ra = g_tk_rows + a * g_tk_n, *rb = g_tk_rows + b * g_tk_n;
    for (int32_t j = 0; j < g_tk_n; j++)
        if (ra[j] != rb[j]) return ra[j] < rb[j] ? -1 : 1;
    return 0;
}

/* Indices of the min(k, nrows) rows with the smallest (score, row) key, in that order. */
int64_t or_topk(const int32_t *rows, const double *scores, int64_t nrows, int32_t n, int64_t k,
                int64_t *out_idx) {
    int64_t *idx = (int64_t *)malloc((size_t)(nrows > 0 ? nrows : 1) * sizeof(int64_t));
    if (!idx) return -3;
    for (int64_t i = 0; i < nrows; i++) idx[i] = i;
    pthread_mutex_lock(&g_tk_lock);
    g_tk_scores = scores;
    g_tk_rows = rows;
    g_tk_n = n;
    qsort(idx, (size_t)nrows, sizeof(int64_t), cmp_score_row);
    pthread_mutex_unlock(&g_tk_lock);
    int64_t m = k < nrows ? k : nrows;
    memcpy(out_idx, idx, (size_t)m * sizeof(int64_t));
    free(idx);
    return m;
}
