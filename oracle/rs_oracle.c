/*
 * rs_oracle.c -- CPU oracle for Robust Spanning Index (RSI) scoring.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and
 * bench.py's cpu_baseline / reference leg may load this code.  It shares no
 * code with the CUDA library.
 *
 * It is the plain definition of the score, evaluated slowly in fp64:
 *
 *   L(u,v)  = {(C(x), freq) : x in N(v), C(x) != C(u)}              (Eq. cont)
 *   H(L)    = -sum p log2 p,  p = f_j / sum_{l != C(u)} f_l         (Eq. entropy)
 *   w_v(u)  = H(L(u,v)) * |L(u,v)|                                  (Eq. weight)
 *   R(u)    = 1/(d(u)(d(u)-1)) * sum_{w in N(u), v in N(w) : 1(u,w,v)}
 *             (w_v(u) w_w(v) w_w(u))^(1/3)  with weights / w_max     (Eq. RSI)
 *   1(u,w,v)= [(u,w,v) is a triad] [C(v) != C(w)] [C(u) != C(w)]    (indicator)
 *
 * Readings of points the paper leaves open:
 *   - log base 2 (the worked example of Sec. V-B gives H = 1 for counts {1,1}
 *     and w_max = 4.754 = 3 log2 3);
 *   - a triad (u,w,v) needs the real edges u-w and w-v and v != u; it is valid
 *     when v is adjacent to u or C(v) = C(u) (Type-I closed triad / Type-II
 *     augmented edge, Sec. III-A; a closed triangle with C(v) = C(u) counts once);
 *   - ordered pairs (w,v): a Type-I triangle counts twice at each apex (the
 *     worked example of Sec. V-B lists (u,v1,w) and (u,w,v1));
 *   - |L| is the number of distinct communities in L (Eq. weight), and a
 *     weight with |L| < 2 is 0 (Alg. 1 Step 2 keeps only |L| > 1); an option
 *     takes Alg. 2's |L| = L_all - 1 for every column instead;
 *   - w_max is the largest w_v(c) over every node v and every community
 *     c in [0,k) (Alg. 1 Step 2 / normalize_weights), so it includes the
 *     value for communities absent from N(v);
 *   - R(u) = 0 when d(u) < 2 or w_max = 0.
 *
 * Numerics: every entropy term is positive and evaluated as
 * (f/Y) log2(Y/f), with log1p((Y-f)/f)/ln 2 when 2f > Y (no cancellation);
 * sums use Neumaier compensation.  Relative error is a few ulps.
 *
 * Threads (OpenMP, rso_set_threads): nodes are shared out over threads, and
 * each node's table, weights and score sum are computed by one thread in the
 * same order as with one thread, so results are bit-identical for any thread
 * count; w_max is a max, which does not depend on the order either.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int64_t n;
    int32_t k;
    int alg2;          /* weights with |L| = L_all - 1 for every column (Alg. 2) */
    int64_t *off;      /* n+1 */
    int32_t *col;      /* nnz */
    int32_t *lab;      /* n */
    /* per-node community table, sorted by community id */
    int64_t *tptr;     /* n+1 */
    int32_t *tcomm;    /* t */
    int32_t *tcnt;     /* t */
    double *tw;        /* t: w_v(c) for the table's community c */
    double *wabs;      /* n: w_v(c) for any c absent from N(v) */
    double wmax;
    char err[200];
} rso_graph;

/* ---- compensated summation (Neumaier) ----------------------------------- */
typedef struct { double s, c; } ksum;
static void kadd(ksum *a, double x) {
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
    a->s = t;
}
static double kval(const ksum *a) { return a->s + a->c; }

/* ---- validation ----------------------------------------------------------- */
static int has_edge(const int64_t *off, const int32_t *col, int32_t a, int32_t b) {
    int64_t lo = off[a], hi = off[a + 1];
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (col[mid] < b) lo = mid + 1; else hi = mid;
    }
    return lo < off[a + 1] && col[lo] == b;
}

static int validate(rso_graph *g) {
    if (g->off[0] != 0) { snprintf(g->err, sizeof g->err, "offsets[0] != 0"); return -1; }
    for (int64_t v = 0; v < g->n; ++v) {
        if (g->lab[v] < 0 || g->lab[v] >= g->k) {
            snprintf(g->err, sizeof g->err, "label of node %lld out of [0,k)", (long long)v);
            return -1;
        }
        if (g->off[v + 1] < g->off[v]) { snprintf(g->err, sizeof g->err, "offsets decrease"); return -1; }
        for (int64_t e = g->off[v]; e < g->off[v + 1]; ++e) {
            int32_t x = g->col[e];
            if (x < 0 || x >= g->n) { snprintf(g->err, sizeof g->err, "column out of range"); return -1; }
            if (x == v) { snprintf(g->err, sizeof g->err, "self-loop at %lld", (long long)v); return -1; }
            if (e > g->off[v] && g->col[e - 1] >= x) {
                snprintf(g->err, sizeof g->err, "row %lld not strictly ascending", (long long)v);
                return -1;
            }
        }
    }
    for (int64_t v = 0; v < g->n; ++v)
        for (int64_t e = g->off[v]; e < g->off[v + 1]; ++e)
            if (!has_edge(g->off, g->col, g->col[e], (int32_t)v)) {
                snprintf(g->err, sizeof g->err, "asymmetric edge %lld-%d", (long long)v, g->col[e]);
                return -1;
            }
    return 0;
}

/* ---- entropy and weight by definition ------------------------------------ */

/* H of the count multiset cnt[0..m) with one copy of the value `skip` left out
   (skip < 0: nothing left out).  cnt must be sorted ascending so that equal
   multisets are summed in the same order.  Returns w = H * |L|, or 0 if |L| < 2,
   where |L| is the number of entries left (Eq. weight), or m - 1 for every
   column when alg2 is set (the convention of Alg. 2, compute_weights). */
static double weight_of_counts(const int32_t *cnt, int m, int32_t skip, int alg2) {
    int L = m - ((skip >= 0 || alg2) ? 1 : 0);     /* alg2: |L| = L_all - 1 for every column */
    if (L < 2) return 0.0;
    double Y = 0.0;
    int skipped = 0;
    for (int i = 0; i < m; ++i) {
        if (!skipped && cnt[i] == skip) { skipped = 1; continue; }
        Y += cnt[i];
    }
    ksum h = {0.0, 0.0};
    skipped = 0;
    for (int i = 0; i < m; ++i) {
        if (!skipped && cnt[i] == skip) { skipped = 1; continue; }
        double f = cnt[i];
        double lg = (2.0 * f > Y) ? log1p((Y - f) / f) / M_LN2 : log2(Y / f);
        kadd(&h, (f / Y) * lg);
    }
    return kval(&h) * (double)L;
}

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* the counts of row v's neighbour labels, sorted: buf[0, d) */
static int64_t sorted_labels(const rso_graph *g, int64_t v, int32_t *buf) {
    int64_t d = g->off[v + 1] - g->off[v];
    for (int64_t i = 0; i < d; ++i) buf[i] = g->lab[g->col[g->off[v] + i]];
    qsort(buf, (size_t)d, sizeof(int32_t), cmp_i32);
    return d;
}

static int build_tables(rso_graph *g) {
    int64_t n = g->n;
    int64_t dmax = 0;
    for (int64_t v = 0; v < n; ++v) {
        int64_t d = g->off[v + 1] - g->off[v];
        if (d > dmax) dmax = d;
    }
    g->tptr = (int64_t *)malloc((size_t)(n + 1) * sizeof(int64_t));
    g->wabs = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    if (!g->tptr || !g->wabs) return -1;
    int fail = 0;
    /* pass 1: table sizes (row v's distinct labels into tptr[v + 1]) */
    g->tptr[0] = 0;
#pragma omp parallel reduction(|:fail)
    {
        int32_t *buf = (int32_t *)malloc((size_t)(dmax + 1) * sizeof(int32_t));
        if (!buf) fail = 1;
#pragma omp for schedule(dynamic, 1024)
        for (int64_t v = 0; v < n; ++v) {
            if (!buf) continue;
            int64_t d = sorted_labels(g, v, buf), t = 0;
            for (int64_t i = 0; i < d; ++i) if (i == 0 || buf[i] != buf[i - 1]) t++;
            g->tptr[v + 1] = t;
        }
        free(buf);
    }
    if (fail) return -1;
    for (int64_t v = 0; v < n; ++v) g->tptr[v + 1] += g->tptr[v];
    int64_t T = g->tptr[n];
    g->tcomm = (int32_t *)malloc((size_t)(T > 0 ? T : 1) * sizeof(int32_t));
    g->tcnt = (int32_t *)malloc((size_t)(T > 0 ? T : 1) * sizeof(int32_t));
    g->tw = (double *)malloc((size_t)(T > 0 ? T : 1) * sizeof(double));
    if (!g->tcomm || !g->tcnt || !g->tw) return -1;
    /* pass 2: counts f_v(c), then weights */
    double wmax = 0.0;
#pragma omp parallel reduction(|:fail) reduction(max:wmax)
    {
        int32_t *buf = (int32_t *)malloc((size_t)(dmax + 1) * sizeof(int32_t));
        int32_t *cs = (int32_t *)malloc((size_t)(dmax + 1) * sizeof(int32_t));
        int32_t *dist = (int32_t *)malloc((size_t)(dmax + 1) * sizeof(int32_t));
        double *dw = (double *)malloc((size_t)(dmax + 1) * sizeof(double));
        if (!buf || !cs || !dist || !dw) fail = 1;
#pragma omp for schedule(dynamic, 1024)
        for (int64_t v = 0; v < n; ++v) {
            if (!buf || !cs || !dist || !dw) continue;
            int64_t d = sorted_labels(g, v, buf);
            int64_t p = g->tptr[v];
            for (int64_t i = 0; i < d; ++i) {
                if (i == 0 || buf[i] != buf[i - 1]) { g->tcomm[p] = buf[i]; g->tcnt[p] = 0; p++; }
                g->tcnt[p - 1]++;
            }
            int m = (int)(g->tptr[v + 1] - g->tptr[v]);
            for (int i = 0; i < m; ++i) cs[i] = g->tcnt[g->tptr[v] + i];
            qsort(cs, (size_t)m, sizeof(int32_t), cmp_i32);
            /* w_v(c) depends on c only through f_v(c): the multiset left after
               removing one copy of f_v(c) is the same for equal counts */
            int nd = 0;
            for (int i = 0; i < m; ++i)
                if (i == 0 || cs[i] != cs[i - 1]) { dist[nd] = cs[i]; dw[nd] = weight_of_counts(cs, m, cs[i], g->alg2); nd++; }
            for (int i = 0; i < m; ++i) {
                int32_t f = g->tcnt[g->tptr[v] + i];
                int lo = 0, hi = nd - 1;
                while (lo < hi) { int mid = (lo + hi) / 2; if (dist[mid] < f) lo = mid + 1; else hi = mid; }
                double w = dw[lo];
                g->tw[g->tptr[v] + i] = w;
                if (w > wmax) wmax = w;
            }
            g->wabs[v] = weight_of_counts(cs, m, -1, g->alg2);
            if (m < g->k && g->wabs[v] > wmax) wmax = g->wabs[v];
        }
        free(buf); free(cs); free(dist); free(dw);
    }
    g->wmax = wmax;
    return fail ? -1 : 0;
}

/* w_v(c) for any community c */
static double omega(const rso_graph *g, int32_t v, int32_t c) {
    int64_t lo = g->tptr[v], hi = g->tptr[v + 1];
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (g->tcomm[mid] < c) lo = mid + 1; else hi = mid;
    }
    if (lo < g->tptr[v + 1] && g->tcomm[lo] == c) return g->tw[lo];
    return g->wabs[v];
}

/* ---- score assembly -------------------------------------------------------- */

/* one weighted triad: geometric mean of its three weights */
double rso_triad_term(double w_vu, double w_wv, double w_wu) { return cbrt(w_vu * w_wv * w_wu); }

/* R(u) from the summed triad terms of un-normalised weights */
double rso_finish(double sum, int64_t d, double wmax) {
    if (d < 2 || wmax <= 0.0) return 0.0;
    return sum / wmax / ((double)d * (double)(d - 1));
}

static double score_sum(const rso_graph *g, int32_t u, int strict) {
    int32_t cu = g->lab[u];
    ksum s = {0.0, 0.0};
    for (int64_t a = g->off[u]; a < g->off[u + 1]; ++a) {
        int32_t w = g->col[a];
        int32_t cw = g->lab[w];
        if (cw == cu) continue;                          /* C(u) != C(w) */
        for (int64_t b = g->off[w]; b < g->off[w + 1]; ++b) {
            int32_t v = g->col[b];
            if (v == u) continue;                        /* a triad has three nodes */
            int32_t cv = g->lab[v];
            if (cv == cw) continue;                      /* C(v) != C(w) */
            int closed = has_edge(g->off, g->col, u, v);
            int triad;
            if (closed) triad = (cv != cu) || !strict;   /* Type-I (all distinct) */
            else triad = (cv == cu);                     /* Type-II augmented edge */
            if (!triad) continue;
            kadd(&s, rso_triad_term(omega(g, v, cu), omega(g, w, cv), omega(g, w, cu)));
        }
    }
    return kval(&s);
}

/* ---- exported API ------------------------------------------------------------ */

rso_graph *rso_new(int64_t n, int32_t k, const int64_t *off, const int32_t *col, const int32_t *lab,
                   int do_validate, int alg2, char *err, int errlen) {
    rso_graph *g = (rso_graph *)calloc(1, sizeof(rso_graph));
    if (!g) return NULL;
    g->n = n; g->k = k; g->alg2 = alg2 ? 1 : 0;
    int64_t nnz = off[n];
    g->off = (int64_t *)malloc((size_t)(n + 1) * sizeof(int64_t));
    g->col = (int32_t *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int32_t));
    g->lab = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    int rc = (!g->off || !g->col || !g->lab) ? -1 : 0;
    if (rc == 0) {
        memcpy(g->off, off, (size_t)(n + 1) * sizeof(int64_t));
        if (nnz) memcpy(g->col, col, (size_t)nnz * sizeof(int32_t));
        if (n) memcpy(g->lab, lab, (size_t)n * sizeof(int32_t));
        if (k < 1) { snprintf(g->err, sizeof g->err, "k < 1"); rc = -1; }
    }
    if (rc == 0 && do_validate) rc = validate(g);
    if (rc == 0 && build_tables(g)) { snprintf(g->err, sizeof g->err, "out of memory"); rc = -1; }
    if (rc) {
        if (err && errlen > 0) snprintf(err, (size_t)errlen, "%s", g->err);
        extern void rso_free(rso_graph *);
        rso_free(g);
        return NULL;
    }
    return g;
}

void rso_free(rso_graph *g) {
    if (!g) return;
    free(g->off); free(g->col); free(g->lab); free(g->tptr); free(g->tcomm); free(g->tcnt);
    free(g->tw); free(g->wabs); free(g);
}

double rso_wmax(const rso_graph *g) { return g->wmax; }
int64_t rso_table_size(const rso_graph *g) { return g->tptr[g->n]; }

void rso_table(const rso_graph *g, int64_t *tptr, int32_t *tcomm, int32_t *tcnt) {
    memcpy(tptr, g->tptr, (size_t)(g->n + 1) * sizeof(int64_t));
    int64_t T = g->tptr[g->n];
    if (T) { memcpy(tcomm, g->tcomm, (size_t)T * sizeof(int32_t)); memcpy(tcnt, g->tcnt, (size_t)T * sizeof(int32_t)); }
}

double rso_omega(const rso_graph *g, int32_t v, int32_t c) { return omega(g, v, c); }

/* R(u) for the listed nodes; strict != 0 drops closed triangles with C(v) = C(u) */
void rso_scores(const rso_graph *g, const int32_t *ids, int64_t m, int strict, double *out) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < m; ++i) {
        int32_t u = ids[i];
        int64_t d = g->off[u + 1] - g->off[u];
        if (d < 2 || g->wmax <= 0.0) { out[i] = 0.0; continue; }
        out[i] = rso_finish(score_sum(g, u, strict), d, g->wmax);
    }
}

void rso_scores_all(const rso_graph *g, int strict, double *out) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t u = 0; u < g->n; ++u) {
        int64_t d = g->off[u + 1] - g->off[u];
        out[u] = (d < 2 || g->wmax <= 0.0) ? 0.0 : rso_finish(score_sum(g, (int32_t)u, strict), d, g->wmax);
    }
}

/* threads used by the loops over nodes (n < 1: all the host's cores); returns the count set */
int rso_set_threads(int n) {
#ifdef _OPENMP
    if (n < 1) n = omp_get_num_procs();
    omp_set_num_threads(n);
    return n;
#else
    (void)n;
    return 1;
#endif
}

/* ---- top-K: order by (score descending, node id ascending) --------------- */
static const double *g_sort_scores;
static int cmp_rank(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    double sx = g_sort_scores[x], sy = g_sort_scores[y];
    if (sx > sy) return -1;
    if (sx < sy) return 1;
    return (x > y) - (x < y);
}
void rso_topk(const double *scores, int64_t n, int64_t K, int32_t *ids_out) {
    int32_t *idx = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    for (int64_t i = 0; i < n; ++i) idx[i] = (int32_t)i;
    g_sort_scores = scores;
    qsort(idx, (size_t)n, sizeof(int32_t), cmp_rank);
    for (int64_t i = 0; i < K && i < n; ++i) ids_out[i] = idx[i];
    free(idx);
}

/* ---- removals on a host CSR copy ----------------------------------------------
 * Node removal deletes every edge incident to the node; edge removal deletes
 * both directions.  Nodes are applied first, then edges.  `applied` counts
 * effective removals: a node already isolated by an earlier removal (listed
 * before, or flagged in `removed`), or an edge that is absent, counts 0.
 * `removed` (n flags, in/out) records removed nodes across calls.
 * Writes the new CSR to out_off (n+1) / out_col (<= old nnz).
 */
int64_t rso_remove(int64_t n, const int64_t *off, const int32_t *col, uint8_t *removed,
                   const int32_t *nodes, int64_t n_nodes, const int32_t *esrc, const int32_t *edst,
                   int64_t n_edges, int64_t *out_off, int32_t *out_col) {
    int64_t nnz = off[n];
    uint8_t *dead = (uint8_t *)calloc((size_t)(nnz > 0 ? nnz : 1), 1);
    int64_t applied = 0;
    for (int64_t i = 0; i < n_nodes; ++i) {
        int32_t v = nodes[i];
        if (v < 0 || v >= n || removed[v]) continue;
        removed[v] = 1;
        applied++;
        for (int64_t e = off[v]; e < off[v + 1]; ++e) {
            dead[e] = 1;
            int32_t x = col[e];
            int64_t lo = off[x], hi = off[x + 1];
            while (lo < hi) { int64_t mid = lo + (hi - lo) / 2; if (col[mid] < v) lo = mid + 1; else hi = mid; }
            if (lo < off[x + 1] && col[lo] == v) dead[lo] = 1;
        }
    }
    for (int64_t i = 0; i < n_edges; ++i) {
        int32_t a = esrc[i], b = edst[i];
        if (a < 0 || b < 0 || a >= n || b >= n || a == b) continue;
        int64_t lo = off[a], hi = off[a + 1];
        while (lo < hi) { int64_t mid = lo + (hi - lo) / 2; if (col[mid] < b) lo = mid + 1; else hi = mid; }
        if (!(lo < off[a + 1] && col[lo] == b) || dead[lo]) continue;
        dead[lo] = 1;
        int64_t lo2 = off[b], hi2 = off[b + 1];
        while (lo2 < hi2) { int64_t mid = lo2 + (hi2 - lo2) / 2; if (col[mid] < a) lo2 = mid + 1; else hi2 = mid; }
        dead[lo2] = 1;
        applied++;
    }
    out_off[0] = 0;
    int64_t p = 0;
    for (int64_t v = 0; v < n; ++v) {
        for (int64_t e = off[v]; e < off[v + 1]; ++e) if (!dead[e]) out_col[p++] = col[e];
        out_off[v + 1] = p;
    }
    free(dead);
    return applied;
}
