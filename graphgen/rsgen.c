/*
 * rsgen.c -- seeded synthetic community-labelled graphs (host C, no CUDA).
 *
 * Input generator shared by the CPU oracle and the GPU path.  It holds none of
 * the scoring arithmetic: it only draws graphs and community labels with the
 * shapes of the paper's workloads (social networks with planted, power-law
 * sized communities; Sec. VI, Tables "Social Networks Dataset").
 *
 * Every random draw is a pure function of (seed, stream, index) through the
 * splitmix64 finaliser (Steele, Lea, Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014), so the output does not depend on iteration order,
 * and Bernoulli trials compare integers, so the plain SBM is bit-identical on
 * every host.  The DC-SBM degree table uses pow(); a platform difference could
 * only move a draw that lands within one ulp of a table boundary.
 *
 * Output: undirected simple graph as symmetric CSR (int64 offsets, int32
 * columns sorted ascending, no self-loops, no duplicates) plus int32 labels in
 * [0, k).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int64_t n, nnz;     /* nodes, CSR entries (= 2 x undirected edges) */
    int32_t k;          /* number of communities */
    int64_t *offsets;   /* n + 1 */
    int32_t *cols;      /* nnz */
    int32_t *labels;    /* n */
    char err[160];
} rsgen_graph;

/* ---- counter-based random numbers ------------------------------------- */

static inline uint64_t sm64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}
static inline uint64_t rnd3(uint64_t seed, uint64_t stream, uint64_t i) {
    return sm64(sm64(seed ^ sm64(stream * 0xD1B54A32D192ED03ull)) + i);
}
/* uniform integer in [0, m) by the multiply-high method */
static inline uint64_t below(uint64_t r, uint64_t m) {
    return (uint64_t)(((unsigned __int128)r * m) >> 64);
}
/* uniform double in [0, 1) with 53 random bits */
static inline double unit(uint64_t r) { return (double)(r >> 11) * (1.0 / 9007199254740992.0); }

enum { ST_LABEL = 1, ST_DEG = 2, ST_INTRA = 3, ST_INTER = 4, ST_SBM = 5 };

/* ---- edge list -> CSR ---------------------------------------------------- */

/* LSD radix sort of 64-bit keys, 16 bits per pass. */
static int radix_sort_u64(uint64_t *a, int64_t m) {
    if (m < 2) return 0;
    uint64_t *tmp = (uint64_t *)malloc((size_t)m * sizeof(uint64_t));
    int64_t *cnt = (int64_t *)malloc(65536 * sizeof(int64_t));
    if (!tmp || !cnt) { free(tmp); free(cnt); return -1; }
    uint64_t *src = a, *dst = tmp;
    for (int pass = 0; pass < 4; ++pass) {
        int sh = pass * 16;
        memset(cnt, 0, 65536 * sizeof(int64_t));
        for (int64_t i = 0; i < m; ++i) cnt[(src[i] >> sh) & 0xFFFF]++;
        int64_t s = 0;
        for (int b = 0; b < 65536; ++b) { int64_t c = cnt[b]; cnt[b] = s; s += c; }
        for (int64_t i = 0; i < m; ++i) dst[cnt[(src[i] >> sh) & 0xFFFF]++] = src[i];
        uint64_t *t = src; src = dst; dst = t;
    }
    /* four passes: result is back in a */
    free(tmp); free(cnt);
    return 0;
}

/* keys are (lo << 32 | hi) with lo < hi; sorted, de-duplicated, then expanded */
static int build_csr(rsgen_graph *g, uint64_t *keys, int64_t m) {
    if (radix_sort_u64(keys, m)) return -1;
    int64_t u = 0;
    for (int64_t i = 0; i < m; ++i)
        if (i == 0 || keys[i] != keys[i - 1]) keys[u++] = keys[i];
    m = u;
    int64_t n = g->n;
    g->offsets = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    g->cols = (int32_t *)malloc((size_t)(2 * m > 0 ? 2 * m : 1) * sizeof(int32_t));
    if (!g->offsets || !g->cols) return -1;
    for (int64_t i = 0; i < m; ++i) {
        g->offsets[(keys[i] >> 32) + 1]++;
        g->offsets[(keys[i] & 0xFFFFFFFFull) + 1]++;
    }
    for (int64_t v = 0; v < n; ++v) g->offsets[v + 1] += g->offsets[v];
    int64_t *fill = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    if (!fill) return -1;
    memcpy(fill, g->offsets, (size_t)n * sizeof(int64_t));
    /* sorted by (lo, hi): row x first receives its smaller neighbours in
       ascending order, then its larger neighbours in ascending order */
    for (int64_t i = 0; i < m; ++i) {
        int32_t a = (int32_t)(keys[i] >> 32), b = (int32_t)(keys[i] & 0xFFFFFFFFull);
        g->cols[fill[a]++] = b;
        g->cols[fill[b]++] = a;
    }
    free(fill);
    g->nnz = 2 * m;
    return 0;
}

static inline uint64_t ekey(int64_t a, int64_t b) {
    return a < b ? ((uint64_t)a << 32) | (uint64_t)b : ((uint64_t)b << 32) | (uint64_t)a;
}

/* ---- plain SBM: equal blocks, Bernoulli over all pairs ------------------- */

/* Labels are the planted blocks: node v is in block v / block_size. */
int rsgen_sbm(rsgen_graph *g, int32_t nblocks, int32_t block_size, double p_in, double p_out,
              uint64_t seed) {
    memset(g, 0, sizeof(*g));
    int64_t n = (int64_t)nblocks * block_size;
    if (nblocks < 1 || block_size < 1 || n > 20000 || p_in < 0 || p_in > 1 || p_out < 0 ||
        p_out > 1) {
        strcpy(g->err, "rsgen_sbm: bad arguments (need n <= 20000, 0 <= p <= 1)");
        return -1;
    }
    g->n = n; g->k = nblocks;
    g->labels = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    for (int64_t v = 0; v < n; ++v) g->labels[v] = (int32_t)(v / block_size);
    /* integer thresholds: edge iff r < p * 2^64 */
    uint64_t t_in = p_in >= 1.0 ? UINT64_MAX : (uint64_t)(p_in * 18446744073709551616.0);
    uint64_t t_out = p_out >= 1.0 ? UINT64_MAX : (uint64_t)(p_out * 18446744073709551616.0);
    int64_t cap = 1024, m = 0;
    uint64_t *keys = (uint64_t *)malloc((size_t)cap * sizeof(uint64_t));
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j) {
            uint64_t r = rnd3(seed, ST_SBM, (uint64_t)i * (uint64_t)n + (uint64_t)j);
            uint64_t t = (g->labels[i] == g->labels[j]) ? t_in : t_out;
            if (r < t) {
                if (m == cap) { cap *= 2; keys = (uint64_t *)realloc(keys, (size_t)cap * 8); }
                keys[m++] = ekey(i, j);
            }
        }
    int rc = build_csr(g, keys, m);
    free(keys);
    if (rc) strcpy(g->err, "rsgen_sbm: out of memory");
    return rc;
}

/* ---- degree-corrected SBM ------------------------------------------------ */

/* Community sizes s_r = max(smin, c / r), r = 1..k, with c chosen so that the
   real-valued sizes sum to n; rounded by largest remainder.  Sizes descend
   with the rank, so community 0 is the largest. */
static int community_sizes(int64_t n, int32_t k, double smin, int64_t *size) {
    double lo = 0.0, hi = (double)n * 2.0;
    for (int it = 0; it < 200; ++it) {
        double c = 0.5 * (lo + hi), s = 0.0;
        for (int32_t r = 1; r <= k; ++r) { double x = c / r; s += x > smin ? x : smin; }
        if (s > (double)n) hi = c; else lo = c;
    }
    double c = 0.5 * (lo + hi);
    double *frac = (double *)malloc((size_t)k * sizeof(double));
    int64_t tot = 0;
    for (int32_t r = 1; r <= k; ++r) {
        double x = c / r; if (x < smin) x = smin;
        size[r - 1] = (int64_t)floor(x);
        frac[r - 1] = x - floor(x);
        tot += size[r - 1];
    }
    /* hand the remaining units to the largest remainders (ties: lower rank) */
    while (tot < n) {
        int32_t best = 0;
        for (int32_t r = 1; r < k; ++r) if (frac[r] > frac[best]) best = r;
        size[best]++; frac[best] = -1.0; tot++;
    }
    while (tot > n) {  /* only if smin * k > n */
        int32_t best = -1;
        for (int32_t r = k - 1; r >= 0; --r) if (size[r] > 1) { best = r; break; }
        if (best < 0) break;
        size[best]--; tot--;
    }
    free(frac);
    return tot == n ? 0 : -1;
}

/* Fisher-Yates shuffle of a[0..m) driven by stream (seed, st). */
static void shuffle_i32(int32_t *a, int64_t m, uint64_t seed, uint64_t st) {
    for (int64_t i = m - 1; i > 0; --i) {
        int64_t j = (int64_t)below(rnd3(seed, st, (uint64_t)i), (uint64_t)i + 1);
        int32_t t = a[i]; a[i] = a[j]; a[j] = t;
    }
}

/*
 * DC-SBM by the configuration model:
 *   - k communities, sizes from community_sizes(); nodes are assigned to
 *     communities by a seeded random permutation;
 *   - node degrees d_v drawn from the discrete power law P(d) ~ d^-gamma on
 *     [dmin, dmax];
 *   - each node splits d_v into round((1 - mu) d_v) intra stubs and the rest
 *     inter stubs; intra stubs beyond (community size - 1) move to inter stubs;
 *   - intra stubs are paired at random inside each community; inter stubs are
 *     paired at random over the whole graph, pairs that land in one community
 *     are re-paired (3 rounds, then dropped);
 *   - self-loops are dropped and multi-edges merged.
 */
int rsgen_dcsbm(rsgen_graph *g, int64_t n, int32_t k, double size_min, double gamma, int32_t dmin,
                int32_t dmax, double mu, uint64_t seed) {
    memset(g, 0, sizeof(*g));
    if (n < 2 || n > 2000000000LL || k < 1 || k > n || dmin < 1 || dmax < dmin || mu < 0 ||
        mu > 1 || gamma <= 1.0) {
        strcpy(g->err, "rsgen_dcsbm: bad arguments");
        return -1;
    }
    g->n = n; g->k = k;
    int64_t *size = (int64_t *)malloc((size_t)k * sizeof(int64_t));
    if (community_sizes(n, k, size_min, size)) {
        strcpy(g->err, "rsgen_dcsbm: community sizes do not fit n");
        free(size);
        return -1;
    }
    /* labels: block expansion, then a seeded permutation */
    g->labels = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int64_t p = 0;
    for (int32_t c = 0; c < k; ++c)
        for (int64_t i = 0; i < size[c]; ++i) g->labels[p++] = c;
    shuffle_i32(g->labels, n, seed, ST_LABEL);

    /* degree table: cumulative weights of d^-gamma */
    int32_t nd = dmax - dmin + 1;
    double *cdf = (double *)malloc((size_t)nd * sizeof(double));
    double acc = 0.0;
    for (int32_t i = 0; i < nd; ++i) { acc += pow((double)(dmin + i), -gamma); cdf[i] = acc; }
    int32_t *deg_in = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *deg_out = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int64_t tot_in = 0, tot_out = 0;
    for (int64_t v = 0; v < n; ++v) {
        double u = unit(rnd3(seed, ST_DEG, (uint64_t)v)) * acc;
        int32_t lo = 0, hi = nd - 1;   /* first i with cdf[i] > u */
        while (lo < hi) { int32_t mid = (lo + hi) / 2; if (cdf[mid] > u) hi = mid; else lo = mid + 1; }
        int32_t d = dmin + lo;
        int32_t din = (int32_t)floor((1.0 - mu) * d + 0.5);
        int64_t room = size[g->labels[v]] - 1;
        if (din > room) din = (int32_t)room;
        deg_in[v] = din; deg_out[v] = d - din;
        tot_in += din; tot_out += d - din;
    }
    free(cdf);

    int64_t cap = (tot_in + tot_out) / 2 + 16, m = 0;
    uint64_t *keys = (uint64_t *)malloc((size_t)cap * sizeof(uint64_t));
    /* intra stubs grouped by community */
    int64_t *cstart = (int64_t *)calloc((size_t)k + 1, sizeof(int64_t));
    for (int64_t v = 0; v < n; ++v) cstart[g->labels[v] + 1] += deg_in[v];
    for (int32_t c = 0; c < k; ++c) cstart[c + 1] += cstart[c];
    int32_t *stubs = (int32_t *)malloc((size_t)(tot_in > tot_out ? tot_in : tot_out) * sizeof(int32_t) + 4);
    int64_t *fill = (int64_t *)malloc((size_t)k * sizeof(int64_t));
    memcpy(fill, cstart, (size_t)k * sizeof(int64_t));
    for (int64_t v = 0; v < n; ++v)
        for (int32_t j = 0; j < deg_in[v]; ++j) stubs[fill[g->labels[v]]++] = (int32_t)v;
    for (int32_t c = 0; c < k; ++c) {
        int64_t a = cstart[c], len = cstart[c + 1] - a;
        shuffle_i32(stubs + a, len, seed, ((uint64_t)ST_INTRA << 32) | (uint64_t)c);
        for (int64_t i = 0; i + 1 < len; i += 2) {
            int32_t x = stubs[a + i], y = stubs[a + i + 1];
            if (x != y) keys[m++] = ekey(x, y);
        }
    }
    free(fill); free(cstart);
    /* inter stubs: global pairing with re-pairing of same-community pairs */
    int64_t ns = 0;
    for (int64_t v = 0; v < n; ++v)
        for (int32_t j = 0; j < deg_out[v]; ++j) stubs[ns++] = (int32_t)v;
    for (int round = 0; round < 4 && ns > 1; ++round) {
        shuffle_i32(stubs, ns, seed, ((uint64_t)ST_INTER << 32) | (uint64_t)round);
        int64_t left = 0;
        for (int64_t i = 0; i + 1 < ns; i += 2) {
            int32_t x = stubs[i], y = stubs[i + 1];
            if (g->labels[x] != g->labels[y]) {
                if (m == cap) { cap = cap * 2; keys = (uint64_t *)realloc(keys, (size_t)cap * 8); }
                keys[m++] = ekey(x, y);
            } else if (round < 3) {
                stubs[left++] = x; stubs[left++] = y;
            }
        }
        ns = left;
    }
    free(stubs); free(deg_in); free(deg_out); free(size);
    int rc = build_csr(g, keys, m);
    free(keys);
    if (rc) strcpy(g->err, "rsgen_dcsbm: out of memory");
    return rc;
}

/* ---- handle API for ctypes ------------------------------------------------ */

rsgen_graph *rsgen_new(void) { return (rsgen_graph *)calloc(1, sizeof(rsgen_graph)); }
void rsgen_free(rsgen_graph *g) {
    if (!g) return;
    free(g->offsets); free(g->cols); free(g->labels); free(g);
}
int64_t rsgen_n(const rsgen_graph *g) { return g->n; }
int64_t rsgen_nnz(const rsgen_graph *g) { return g->nnz; }
int32_t rsgen_k(const rsgen_graph *g) { return g->k; }
const char *rsgen_err(const rsgen_graph *g) { return g->err; }
void rsgen_copy(const rsgen_graph *g, int64_t *offsets, int32_t *cols, int32_t *labels) {
    memcpy(offsets, g->offsets, (size_t)(g->n + 1) * sizeof(int64_t));
    if (g->nnz) memcpy(cols, g->cols, (size_t)g->nnz * sizeof(int32_t));
    memcpy(labels, g->labels, (size_t)g->n * sizeof(int32_t));
}
