// rs_score.cu -- the Robust Spanning Index of every node on the GPU.
//
// The score (Sec. III-B, Eq. RSI) sums, for each node u, the geometric means
// (w_v(u) w_w(v) w_w(u))^(1/3) over ordered pairs (w, v) with w in N(u),
// C(w) != C(u), v in N(w), v != u, C(v) != C(w) and (v in N(u) or
// C(v) = C(u)).  By Lemma 1 a weight depends on the target only through its
// community, w_v(u) = w_v(C(u)), so with sigma_v(c) = w_v(c)^(1/3) the sum
// splits exactly into two kinds of triads:
//
//  * Type-II (Sec. III-A), every v with C(v) = C(u), adjacent to u or not:
//      sum_w sigma_w(C(u))^2 (Q_w(C(u)) - s_u),
//    with s_x = sigma_x(C(x)) (Lemma 2) and Q_w(c) = sum of s_x over the
//    neighbours x of w in community c;
//  * Type-I, v adjacent to u with three distinct communities: the triangles of
//    the cross-community subgraph G_x (every edge of which joins two
//    communities, so each of its triangles spans three); the two ordered
//    triads at apex a of triangle {a, b, c} add
//      S(b->a) S(c->a) (S(b->c) + S(c->b)),   S(x->y) = sigma_x(C(y)).
//
// Passes (Alg. 1 Steps 1-3 and the kernels of Sec. V-B, re-planned):
//   P1  per row v: neighbour-community counts f_v(c) (the interaction_matrix
//       row), aggregates T, L, X, the row's largest weight (-> w_max, Alg. 1
//       Step 2 / normalize_weights), s_v, the cross degree dx(v) (border
//       vertex iff dx > 0, Alg. 1 Step 1);
//   GX  offsets of the cross subgraph rows (nodes with dx >= 2);
//   P2  per row w: counts and Q_w again, sigma_w per column, the Type-II
//       terms pushed to the neighbours, and the G_x rows of w (out-neighbours
//       of higher (dx, id) rank first, in-neighbours from the back);
//   P3  per node a: oriented triangle listing on G_x (merge by binary search),
//       the Type-I terms of the three apexes;
//   FIN R(u) = acc(u) / (w_max d(u)(d(u)-1)), 0 when d(u) < 2 or w_max = 0.
// All terms are added into 128-bit fixed-point accumulators, so the scores do
// not depend on the order in which threads run.
#include "rs.h"
#include "rs_internal.cuh"

using namespace rs;

#define FULL 0xFFFFFFFFu

namespace {

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ uint32_t dev_pow2_at_least(uint32_t x) {
    return x <= 1 ? 1u : 1u << (32 - __clz(x - 1));
}

__device__ __forceinline__ unsigned long long double_bits(df a) {
    return (unsigned long long)__double_as_longlong(df_to_double(a));
}

// ---- hash tables keyed by community (shared or global memory) ----------------
struct Tab {
    int32_t *key;
    uint32_t *cnt;
    unsigned long long *q;   // 2 words per slot (Type-II sums), may be null
    df *sig;                 // per slot sigma, may be null
    uint32_t mask;
};

__device__ __forceinline__ uint32_t slot_of(int32_t c, uint32_t mask) {
    uint32_t h = hash_label(c);
    h ^= h >> 15;
    return h & mask;
}

__device__ __forceinline__ int tab_insert(const Tab &t, int32_t c, uint32_t add, int *err) {
    uint32_t h = slot_of(c, t.mask);
    for (uint32_t it = 0; it <= t.mask; ++it) {
        int32_t prev = atomicCAS(&t.key[h], kEmpty, c);
        if (prev == kEmpty || prev == c) {
            if (add) atomicAdd(&t.cnt[h], add);
            return (int)h;
        }
        h = (h + 1) & t.mask;
    }
    atomicOr(err, 1);
    return -1;
}

__device__ __forceinline__ int tab_find(const Tab &t, int32_t c) {
    uint32_t h = slot_of(c, t.mask);
    for (uint32_t it = 0; it <= t.mask; ++it) {
        int32_t k = t.key[h];
        if (k == c) return (int)h;
        if (k == kEmpty) return -1;
        h = (h + 1) & t.mask;
    }
    return -1;
}

// ---- block reductions (every thread of the CTA must call) ----------------------
template <int NT>
__device__ __forceinline__ uint32_t block_sum_u32(uint32_t v, uint32_t *sh) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    uint32_t s = 0;
    for (int i = 0; i < NT / 32; ++i) s += sh[i];
    return s;
}
template <int NT>
__device__ __forceinline__ u128 block_sum_u128(u128 v, u128 *sh) {
    v = warp_sum_u128(v);
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    u128 s = 0;
    for (int i = 0; i < NT / 32; ++i) s += sh[i];
    return s;
}
template <int NT>
__device__ __forceinline__ df block_max_df(df v, df *sh) {
    v = warp_max_df(v);
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    df m = sh[0];
    for (int i = 1; i < NT / 32; ++i) m = df_max(m, sh[i]);
    return m;
}

// sum of x over the lanes of `grp` other than this lane (exact, fixed order)
__device__ __forceinline__ u128 group_sum_others(const uint64_t *stage, unsigned grp, int lane) {
    u128 q = 0;
    unsigned m = grp & ~(1u << lane);
    while (m) {
        int j = __ffs(m) - 1;
        q += stage[j];
        m &= m - 1;
    }
    return q;
}
__device__ __forceinline__ u128 group_sum_all(const uint64_t *stage, unsigned grp) {
    u128 q = 0;
    while (grp) {
        int j = __ffs(grp) - 1;
        q += stage[j];
        grp &= grp - 1;
    }
    return q;
}

// Type-II term sigma^2 (Q - s_u) pushed to u
__device__ __forceinline__ void push_type2(unsigned long long *acc, int32_t u, df sig, u128 rest) {
    if (rest == 0 || !(sig.hi > 0.0f)) return;
    df t = df_mul(df_mul(sig, sig), df_from_u128(rest, -kSFrac));
    atomic_add_u128(acc + 2 * (int64_t)u, df_to_fixed(t, kAccFrac));
}

// finishing a row in P1: the row's largest weight, s_v and the node record
__device__ __forceinline__ df p1_row_result(const RowAgg &a, uint32_t own, df col_max, int32_t k,
                                            const uint64_t *LG, NodeRec &out, int32_t cv) {
    df wabs = column_weight(a, 0, LG);                    // community absent from N(v)
    df m = col_max;
    if (a.L < (uint32_t)k) m = df_max(m, wabs);
    df wown = own > 0 ? column_weight(a, own, LG) : wabs;
    df s = df_cbrt(wown);
    out.s_fix = (uint64_t)df_to_fixed(s, kSFrac);
    out.label = cv;
    out.dx = (int32_t)(a.T - own);
    return m;
}

// ======================================================================================
// P1
// ======================================================================================
__global__ void __launch_bounds__(kThreads) p1_small_kernel(
    const int64_t *__restrict__ off, const int32_t *__restrict__ col, const int32_t *__restrict__ lab,
    const int32_t *__restrict__ rows, int64_t nrows, int32_t k, const uint64_t *__restrict__ LG,
    NodeRec *__restrict__ rec, int32_t *__restrict__ Lall, unsigned long long *wmax_bits) {
    int lane = threadIdx.x & 31;
    int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    df best{0.0f, 0.0f};
    for (int64_t i = warp; i < nrows; i += nwarps) {
        int32_t v = rows[i];
        int64_t b = off[v];
        int d = (int)(off[v + 1] - b);
        int32_t cv = lab[v];
        bool act = lane < d;
        int32_t c = act ? lab[col[b + lane]] : -1;
        unsigned amask = __ballot_sync(FULL, act);
        unsigned grp = 0;
        if (act) grp = __match_any_sync(amask, c);
        uint32_t f = __popc(grp);
        bool leader = act && (__ffs(grp) - 1 == lane);
        uint32_t L = __popc(__ballot_sync(FULL, leader));
        uint32_t own = __popc(__ballot_sync(FULL, act && c == cv));
        u128 x = leader ? (u128)f * LG[f] : (u128)0;
        RowAgg a{(uint32_t)d, L, warp_sum_u128(x)};
        df w{0.0f, 0.0f};
        if (leader) w = column_weight(a, f, LG);
        df cm = warp_max_df(w);
        NodeRec r;
        df m = p1_row_result(a, own, cm, k, LG, r, cv);
        if (lane == 0) {
            rec[v] = r;
            Lall[v] = (int32_t)L;
        }
        best = df_max(best, m);
    }
    if (lane == 0 && best.hi > 0.0f) atomicMax(wmax_bits, double_bits(best));
}

template <int NT>
__global__ void __launch_bounds__(NT) p1_mid_kernel(
    const int64_t *__restrict__ off, const int32_t *__restrict__ col, const int32_t *__restrict__ lab,
    const int32_t *__restrict__ rows, int64_t nrows, int32_t k, const uint64_t *__restrict__ LG,
    NodeRec *__restrict__ rec, int32_t *__restrict__ Lall, unsigned long long *wmax_bits, int *err) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint32_t sh_u32[NT / 32];
    __shared__ u128 sh_u128[NT / 32];
    __shared__ df sh_df[NT / 32];
    int tid = threadIdx.x, lane = tid & 31;
    df best{0.0f, 0.0f};
    for (int64_t i = blockIdx.x; i < nrows; i += gridDim.x) {
        int32_t v = rows[i];
        int64_t b = off[v];
        int d = (int)(off[v + 1] - b);
        int32_t cv = lab[v];
        uint32_t cap = dev_pow2_at_least(2u * (uint32_t)min(d, k));
        Tab t{(int32_t *)smem, (uint32_t *)(smem + 4 * cap), nullptr, nullptr, cap - 1};
        for (uint32_t j = tid; j < cap; j += NT) { t.key[j] = kEmpty; t.cnt[j] = 0; }
        __syncthreads();
        uint32_t own = 0;
        for (int base = 0; base < d; base += NT) {
            int e = base + tid;
            bool act = e < d;
            int32_t c = act ? lab[col[b + e]] : -1;
            own += (act && c == cv);
            bool foreign = act && c != cv;
            unsigned fm = __ballot_sync(FULL, foreign);
            if (foreign) {
                unsigned grp = __match_any_sync(fm, c);
                if (lane == __ffs(grp) - 1) tab_insert(t, c, __popc(grp), err);
            }
        }
        own = block_sum_u32<NT>(own, sh_u32);      // syncs: the table is complete
        uint32_t Lf = 0;
        u128 X = 0;
        for (uint32_t j = tid; j < cap; j += NT)
            if (t.key[j] != kEmpty) { Lf++; X += (u128)t.cnt[j] * LG[t.cnt[j]]; }
        Lf = block_sum_u32<NT>(Lf, sh_u32);
        X = block_sum_u128<NT>(X, sh_u128);
        RowAgg a{(uint32_t)d, Lf + (own > 0 ? 1u : 0u), X + (u128)own * LG[own]};
        df cm{0.0f, 0.0f};
        for (uint32_t j = tid; j < cap; j += NT)
            if (t.key[j] != kEmpty) cm = df_max(cm, column_weight(a, t.cnt[j], LG));
        if (own > 0) cm = df_max(cm, column_weight(a, own, LG));
        cm = block_max_df<NT>(cm, sh_df);
        if (tid == 0) {
            NodeRec r;
            df m = p1_row_result(a, own, cm, k, LG, r, cv);
            rec[v] = r;
            Lall[v] = (int32_t)a.L;
            best = df_max(best, m);
        }
        __syncthreads();                              // table reuse
    }
    if (tid == 0 && best.hi > 0.0f) atomicMax(wmax_bits, double_bits(best));
}

// hub rows: chunks insert foreign communities into the row's global table
template <int NT>
__global__ void __launch_bounds__(NT) hub_p1_insert_kernel(
    const int64_t *__restrict__ off, const int32_t *__restrict__ col, const int32_t *__restrict__ lab,
    const HubInfo *__restrict__ hubs, const int32_t *__restrict__ items, const int32_t *__restrict__ chunks,
    int64_t nitems, int32_t *hkey, uint32_t *hcnt, HubAgg *hagg, int *err) {
    __shared__ uint32_t sh_u32[NT / 32];
    int tid = threadIdx.x, lane = tid & 31;
    for (int64_t it = blockIdx.x; it < nitems; it += gridDim.x) {
        HubInfo h = hubs[items[it]];
        int64_t b = off[h.row];
        int64_t d = off[h.row + 1] - b;
        int64_t lo = (int64_t)chunks[it] * kHubChunk;
        int64_t hi = min(d, lo + kHubChunk);
        int32_t cv = lab[h.row];
        Tab t{hkey + h.tab, hcnt + h.tab, nullptr, nullptr, (uint32_t)h.cap - 1};
        uint32_t own = 0;
        for (int64_t base = lo; base < hi; base += NT) {
            int64_t e = base + tid;
            bool act = e < hi;
            int32_t c = act ? lab[col[b + e]] : -1;
            own += (act && c == cv);
            bool foreign = act && c != cv;
            unsigned fm = __ballot_sync(FULL, foreign);
            if (foreign) {
                unsigned grp = __match_any_sync(fm, c);
                if (lane == __ffs(grp) - 1) tab_insert(t, c, __popc(grp), err);
            }
        }
        own = block_sum_u32<NT>(own, sh_u32);
        if (tid == 0 && own) atomicAdd(&hagg[items[it]].own, own);
        __syncthreads();
    }
}

template <int NT>
__global__ void __launch_bounds__(NT) hub_p1_finish_kernel(
    const int64_t *__restrict__ off, const int32_t *__restrict__ lab, const HubInfo *__restrict__ hubs,
    int64_t nhubs, int32_t k, const uint64_t *__restrict__ LG, const int32_t *hkey, const uint32_t *hcnt,
    HubAgg *hagg, NodeRec *__restrict__ rec, int32_t *__restrict__ Lall, unsigned long long *wmax_bits) {
    __shared__ uint32_t sh_u32[NT / 32];
    __shared__ u128 sh_u128[NT / 32];
    __shared__ df sh_df[NT / 32];
    int tid = threadIdx.x;
    df best{0.0f, 0.0f};
    for (int64_t hi = blockIdx.x; hi < nhubs; hi += gridDim.x) {
        HubInfo h = hubs[hi];
        int64_t d = off[h.row + 1] - off[h.row];
        uint32_t own = hagg[hi].own;
        uint32_t Lf = 0;
        u128 X = 0;
        for (int64_t j = tid; j < h.cap; j += NT) {
            int64_t s = h.tab + j;
            if (hkey[s] != kEmpty) { Lf++; X += (u128)hcnt[s] * LG[hcnt[s]]; }
        }
        Lf = block_sum_u32<NT>(Lf, sh_u32);
        X = block_sum_u128<NT>(X, sh_u128);
        RowAgg a{(uint32_t)d, Lf + (own > 0 ? 1u : 0u), X + (u128)own * LG[own]};
        df cm{0.0f, 0.0f};
        for (int64_t j = tid; j < h.cap; j += NT) {
            int64_t s = h.tab + j;
            if (hkey[s] != kEmpty) cm = df_max(cm, column_weight(a, hcnt[s], LG));
        }
        if (own > 0) cm = df_max(cm, column_weight(a, own, LG));
        cm = block_max_df<NT>(cm, sh_df);
        if (tid == 0) {
            HubAgg g = hagg[hi];
            g.X = a.X;
            g.L = a.L;
            hagg[hi] = g;
            NodeRec r;
            df m = p1_row_result(a, own, cm, k, LG, r, lab[h.row]);
            rec[h.row] = r;
            Lall[h.row] = (int32_t)a.L;
            best = df_max(best, m);
        }
        __syncthreads();
    }
    if (tid == 0 && best.hi > 0.0f) atomicMax(wmax_bits, double_bits(best));
}

// ======================================================================================
// G_x row capacity: nodes with dx >= 2 keep dx slots
// ======================================================================================
__global__ void gx_capacity_kernel(const NodeRec *__restrict__ rec, int64_t n, int64_t *xoff) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v == 0) xoff[0] = 0;
    if (v < n) {
        int32_t dx = rec[v].dx;
        xoff[v + 1] = dx >= 2 ? dx : 0;
    }
}

// ======================================================================================
// P2
// ======================================================================================
__global__ void __launch_bounds__(kThreads) p2_small_kernel(
    const int64_t *__restrict__ off, const int32_t *__restrict__ col, const int32_t *__restrict__ rows,
    int64_t nrows, const uint64_t *__restrict__ LG, const NodeRec *__restrict__ rec,
    unsigned long long *acc, const int64_t *__restrict__ xoff, int32_t *__restrict__ xcol,
    df *__restrict__ xS, int32_t *__restrict__ xout, int32_t *__restrict__ xin) {
    __shared__ uint64_t stage[kThreads];
    int lane = threadIdx.x & 31;
    uint64_t *st = stage + (threadIdx.x & ~31);
    int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < nrows; i += nwarps) {
        int32_t w = rows[i];
        int64_t b = off[w];
        int d = (int)(off[w + 1] - b);
        NodeRec rw = rec[w];
        bool act = lane < d;
        int32_t u = act ? col[b + lane] : -1;
        NodeRec ru{0, -1, 0};
        if (act) ru = rec[u];
        int32_t c = ru.label;
        unsigned amask = __ballot_sync(FULL, act);
        unsigned grp = 0;
        if (act) grp = __match_any_sync(amask, c);
        uint32_t f = __popc(grp);
        bool leader = act && (__ffs(grp) - 1 == lane);
        uint32_t L = __popc(__ballot_sync(FULL, leader));
        u128 x = leader ? (u128)f * LG[f] : (u128)0;
        RowAgg a{(uint32_t)d, L, warp_sum_u128(x)};
        bool cross = act && c != rw.label;
        df sig{0.0f, 0.0f};
        if (cross) sig = df_cbrt(column_weight(a, f, LG));
        st[lane] = ru.s_fix;
        __syncwarp();
        if (cross && f > 1) push_type2(acc, u, sig, group_sum_others(st, grp, lane));
        __syncwarp();
        // G_x row of w: cross neighbours with dx >= 2, ordered by id
        int32_t cnt_out = 0, cnt_in = 0;
        if (rw.dx >= 2) {
            bool inx = cross && ru.dx >= 2;
            bool out = inx && rank_after(ru.dx, u, rw.dx, w);
            bool in = inx && !out;
            unsigned mo = __ballot_sync(FULL, out), mi = __ballot_sync(FULL, in);
            int64_t xb = xoff[w];
            if (out) {
                int64_t p = xb + __popc(mo & lanemask_lt());
                xcol[p] = u; xS[p] = sig;
            }
            if (in) {
                int64_t p = xb + rw.dx - 1 - __popc(mi & lanemask_lt());
                xcol[p] = u; xS[p] = sig;
            }
            cnt_out = __popc(mo); cnt_in = __popc(mi);
        }
        if (lane == 0) { xout[w] = cnt_out; xin[w] = cnt_in; }
    }
}

// slot layout of the P2 tables: key[cap] | cnt[cap] | q[2 cap] | sig[cap]  (32 B per slot)
__device__ __forceinline__ Tab p2_table(unsigned char *base, uint32_t cap) {
    Tab t;
    t.q = (unsigned long long *)base;
    t.sig = (df *)(base + 16 * (size_t)cap);
    t.key = (int32_t *)(base + 24 * (size_t)cap);
    t.cnt = (uint32_t *)(base + 28 * (size_t)cap);
    t.mask = cap - 1;
    return t;
}

// CTA-ordered compaction of the G_x entries of one round; returns this thread's position
template <int NT>
__device__ __forceinline__ void gx_round(bool out, bool in, int64_t xb, int32_t dxw, int32_t u, df sig,
                                         int32_t &base_out, int32_t &base_in, int32_t *xcol, df *xS,
                                         int32_t *sh_cnt /* 2 * NT/32 */) {
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned mo = __ballot_sync(FULL, out), mi = __ballot_sync(FULL, in);
    if (lane == 0) { sh_cnt[wid] = __popc(mo); sh_cnt[NT / 32 + wid] = __popc(mi); }
    __syncthreads();
    int32_t po = base_out, pi = base_in, to = 0, ti = 0;
    for (int j = 0; j < NT / 32; ++j) {
        if (j < wid) { po += sh_cnt[j]; pi += sh_cnt[NT / 32 + j]; }
        to += sh_cnt[j]; ti += sh_cnt[NT / 32 + j];
    }
    if (out) {
        int64_t p = xb + po + __popc(mo & lanemask_lt());
        xcol[p] = u; xS[p] = sig;
    }
    if (in) {
        int64_t p = xb + dxw - 1 - (pi + __popc(mi & lanemask_lt()));
        xcol[p] = u; xS[p] = sig;
    }
    base_out += to; base_in += ti;
    __syncthreads();
}

template <int NT>
__global__ void __launch_bounds__(NT) p2_mid_kernel(
    const int64_t *__restrict__ off, const int32_t *__restrict__ col, const int32_t *__restrict__ rows,
    int64_t nrows, int32_t k, const uint64_t *__restrict__ LG, const NodeRec *__restrict__ rec,
    unsigned long long *acc, const int64_t *__restrict__ xoff, int32_t *__restrict__ xcol,
    df *__restrict__ xS, int32_t *__restrict__ xout, int32_t *__restrict__ xin, int *err) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint32_t sh_u32[NT / 32];
    __shared__ u128 sh_u128[NT / 32];
    __shared__ int32_t sh_cnt[2 * NT / 32];
    __shared__ uint64_t stage[NT];
    int tid = threadIdx.x, lane = tid & 31;
    uint64_t *st = stage + (tid & ~31);
    for (int64_t i = blockIdx.x; i < nrows; i += gridDim.x) {
        int32_t w = rows[i];
        int64_t b = off[w];
        int d = (int)(off[w + 1] - b);
        NodeRec rw = rec[w];
        uint32_t cap = dev_pow2_at_least(2u * (uint32_t)min(d, k));
        Tab t = p2_table(smem, cap);
        for (uint32_t j = tid; j < cap; j += NT) {
            t.key[j] = kEmpty; t.cnt[j] = 0; t.q[2 * j] = 0; t.q[2 * j + 1] = 0;
        }
        __syncthreads();
        uint32_t own = 0;
        for (int base = 0; base < d; base += NT) {
            int e = base + tid;
            bool act = e < d;
            NodeRec ru{0, -1, 0};
            if (act) ru = rec[col[b + e]];
            own += (act && ru.label == rw.label);
            bool foreign = act && ru.label != rw.label;
            st[lane] = ru.s_fix;
            __syncwarp();
            unsigned fm = __ballot_sync(FULL, foreign);
            if (foreign) {
                unsigned grp = __match_any_sync(fm, ru.label);
                if (lane == __ffs(grp) - 1) {
                    int s = tab_insert(t, ru.label, __popc(grp), err);
                    if (s >= 0) atomic_add_u128(t.q + 2 * s, group_sum_all(st, grp));
                }
            }
            __syncwarp();
        }
        own = block_sum_u32<NT>(own, sh_u32);
        uint32_t Lf = 0;
        u128 X = 0;
        for (uint32_t j = tid; j < cap; j += NT)
            if (t.key[j] != kEmpty) { Lf++; X += (u128)t.cnt[j] * LG[t.cnt[j]]; }
        Lf = block_sum_u32<NT>(Lf, sh_u32);
        X = block_sum_u128<NT>(X, sh_u128);
        RowAgg a{(uint32_t)d, Lf + (own > 0 ? 1u : 0u), X + (u128)own * LG[own]};
        for (uint32_t j = tid; j < cap; j += NT)
            if (t.key[j] != kEmpty) t.sig[j] = df_cbrt(column_weight(a, t.cnt[j], LG));
        __syncthreads();
        int64_t xb = xoff[w];
        int32_t bo = 0, bi = 0;
        for (int base = 0; base < d; base += NT) {
            int e = base + tid;
            bool act = e < d;
            int32_t u = act ? col[b + e] : -1;
            NodeRec ru{0, -1, 0};
            if (act) ru = rec[u];
            bool cross = act && ru.label != rw.label;
            df sig{0.0f, 0.0f};
            if (cross) {
                int s = tab_find(t, ru.label);
                if (s < 0) { atomicOr(err, 2); cross = false; }
                else {
                    sig = t.sig[s];
                    if (t.cnt[s] > 1) {
                        u128 q = ((u128)t.q[2 * s + 1] << 64) | t.q[2 * s];
                        push_type2(acc, u, sig, q - ru.s_fix);
                    }
                }
            }
            if (rw.dx >= 2) {
                bool inx = cross && ru.dx >= 2;
                bool o = inx && rank_after(ru.dx, u, rw.dx, w);
                gx_round<NT>(o, inx && !o, xb, rw.dx, u, sig, bo, bi, xcol, xS, sh_cnt);
            }
        }
        if (tid == 0) { xout[w] = bo; xin[w] = bi; }
        __syncthreads();
    }
}

// hub rows, P2 step 1: Type-II group sums and per-chunk G_x counts
template <int NT>
__global__ void __launch_bounds__(NT) hub_p2_insert_kernel(
    const int64_t *__restrict__ off, const int32_t *__restrict__ col, const HubInfo *__restrict__ hubs,
    const int32_t *__restrict__ items, const int32_t *__restrict__ chunks, int64_t nitems,
    const NodeRec *__restrict__ rec, const int32_t *hkey, unsigned long long *hq,
    int32_t *hitem_out, int32_t *hitem_in, int *err) {
    __shared__ uint32_t sh_u32[NT / 32];
    __shared__ uint64_t stage[NT];
    int tid = threadIdx.x, lane = tid & 31;
    uint64_t *st = stage + (tid & ~31);
    for (int64_t it = blockIdx.x; it < nitems; it += gridDim.x) {
        HubInfo h = hubs[items[it]];
        int64_t b = off[h.row];
        int64_t d = off[h.row + 1] - b;
        int64_t lo = (int64_t)chunks[it] * kHubChunk;
        int64_t hi = min(d, lo + kHubChunk);
        NodeRec rw = rec[h.row];
        Tab t{(int32_t *)hkey + h.tab, nullptr, hq + 2 * h.tab, nullptr, (uint32_t)h.cap - 1};
        uint32_t no = 0, ni = 0;
        for (int64_t base = lo; base < hi; base += NT) {
            int64_t e = base + tid;
            bool act = e < hi;
            int32_t u = act ? col[b + e] : -1;
            NodeRec ru{0, -1, 0};
            if (act) ru = rec[u];
            bool foreign = act && ru.label != rw.label;
            st[lane] = ru.s_fix;
            __syncwarp();
            unsigned fm = __ballot_sync(FULL, foreign);
            if (foreign) {
                unsigned grp = __match_any_sync(fm, ru.label);
                if (lane == __ffs(grp) - 1) {
                    int s = tab_find(t, ru.label);
                    if (s < 0) atomicOr(err, 4);
                    else atomic_add_u128(t.q + 2 * s, group_sum_all(st, grp));
                }
            }
            __syncwarp();
            if (rw.dx >= 2 && foreign && ru.dx >= 2) {
                if (rank_after(ru.dx, u, rw.dx, h.row)) no++; else ni++;
            }
        }
        no = block_sum_u32<NT>(no, sh_u32);
        ni = block_sum_u32<NT>(ni, sh_u32);
        if (tid == 0) { hitem_out[it] = (int32_t)no; hitem_in[it] = (int32_t)ni; }
        __syncthreads();
    }
}

// hub rows, P2 step 2: sigma per table slot, G_x counts of the row
template <int NT>
__global__ void __launch_bounds__(NT) hub_p2_sigma_kernel(
    const HubInfo *__restrict__ hubs, int64_t nhubs, const uint64_t *__restrict__ LG,
    const HubAgg *__restrict__ hagg, const int64_t *__restrict__ off, const int32_t *hkey,
    const uint32_t *hcnt, df *hsig, const int32_t *hitem_out, const int32_t *hitem_in,
    int32_t *xout, int32_t *xin) {
    for (int64_t hi = blockIdx.x; hi < nhubs; hi += gridDim.x) {
        HubInfo h = hubs[hi];
        HubAgg g = hagg[hi];
        RowAgg a{(uint32_t)(off[h.row + 1] - off[h.row]), g.L, g.X};
        for (int64_t j = threadIdx.x; j < h.cap; j += NT) {
            int64_t s = h.tab + j;
            if (hkey[s] != kEmpty) hsig[s] = df_cbrt(column_weight(a, hcnt[s], LG));
        }
        if (threadIdx.x == 0) {
            int32_t so = 0, si = 0;
            for (int j = 0; j < h.n_items; ++j) {
                so += hitem_out[h.first_item + j];
                si += hitem_in[h.first_item + j];
            }
            xout[h.row] = so; xin[h.row] = si;
        }
    }
}

// hub rows, P2 step 3: Type-II terms and the G_x entries of each chunk
template <int NT>
__global__ void __launch_bounds__(NT) hub_p2_emit_kernel(
    const int64_t *__restrict__ off, const int32_t *__restrict__ col, const HubInfo *__restrict__ hubs,
    const int32_t *__restrict__ items, const int32_t *__restrict__ chunks, int64_t nitems,
    const NodeRec *__restrict__ rec, const int32_t *hkey, const uint32_t *hcnt,
    const unsigned long long *hq, const df *hsig, const int32_t *hitem_out, const int32_t *hitem_in,
    unsigned long long *acc, const int64_t *__restrict__ xoff, int32_t *__restrict__ xcol,
    df *__restrict__ xS, int *err) {
    __shared__ int32_t sh_cnt[2 * NT / 32];
    int tid = threadIdx.x;
    for (int64_t it = blockIdx.x; it < nitems; it += gridDim.x) {
        int32_t hidx = items[it];
        HubInfo h = hubs[hidx];
        int64_t b = off[h.row];
        int64_t d = off[h.row + 1] - b;
        int32_t ch = chunks[it];
        int64_t lo = (int64_t)ch * kHubChunk;
        int64_t hi = min(d, lo + kHubChunk);
        NodeRec rw = rec[h.row];
        Tab t{(int32_t *)hkey + h.tab, (uint32_t *)hcnt + h.tab, nullptr, nullptr, (uint32_t)h.cap - 1};
        int32_t bo = 0, bi = 0;
        for (int j = 0; j < ch; ++j) { bo += hitem_out[h.first_item + j]; bi += hitem_in[h.first_item + j]; }
        int64_t xb = xoff[h.row];
        for (int64_t base = lo; base < hi; base += NT) {
            int64_t e = base + tid;
            bool act = e < hi;
            int32_t u = act ? col[b + e] : -1;
            NodeRec ru{0, -1, 0};
            if (act) ru = rec[u];
            bool cross = act && ru.label != rw.label;
            df sig{0.0f, 0.0f};
            if (cross) {
                int s = tab_find(t, ru.label);
                if (s < 0) { atomicOr(err, 8); cross = false; }
                else {
                    int64_t gs = h.tab + s;
                    sig = hsig[gs];
                    if (hcnt[gs] > 1) {
                        u128 q = ((u128)hq[2 * gs + 1] << 64) | hq[2 * gs];
                        push_type2(acc, u, sig, q - ru.s_fix);
                    }
                }
            }
            if (rw.dx >= 2) {
                bool inx = cross && ru.dx >= 2;
                bool o = inx && rank_after(ru.dx, u, rw.dx, h.row);
                gx_round<NT>(o, inx && !o, xb, rw.dx, u, sig, bo, bi, xcol, xS, sh_cnt);
            }
        }
    }
}

// ======================================================================================
// P3: Type-I triads from G_x triangles
// ======================================================================================
__device__ __forceinline__ int64_t find_out(const int32_t *xcol, int64_t lo, int64_t hi, int32_t key) {
    while (lo < hi) {
        int64_t mid = lo + ((hi - lo) >> 1);
        if (xcol[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}
// S(x -> y) for an in-neighbour y of x: the in-list sits at the back of x's
// slots in descending position order of ascending ids
__device__ __forceinline__ df in_value(const int64_t *xoff, const int32_t *xcol, const df *xS,
                                       const int32_t *xin, const NodeRec *rec, int32_t x, int32_t y,
                                       int *err) {
    int64_t end = xoff[x] + rec[x].dx - 1;      // position of in-rank 0
    int32_t lo = 0, hi = xin[x];
    while (lo < hi) {
        int32_t mid = (lo + hi) >> 1;
        if (xcol[end - mid] < y) lo = mid + 1; else hi = mid;
    }
    if (lo < xin[x] && xcol[end - lo] == y) return xS[end - lo];
    atomicOr(err, 16);
    return df{0.0f, 0.0f};
}

__global__ void __launch_bounds__(kThreads) p3_triangles_kernel(
    int64_t n, const int64_t *__restrict__ xoff, const int32_t *__restrict__ xcol, const df *__restrict__ xS,
    const int32_t *__restrict__ xout, const int32_t *__restrict__ xin, const NodeRec *__restrict__ rec,
    unsigned long long *acc, int *err) {
    int lane = threadIdx.x & 31;
    int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t av = warp; av < n; av += nwarps) {
        int32_t a = (int32_t)av;
        int32_t da = xout[a];
        if (da < 2) continue;
        int64_t ba = xoff[a];
        for (int32_t j = lane; j < da; j += 32) {
            int32_t b = xcol[ba + j];
            df Sab = xS[ba + j];
            int64_t bb = xoff[b];
            int32_t db = xout[b];
            for (int32_t tb = 0; tb < db; ++tb) {
                int32_t c = xcol[bb + tb];
                int64_t p = find_out(xcol, ba, ba + da, c);
                if (p >= ba + da || xcol[p] != c) continue;
                df Sac = xS[p], Sbc = xS[bb + tb];
                df Sba = in_value(xoff, xcol, xS, xin, rec, b, a, err);
                df Sca = in_value(xoff, xcol, xS, xin, rec, c, a, err);
                df Scb = in_value(xoff, xcol, xS, xin, rec, c, b, err);
                df ta = df_mul(df_mul(Sba, Sca), df_add(Sbc, Scb));
                df tb2 = df_mul(df_mul(Sab, Scb), df_add(Sac, Sca));
                df tc = df_mul(df_mul(Sac, Sbc), df_add(Sab, Sba));
                atomic_add_u128(acc + 2 * (int64_t)a, df_to_fixed(ta, kAccFrac));
                atomic_add_u128(acc + 2 * (int64_t)b, df_to_fixed(tb2, kAccFrac));
                atomic_add_u128(acc + 2 * (int64_t)c, df_to_fixed(tc, kAccFrac));
            }
        }
    }
}

// ======================================================================================
// finalize: R(u) = acc(u) / (w_max d (d - 1))
// ======================================================================================
__global__ void __launch_bounds__(kThreads) finalize_kernel(
    int64_t n, const int64_t *__restrict__ off, const unsigned long long *__restrict__ acc,
    const unsigned long long *__restrict__ wmax_bits, const double *__restrict__ RD, double *scores) {
    __shared__ double sW;
    if (threadIdx.x == 0) {
        double wm = __longlong_as_double((long long)*wmax_bits);
        sW = wm > 0.0 ? 1.0 / wm : 0.0;
    }
    __syncthreads();
    double W = sW;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
        int64_t d = off[u + 1] - off[u];
        double r = 0.0;
        if (d >= 2 && W > 0.0) {
            u128 s = ((u128)acc[2 * u + 1] << 64) | acc[2 * u];
            if (s) r = u128_to_double(s, -kAccFrac) * W * RD[d];
        }
        scores[u] = r;
    }
}

}  // namespace

// ======================================================================================
// host orchestration
// ======================================================================================
int rs::score_graph(rs_graph *g, double *scores, cudaStream_t s) {
    int64_t n = g->n;
    if (n == 0) return 0;
    constexpr int NT = kThreads;
    int *err = g->d_flag + 4;
    RS_CUDA_TRY(cudaMemsetAsync(g->wmax_bits, 0, sizeof(unsigned long long), s));
    RS_CUDA_TRY(cudaMemsetAsync(g->acc, 0, 2 * n * sizeof(unsigned long long), s));
    RS_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), s));
    if (g->n_hubs) {
        RS_CUDA_TRY(cudaMemsetAsync(g->hkey, 0xFF, g->hub_slots * sizeof(int32_t), s));
        RS_CUDA_TRY(cudaMemsetAsync(g->hcnt, 0, g->hub_slots * sizeof(uint32_t), s));
        RS_CUDA_TRY(cudaMemsetAsync(g->hq, 0, 2 * g->hub_slots * sizeof(unsigned long long), s));
        RS_CUDA_TRY(cudaMemsetAsync(g->hagg, 0, g->n_hubs * sizeof(HubAgg), s));
    }
    size_t p1_smem = 8 * (size_t)g->mid_cap, p2_smem = 32 * (size_t)g->mid_cap;
    static bool attr_done = false;
    if (!attr_done) {
        RS_CUDA_TRY(cudaFuncSetAttribute(p1_mid_kernel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 8 * kMidCap));
        RS_CUDA_TRY(cudaFuncSetAttribute(p2_mid_kernel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 32 * kMidCap));
        attr_done = true;
    }
    // ---- P1
    if (g->n_small) {
        p1_small_kernel<<<grid_for(g->n_small * 32, NT, 8), NT, 0, s>>>(
            g->off, g->col, g->lab, g->rows_small, g->n_small, g->k, g->LG, g->rec, g->Lall, g->wmax_bits);
        RS_CUDA_TRY(cudaGetLastError());
    }
    if (g->n_mid) {
        p1_mid_kernel<NT><<<grid_for(g->n_mid, 1, 4), NT, p1_smem, s>>>(
            g->off, g->col, g->lab, g->rows_mid, g->n_mid, g->k, g->LG, g->rec, g->Lall, g->wmax_bits, err);
        RS_CUDA_TRY(cudaGetLastError());
    }
    if (g->n_hubs) {
        hub_p1_insert_kernel<NT><<<grid_for(g->n_hub_items, 1, 8), NT, 0, s>>>(
            g->off, g->col, g->lab, g->hubs, g->hub_items, g->hub_item_chunk, g->n_hub_items, g->hkey,
            g->hcnt, g->hagg, err);
        RS_CUDA_TRY(cudaGetLastError());
        hub_p1_finish_kernel<NT><<<grid_for(g->n_hubs, 1, 8), NT, 0, s>>>(
            g->off, g->lab, g->hubs, g->n_hubs, g->k, g->LG, g->hkey, g->hcnt, g->hagg, g->rec, g->Lall,
            g->wmax_bits);
        RS_CUDA_TRY(cudaGetLastError());
    }
    // ---- G_x offsets
    gx_capacity_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(g->rec, n, g->xoff);
    RS_CUDA_TRY(cudaGetLastError());
    if (int rc = inclusive_scan_i64(g->xoff + 1, n, g->scan_tmp, s)) return rc;
    // ---- P2
    if (g->n_small) {
        p2_small_kernel<<<grid_for(g->n_small * 32, NT, 8), NT, 0, s>>>(
            g->off, g->col, g->rows_small, g->n_small, g->LG, g->rec, g->acc, g->xoff, g->xcol, g->xS,
            g->xout, g->xin);
        RS_CUDA_TRY(cudaGetLastError());
    }
    if (g->n_mid) {
        p2_mid_kernel<NT><<<grid_for(g->n_mid, 1, 4), NT, p2_smem, s>>>(
            g->off, g->col, g->rows_mid, g->n_mid, g->k, g->LG, g->rec, g->acc, g->xoff, g->xcol, g->xS,
            g->xout, g->xin, err);
        RS_CUDA_TRY(cudaGetLastError());
    }
    if (g->n_hubs) {
        hub_p2_insert_kernel<NT><<<grid_for(g->n_hub_items, 1, 8), NT, 0, s>>>(
            g->off, g->col, g->hubs, g->hub_items, g->hub_item_chunk, g->n_hub_items, g->rec, g->hkey, g->hq,
            g->hitem_out, g->hitem_in, err);
        RS_CUDA_TRY(cudaGetLastError());
        hub_p2_sigma_kernel<NT><<<grid_for(g->n_hubs, 1, 8), NT, 0, s>>>(
            g->hubs, g->n_hubs, g->LG, g->hagg, g->off, g->hkey, g->hcnt, g->hsig, g->hitem_out, g->hitem_in,
            g->xout, g->xin);
        RS_CUDA_TRY(cudaGetLastError());
        hub_p2_emit_kernel<NT><<<grid_for(g->n_hub_items, 1, 8), NT, 0, s>>>(
            g->off, g->col, g->hubs, g->hub_items, g->hub_item_chunk, g->n_hub_items, g->rec, g->hkey, g->hcnt,
            g->hq, g->hsig, g->hitem_out, g->hitem_in, g->acc, g->xoff, g->xcol, g->xS, err);
        RS_CUDA_TRY(cudaGetLastError());
    }
    // ---- P3
    p3_triangles_kernel<<<grid_for(n * 32, NT, 8), NT, 0, s>>>(n, g->xoff, g->xcol, g->xS, g->xout, g->xin,
                                                                g->rec, g->acc, err);
    RS_CUDA_TRY(cudaGetLastError());
    // ---- finalize
    finalize_kernel<<<grid_for(n, NT, 8), NT, 0, s>>>(n, g->off, g->acc, g->wmax_bits, g->RD, scores);
    RS_CUDA_TRY(cudaGetLastError());
    return 0;
}
