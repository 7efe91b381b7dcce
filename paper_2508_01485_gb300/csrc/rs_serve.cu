// rs_serve.cu -- what-if rescoring of resident graphs under node and edge
// removals, and the request loop that serves such requests concurrently.
//
// A request removes nodes (every incident edge) and edges from one resident
// base graph and asks for the new scores' top-K.  Removals are what-if: every
// request applies to the base graph, never to another request's result, so a
// result does not depend on what else is in flight.
//
// Incremental path.  Every sum of the score is an exact 128-bit fixed-point
// sum of terms, and each term is a deterministic function of a few rows.  A
// request therefore takes away the base terms that change and adds their new
// values, and obtains the bits a full rescoring of the changed graph gives:
//   T  = rows that lose an entry (removed nodes, their neighbours, edge ends):
//        recounted (interaction_matrix row, aggregates, s, dx, largest weight);
//   W  = T and its neighbours: the Type-II terms pushed by these rows are the
//        only ones that change (a row's pushes depend on its own weights and
//        on the s of its neighbours), so each row of W pushes its old terms
//        with a minus sign and its new ones with a plus sign;
//   triangles of G_x with a vertex in T: old terms taken away, and added back
//        with the new values when the triangle survives (removals only shrink
//        G_x, so no new triangle appears);
//   w_max = the largest of the untouched rows' maxima (kept from the base
//        state) and the touched rows' new maxima; finalize and top-K run over
//        all nodes, because a new w_max rescales every score.
// The kernels evaluate each term with the functions the scoring kernels use
// (rs_device.cuh), in the same operand order, so the bits agree.
//
// Full path.  A slot may instead restore a copy of the base graph, apply the
// removals and rescore it completely: the plain baseline, and the fallback for
// requests whose touched rows exceed a slot's buffers.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <vector>

#include "rs.h"
#include "rs_internal.cuh"
#include "rs_device.cuh"

using namespace rs;

#define FULL 0xFFFFFFFFu

namespace {

constexpr int32_t kInT = 1, kRemoved = 2, kInW = 4;
constexpr int kSvThreads = 256;
constexpr int kWarpTab = 256;           // per-warp table slots of the Type-II warp kernel
constexpr int kCtaTab = 1024;           // per-CTA shared table slots of the Type-II CTA kernel

// a touched row after the removals
struct __align__(16) TRow {
    NodeRec rec;                     // s', label, dx'
    uint64_t xlo, xhi;               // X' = sum_c f' LG[f']
    uint32_t T, L;                   // d', L'
    unsigned long long rowmax;       // double bits of the row's largest weight (0: none)
    int64_t tab;                     // first slot of the row's table in the pool
    int64_t xoff;                    // first entry of the row's new cross list in the pool
    uint32_t cap;                    // table slots
    int32_t xlen;                    // entries of the new cross list (= dx')
};

// frozen base state of a resident graph
struct BaseView {
    int64_t n;
    int32_t k;
    const int64_t *off;
    const int32_t *col, *lab;
    const NodeRec *rec;
    const RowSum *rsum;
    const int32_t *cl_col, *cl_lab;
    const int64_t *xoff;
    const int32_t *xcol;
    const df *xS;
    const int32_t *xout, *xin;
    const uint64_t *LG;
    const double *RD;
    const unsigned long long *rowmax;
};

// counters of a slot
enum { C_T = 0, C_WS, C_WB, C_TAB, C_X, C_WMAX, C_PAIR, C_TRI, C_NCTR = 8 };

// per-request device state of a slot
struct SlotView {
    uint32_t *dead;                  // removed CSR entries (bits)
    int32_t *flag;                   // kInT | kRemoved | kInW per node
    int32_t *tidx;                   // index in tlist (valid with kInT)
    int32_t *tlist, *wsmall, *wbig;
    int64_t tcap, wcap;
    TRow *trow;
    int32_t *tkey;                   // touched rows' tables
    uint32_t *tcnt;
    int64_t pool_cap;
    int32_t *xnew_col, *xnew_lab;    // touched rows' new cross lists
    int64_t xpool_cap;
    unsigned long long *ctr;
    unsigned long long *acc;
    double *scores;
    int32_t *hkey;                   // per-CTA global tables of the Type-II CTA kernel (large rows)
    uint32_t *hcnt;
    unsigned long long *hq;
    int64_t hub_cap;                 // slots per CTA
    int32_t *pairs;                  // (x, y): a touched node and a G_x neighbour (2 words each)
    int32_t *tris;                   // (x, y, z): base triangles through touched nodes (3 words each)
    int64_t pair_cap, tri_cap;
    int32_t *err;
};

__device__ __forceinline__ bool is_dead(const uint32_t *dead, int64_t e) { return (dead[e >> 5] >> (e & 31)) & 1u; }
__device__ __forceinline__ void set_dead(uint32_t *dead, int64_t e) { atomicOr(&dead[e >> 5], 1u << (e & 31)); }

__device__ __forceinline__ int64_t row_find(const int64_t *off, const int32_t *col, int32_t row, int32_t key) {
    int64_t lo = off[row], hi = off[row + 1], end = hi;
    while (lo < hi) {
        int64_t mid = lo + ((hi - lo) >> 1);
        if (col[mid] < key) lo = mid + 1; else hi = mid;
    }
    return (lo < end && col[lo] == key) ? lo : -1;
}

__device__ __forceinline__ uint32_t table_cap(int64_t d, int32_t k) {
    int64_t m = d < k ? d : k;
    uint32_t c = 1;
    while ((int64_t)c < 2 * m) c <<= 1;
    return c;
}

__device__ __forceinline__ void add_T(const SlotView &S, int32_t x) {
    int32_t old = atomicOr(&S.flag[x], kInT);
    if (old & kInT) return;
    unsigned long long i = atomicAdd(&S.ctr[C_T], 1ull);
    if ((int64_t)i < S.tcap) {
        S.tlist[i] = x;
        S.tidx[x] = (int32_t)i;
    } else {
        atomicOr(S.err, 1);
    }
}

// ---- 1. removals: dead entries and the touched rows ------------------------------
__global__ void sv_mark_nodes(BaseView B, SlotView S, const int32_t *nodes, int64_t m) {
    int lane = threadIdx.x & 31;
    int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = w; i < m; i += nw) {
        int32_t v = nodes[i];
        int first = 0;
        if (lane == 0) first = !(atomicOr(&S.flag[v], kRemoved) & kRemoved);
        first = __shfl_sync(FULL, first, 0);
        if (!first) continue;
        if (lane == 0) add_T(S, v);
        for (int64_t e = B.off[v] + lane; e < B.off[v + 1]; e += 32) {
            set_dead(S.dead, e);
            int32_t u = B.col[e];
            int64_t r = row_find(B.off, B.col, u, v);
            if (r >= 0) set_dead(S.dead, r);
            add_T(S, u);
        }
    }
}

__global__ void sv_mark_edges(BaseView B, SlotView S, const int32_t *src, const int32_t *dst, int64_t m) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        int32_t a = src[i], b = dst[i];
        if (a == b) continue;
        int64_t e = row_find(B.off, B.col, a, b);
        if (e < 0) continue;                          // not an edge: nothing to remove
        set_dead(S.dead, e);
        int64_t r = row_find(B.off, B.col, b, a);
        if (r >= 0) set_dead(S.dead, r);
        add_T(S, a);
        add_T(S, b);
    }
}

// ---- block reductions ------------------------------------------------------------
__device__ __forceinline__ uint32_t blk_sum_u32(uint32_t v, uint32_t *sh) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    uint32_t t = 0;
    for (int j = 0; j < nw; ++j) t += sh[j];
    return t;
}
__device__ __forceinline__ u128 blk_sum_u128(u128 v, u128 *sh) {
    v = warp_sum_u128(v);
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    u128 t = 0;
    for (int j = 0; j < nw; ++j) t += sh[j];
    return t;
}
__device__ __forceinline__ df blk_max_df(df v, df *sh) {
    v = warp_max_df(v);
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    df t{0.0f, 0.0f};
    for (int j = 0; j < nw; ++j) t = df_max(t, sh[j]);
    return t;
}

// the largest weight, s and record of a row from its counts (table + own), as P1 computes them
__device__ void finish_row(const Tab &t, uint32_t cap, uint32_t own, uint32_t alive, int32_t cv, int32_t k,
                           const uint64_t *LG, RowAgg &a, NodeRec &rec, df &m, uint32_t *sh_u32, u128 *sh_u128,
                           df *sh_df) {
    uint32_t Lf = 0;
    u128 X = 0;
    for (uint32_t j = threadIdx.x; j < cap; j += blockDim.x)
        if (t.key[j] != kEmpty) { Lf++; X += (u128)t.cnt[j] * LG[t.cnt[j]]; }
    Lf = blk_sum_u32(Lf, sh_u32);
    X = blk_sum_u128(X, sh_u128);
    a = RowAgg{alive, Lf + (own > 0 ? 1u : 0u), X + (u128)own * LG[own]};
    df cm{0.0f, 0.0f};
    for (uint32_t j = threadIdx.x; j < cap; j += blockDim.x)
        if (t.key[j] != kEmpty) cm = df_max(cm, column_weight(a, t.cnt[j], LG));
    cm = blk_max_df(cm, sh_df);
    df wown{0.0f, 0.0f};
    if (own > 0) { wown = column_weight(a, own, LG); cm = df_max(cm, wown); }
    m = p1_row_result(a, own, cm, k, LG, rec, cv, wown, true);
}

// ---- 2. touched rows: recount without the dead entries -----------------------------
__global__ void __launch_bounds__(kSvThreads) sv_trows(BaseView B, SlotView S) {
    __shared__ uint32_t sh_u32[kSvThreads / 32];
    __shared__ u128 sh_u128[kSvThreads / 32];
    __shared__ df sh_df[kSvThreads / 32];
    __shared__ long long sh_tab, sh_x;
    __shared__ int sh_n, sh_ok;
    int64_t nT = min((int64_t)*(volatile unsigned long long *)&S.ctr[C_T], S.tcap);
    for (int64_t i = blockIdx.x; i < nT; i += gridDim.x) {
        int32_t x = S.tlist[i];
        int64_t b = B.off[x];
        int64_t d = B.off[x + 1] - b;
        int32_t cv = B.lab[x];
        uint32_t cap = table_cap(d, B.k);
        __syncthreads();
        if (threadIdx.x == 0) {
            sh_tab = (long long)atomicAdd(&S.ctr[C_TAB], (unsigned long long)cap);
            sh_x = (long long)atomicAdd(&S.ctr[C_X], (unsigned long long)d);
            sh_ok = sh_tab + cap <= S.pool_cap && sh_x + d <= S.xpool_cap;
            if (!sh_ok) atomicOr(S.err, 2);
            sh_n = 0;
        }
        __syncthreads();
        if (!sh_ok) {                                  // never read outside the pools (the request fails)
            if (threadIdx.x == 0) {
                TRow r{};
                r.rec.label = cv;
                S.trow[i] = r;
            }
            continue;
        }
        int64_t tab = sh_tab, xo = sh_x;
        Tab t{S.tkey + tab, S.tcnt + tab, nullptr, nullptr, cap - 1};
        for (uint32_t j = threadIdx.x; j < cap; j += blockDim.x) { t.key[j] = kEmpty; t.cnt[j] = 0; }
        __syncthreads();
        uint32_t own = 0, alive = 0;
        for (int64_t e = threadIdx.x; e < d; e += blockDim.x) {
            if (is_dead(S.dead, b + e)) continue;
            alive++;
            int32_t u = B.col[b + e];
            int32_t c = B.lab[u];
            if (c == cv) { own++; continue; }
            tab_insert(t, c, 1, S.err);
            int p = atomicAdd(&sh_n, 1);
            S.xnew_col[xo + p] = u;
            S.xnew_lab[xo + p] = c;
        }
        own = blk_sum_u32(own, sh_u32);              // syncs: the table is complete
        alive = blk_sum_u32(alive, sh_u32);
        RowAgg a;
        NodeRec rec;
        df m;
        finish_row(t, cap, own, alive, cv, B.k, B.LG, a, rec, m, sh_u32, sh_u128, sh_df);
        if (threadIdx.x == 0) {
            TRow r;
            r.rec = rec;
            r.xlo = (uint64_t)a.X;
            r.xhi = (uint64_t)(a.X >> 64);
            r.T = a.T;
            r.L = a.L;
            r.rowmax = m.hi > 0.0f ? double_bits(m) : 0ull;
            r.tab = tab;
            r.xoff = xo;
            r.cap = cap;
            r.xlen = sh_n;
            S.trow[i] = r;
        }
    }
}

// ---- 3. W = T and its neighbours, split by table size --------------------------------
__device__ __forceinline__ void add_W(const BaseView &B, const SlotView &S, int32_t u) {
    int32_t old = atomicOr(&S.flag[u], kInW);
    if (old & kInW) return;
    int64_t d = B.off[u + 1] - B.off[u];
    bool small = table_cap(d, B.k) <= (uint32_t)kWarpTab;
    unsigned long long i = atomicAdd(&S.ctr[small ? C_WS : C_WB], 1ull);
    if ((int64_t)i < S.wcap) (small ? S.wsmall : S.wbig)[i] = u;
    else atomicOr(S.err, 4);
}

__global__ void __launch_bounds__(kSvThreads) sv_mark_w(BaseView B, SlotView S) {
    int64_t nT = min((int64_t)S.ctr[C_T], S.tcap);
    for (int64_t i = blockIdx.x; i < nT; i += gridDim.x) {          // a CTA per touched row
        int32_t x = S.tlist[i];
        if (threadIdx.x == 0) add_W(B, S, x);
        for (int64_t e = B.off[x] + threadIdx.x; e < B.off[x + 1]; e += blockDim.x) add_W(B, S, B.col[e]);
    }
}

// ---- 4. Type-II: old pushes of W rows taken away, new pushes added ------------------
struct RowSide {
    const int32_t *ucol, *ulab;      // cross list (ids, labels)
    int32_t len;
    RowAgg a;
};

__device__ __forceinline__ RowSide old_side(const BaseView &B, int32_t w) {
    int64_t b = B.off[w];
    RowSum rs = B.rsum[w];
    return RowSide{B.cl_col + b, B.cl_lab + b, B.rec[w].dx,
                   RowAgg{(uint32_t)(B.off[w + 1] - b), rs.L, ((u128)rs.xhi << 64) | rs.xlo}};
}
__device__ __forceinline__ RowSide new_side(const BaseView &B, const SlotView &S, int32_t w) {
    if (!(S.flag[w] & kInT)) return old_side(B, w);
    TRow r = S.trow[S.tidx[w]];
    return RowSide{S.xnew_col + r.xoff, S.xnew_lab + r.xoff, r.xlen, RowAgg{r.T, r.L, ((u128)r.xhi << 64) | r.xlo}};
}
__device__ __forceinline__ uint64_t s_new(const BaseView &B, const SlotView &S, int32_t x) {
    return (S.flag[x] & kInT) ? S.trow[S.tidx[x]].rec.s_fix : B.rec[x].s_fix;
}

// A row w of W that is not touched keeps its cross list and weights; only the
// communities of its touched cross neighbours get new group sums Q_w(c), so only
// the terms it pushes to those communities change.  Such rows mark these
// communities in the table first (count 0) and both sides then take only the
// entries of marked communities.  A touched row redoes every entry.

// warp: mark the affected communities of an untouched row
__device__ __forceinline__ void mark_affected_warp(const SlotView &S, const RowSide &R, Tab t, uint32_t cap,
                                                   int lane) {
    for (uint32_t j = lane; j < cap; j += 32) t.key[j] = kEmpty;
    __syncwarp();
    for (int32_t e = lane; e < R.len; e += 32)
        if (S.flag[R.ucol[e]] & kInT) tab_insert(t, R.ulab[e], 0, S.err);
    __syncwarp();
}

// one side of a row on a warp: group sums by community, then every pushed term
__device__ void type2_side_warp(const BaseView &B, const SlotView &S, const RowSide &R, bool neg, bool filter,
                                Tab t, uint32_t cap, int lane) {
    for (uint32_t j = lane; j < cap; j += 32) {
        if (!filter) t.key[j] = kEmpty;
        t.cnt[j] = 0; t.q[2 * j] = 0; t.q[2 * j + 1] = 0;
    }
    __syncwarp();
    for (int32_t e = lane; e < R.len; e += 32) {
        int32_t x = R.ucol[e];
        int sl;
        if (filter) {
            sl = tab_find(t, R.ulab[e]);
            if (sl < 0) continue;
            atomicAdd(&t.cnt[sl], 1u);
        } else {
            sl = tab_insert(t, R.ulab[e], 1, S.err);
        }
        if (sl >= 0) atomic_add_u128(t.q + 2 * sl, (u128)(neg ? B.rec[x].s_fix : s_new(B, S, x)));
    }
    __syncwarp();
    for (int32_t e = lane; e < R.len; e += 32) {
        int32_t u = R.ucol[e];
        int sl = tab_find(t, R.ulab[e]);
        if (sl < 0) { if (!filter) atomicOr(S.err, 8); continue; }
        uint32_t f = t.cnt[sl];
        if (f < 2) continue;                           // Q - s_u = 0
        u128 q = ((u128)t.q[2 * sl + 1] << 64) | t.q[2 * sl];
        uint64_t su = neg ? B.rec[u].s_fix : s_new(B, S, u);
        push_type2(S.acc, u, df_cbrt(column_weight(R.a, f, B.LG)), q - su, neg);
    }
    __syncwarp();
}

__global__ void __launch_bounds__(kSvThreads) sv_type2_warp(BaseView B, SlotView S) {
    __shared__ int32_t skey[kSvThreads / 32][kWarpTab];
    __shared__ uint32_t scnt[kSvThreads / 32][kWarpTab];
    __shared__ unsigned long long sq[kSvThreads / 32][2 * kWarpTab];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int64_t nW = min((int64_t)S.ctr[C_WS], S.wcap);
    for (int64_t i = w0; i < nW; i += nw) {
        int32_t w = S.wsmall[i];
        bool touched = S.flag[w] & kInT;
        RowSide ro = old_side(B, w);
        RowSide rn = touched ? new_side(B, S, w) : ro;
        uint32_t cap = table_cap(max(ro.len, rn.len), B.k);
        Tab t{skey[wid], scnt[wid], sq[wid], nullptr, cap - 1};
        if (!touched) mark_affected_warp(S, ro, t, cap, lane);
        type2_side_warp(B, S, ro, true, !touched, t, cap, lane);
        type2_side_warp(B, S, rn, false, !touched, t, cap, lane);
    }
}

__device__ void type2_side_cta(const BaseView &B, const SlotView &S, const RowSide &R, bool neg, bool filter, Tab t,
                               uint32_t cap) {
    for (uint32_t j = threadIdx.x; j < cap; j += blockDim.x) {
        if (!filter) t.key[j] = kEmpty;
        t.cnt[j] = 0; t.q[2 * j] = 0; t.q[2 * j + 1] = 0;
    }
    __syncthreads();
    for (int32_t e = threadIdx.x; e < R.len; e += blockDim.x) {
        int32_t x = R.ucol[e];
        int sl;
        if (filter) {
            sl = tab_find(t, R.ulab[e]);
            if (sl < 0) continue;
            atomicAdd(&t.cnt[sl], 1u);
        } else {
            sl = tab_insert(t, R.ulab[e], 1, S.err);
        }
        if (sl >= 0) atomic_add_u128(t.q + 2 * sl, (u128)(neg ? B.rec[x].s_fix : s_new(B, S, x)));
    }
    __syncthreads();
    for (int32_t e = threadIdx.x; e < R.len; e += blockDim.x) {
        int32_t u = R.ucol[e];
        int sl = tab_find(t, R.ulab[e]);
        if (sl < 0) { if (!filter) atomicOr(S.err, 8); continue; }
        uint32_t f = t.cnt[sl];
        if (f < 2) continue;
        u128 q = ((u128)t.q[2 * sl + 1] << 64) | t.q[2 * sl];
        uint64_t su = neg ? B.rec[u].s_fix : s_new(B, S, u);
        push_type2(S.acc, u, df_cbrt(column_weight(R.a, f, B.LG)), q - su, neg);
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kSvThreads) sv_type2_cta(BaseView B, SlotView S) {
    __shared__ int32_t skey[kCtaTab];
    __shared__ uint32_t scnt[kCtaTab];
    __shared__ unsigned long long sq[2 * kCtaTab];
    int64_t nW = min((int64_t)S.ctr[C_WB], S.wcap);
    for (int64_t i = blockIdx.x; i < nW; i += gridDim.x) {
        int32_t w = S.wbig[i];
        bool touched = S.flag[w] & kInT;
        RowSide ro = old_side(B, w);
        RowSide rn = touched ? new_side(B, S, w) : ro;
        uint32_t cap = table_cap(max(ro.len, rn.len), B.k);
        Tab t;
        if (cap <= (uint32_t)kCtaTab) {
            t = Tab{skey, scnt, sq, nullptr, cap - 1};
        } else {
            if ((int64_t)cap > S.hub_cap) { if (threadIdx.x == 0) atomicOr(S.err, 16); continue; }
            int64_t o = (int64_t)blockIdx.x * S.hub_cap;
            t = Tab{S.hkey + o, S.hcnt + o, S.hq + 2 * o, nullptr, cap - 1};
        }
        if (!touched) {                                  // mark the affected communities
            __syncthreads();
            for (uint32_t j = threadIdx.x; j < cap; j += blockDim.x) t.key[j] = kEmpty;
            __syncthreads();
            for (int32_t e = threadIdx.x; e < ro.len; e += blockDim.x)
                if (S.flag[ro.ucol[e]] & kInT) tab_insert(t, ro.ulab[e], 0, S.err);
            __syncthreads();
        }
        type2_side_cta(B, S, ro, true, !touched, t, cap);
        type2_side_cta(B, S, rn, false, !touched, t, cap);
    }
}

// ---- 5. Type-I: triangles of G_x with a touched vertex -----------------------------
__device__ __forceinline__ bool rank_lt(int32_t dx1, int32_t id1, int32_t dx2, int32_t id2) {
    return dx1 < dx2 || (dx1 == dx2 && id1 < id2);
}

// slot of q in p's base G_x lists (out-list if q ranks above p, else in-list), or -1
__device__ __forceinline__ int64_t gx_slot(const BaseView &B, int32_t p, int32_t q) {
    int32_t dxp = B.rec[p].dx, dxq = B.rec[q].dx;
    int64_t base = B.xoff[p];
    if (rank_lt(dxp, p, dxq, q)) {
        int32_t l = 0, h = B.xout[p];
        while (l < h) {
            int32_t mid = (l + h) >> 1;
            if (B.xcol[base + mid] < q) l = mid + 1; else h = mid;
        }
        return (l < B.xout[p] && B.xcol[base + l] == q) ? base + l : -1;
    }
    int64_t end = base + dxp - 1;                       // in-rank 0 at the last slot
    int32_t l = 0, h = B.xin[p];
    while (l < h) {
        int32_t mid = (l + h) >> 1;
        if (B.xcol[end - mid] < q) l = mid + 1; else h = mid;
    }
    return (l < B.xin[p] && B.xcol[end - l] == q) ? end - l : -1;
}

__device__ __forceinline__ df s_base(const BaseView &B, const SlotView &S, int32_t p, int32_t q) {
    int64_t sl = gx_slot(B, p, q);
    if (sl < 0) { atomicOr(S.err, 32); return df{0.0f, 0.0f}; }
    return B.xS[sl];
}

// S'(p -> q) after the removals
__device__ __forceinline__ df s_after(const BaseView &B, const SlotView &S, int32_t p, int32_t q) {
    if (!(S.flag[p] & kInT)) return s_base(B, S, p, q);
    TRow r = S.trow[S.tidx[p]];
    if (r.cap == 0) return df{0.0f, 0.0f};
    Tab t{S.tkey + r.tab, S.tcnt + r.tab, nullptr, nullptr, r.cap - 1};
    int sl = tab_find(t, B.lab[q]);
    uint32_t f = sl >= 0 ? t.cnt[sl] : 0u;
    RowAgg a{r.T, r.L, ((u128)r.xhi << 64) | r.xlo};
    return df_cbrt(column_weight(a, f, B.LG));
}

__device__ __forceinline__ int32_t dx_after(const BaseView &B, const SlotView &S, int32_t p) {
    return (S.flag[p] & kInT) ? S.trow[S.tidx[p]].rec.dx : B.rec[p].dx;
}

__device__ __forceinline__ bool edge_alive(const BaseView &B, const SlotView &S, int32_t p, int32_t q) {
    if (!(S.flag[p] & kInT) || !(S.flag[q] & kInT)) return true;   // a removal touches both ends
    int64_t e = row_find(B.off, B.col, p, q);
    return e >= 0 && !is_dead(S.dead, e);
}

// order three nodes by rank (dx, id) given their dx
__device__ __forceinline__ void order3(int32_t &a, int32_t &b, int32_t &c, int32_t da, int32_t db, int32_t dc) {
    if (rank_lt(db, b, da, a)) { int32_t t = a; a = b; b = t; int32_t u = da; da = db; db = u; }
    if (rank_lt(dc, c, db, b)) { int32_t t = b; b = c; c = t; int32_t u = db; db = dc; dc = u; }
    if (rank_lt(db, b, da, a)) { int32_t t = a; a = b; b = t; int32_t u = da; da = db; db = u; }
}

__device__ void triangle_delta(const BaseView &B, const SlotView &S, int32_t x, int32_t y, int32_t z) {
    // old terms, by base rank
    int32_t a = x, b = y, c = z;
    order3(a, b, c, B.rec[a].dx, B.rec[b].dx, B.rec[c].dx);
    TriTerms to = triangle_term_values(s_base(B, S, a, b), s_base(B, S, b, a), s_base(B, S, a, c),
                                       s_base(B, S, c, a), s_base(B, S, b, c), s_base(B, S, c, b));
    add_triangle(S.acc, a, b, c, to, true);
    // new terms, when the triangle survives, by new rank
    int32_t dxa = dx_after(B, S, x), dxb = dx_after(B, S, y), dxc = dx_after(B, S, z);
    if (dxa < 2 || dxb < 2 || dxc < 2) return;
    if (!edge_alive(B, S, x, y) || !edge_alive(B, S, x, z) || !edge_alive(B, S, y, z)) return;
    a = x; b = y; c = z;
    order3(a, b, c, dxa, dxb, dxc);
    TriTerms tn = triangle_term_values(s_after(B, S, a, b), s_after(B, S, b, a), s_after(B, S, a, c),
                                       s_after(B, S, c, a), s_after(B, S, b, c), s_after(B, S, c, b));
    add_triangle(S.acc, a, b, c, tn, false);
}

// the base G_x neighbour of p with list index j (out-list first, then in-list)
__device__ __forceinline__ int32_t gx_nbr(const BaseView &B, int32_t p, int32_t j, int32_t nout) {
    int64_t base = B.xoff[p];
    if (j < nout) return B.xcol[base + j];
    return B.xcol[base + B.rec[p].dx - 1 - (j - nout)];
}

// 5a. pairs (x, y): x touched, y a base G_x neighbour of x; a triangle through
//     several touched nodes belongs to the smallest of them, so y is skipped when
//     it is touched and smaller than x
__global__ void __launch_bounds__(kSvThreads) sv_tri_pairs(BaseView B, SlotView S) {
    int lane = threadIdx.x & 31;
    int64_t nT = min((int64_t)S.ctr[C_T], S.tcap);
    for (int64_t i = blockIdx.x; i < nT; i += gridDim.x) {              // a CTA per touched row
        int32_t x = S.tlist[i];
        if (B.rec[x].dx < 2) continue;                  // not in G_x: no base triangle
        int32_t xo = B.xout[x], xi = B.xin[x];
        for (int32_t j0 = 0; j0 < xo + xi; j0 += blockDim.x) {
            int32_t j = j0 + threadIdx.x;
            bool keep = false;
            int32_t y = 0;
            if (j < xo + xi) {
                y = gx_nbr(B, x, j, xo);
                keep = !((S.flag[y] & kInT) && y < x);
            }
            unsigned m = __ballot_sync(FULL, keep);
            unsigned long long b0 = 0;
            if (lane == 0 && m) b0 = atomicAdd(&S.ctr[C_PAIR], (unsigned long long)__popc(m));
            b0 = __shfl_sync(FULL, b0, 0);
            if (keep) {
                unsigned long long p = b0 + __popc(m & ((1u << lane) - 1));
                if ((int64_t)p < S.pair_cap) { S.pairs[2 * p] = x; S.pairs[2 * p + 1] = y; }
                else atomicOr(S.err, 64);
            }
        }
    }
}

// is q a base G_x neighbour of p (either list)
__device__ __forceinline__ bool gx_adj(const BaseView &B, int32_t p, int32_t q) { return gx_slot(B, p, q) >= 0; }

// 5b. a warp per pair (x, y): the common G_x neighbours z > y of x and y (the
//     lanes walk the shorter list, each z searched in the longer), each a base
//     triangle {x, y, z}
__global__ void __launch_bounds__(kSvThreads) sv_tri_find(BaseView B, SlotView S) {
    int lane = threadIdx.x & 31;
    int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nwp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int64_t nP = min((int64_t)S.ctr[C_PAIR], S.pair_cap);
    for (int64_t i = w0; i < nP; i += nwp) {
        int32_t x = S.pairs[2 * i], y = S.pairs[2 * i + 1];
        int32_t nx = B.xout[x] + B.xin[x], ny = B.xout[y] + B.xin[y];
        bool walk_x = nx <= ny;
        int32_t w = walk_x ? x : y, o = walk_x ? y : x;
        int32_t wo = B.xout[w], len = walk_x ? nx : ny;
        for (int32_t j = lane; j < len; j += 32) {
            int32_t z = gx_nbr(B, w, j, wo);
            if (z <= y || z == x) continue;
            if ((S.flag[z] & kInT) && z < x) continue;
            if (!gx_adj(B, o, z)) continue;
            unsigned long long t = atomicAdd(&S.ctr[C_TRI], 1ull);
            if ((int64_t)t < S.tri_cap) { S.tris[3 * t] = x; S.tris[3 * t + 1] = y; S.tris[3 * t + 2] = z; }
            else triangle_delta(B, S, x, y, z);          // buffer full: finish it here
        }
    }
}

// 5c. one thread per triangle: old terms away, new ones back if it survives
__global__ void __launch_bounds__(kSvThreads) sv_tri_delta(BaseView B, SlotView S) {
    int64_t nt = min((int64_t)S.ctr[C_TRI], S.tri_cap);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nt; i += (int64_t)gridDim.x * blockDim.x)
        triangle_delta(B, S, S.tris[3 * i], S.tris[3 * i + 1], S.tris[3 * i + 2]);
}

// ---- 6. w_max, finalize ----------------------------------------------------------------
__global__ void __launch_bounds__(kSvThreads) sv_wmax(BaseView B, SlotView S) {
    unsigned long long m = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < B.n; v += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long r = (S.flag[v] & kInT) ? S.trow[S.tidx[v]].rowmax : B.rowmax[v];
        m = r > m ? r : m;
    }
    for (int o = 16; o; o >>= 1) {
        unsigned long long y = __shfl_xor_sync(FULL, m, o);
        m = y > m ? y : m;
    }
    if ((threadIdx.x & 31) == 0 && m) atomicMax(&S.ctr[C_WMAX], m);
}

__global__ void __launch_bounds__(kSvThreads) sv_finalize(BaseView B, SlotView S) {
    double wm = __longlong_as_double((long long)S.ctr[C_WMAX]);
    double W = wm > 0.0 ? 1.0 / wm : 0.0;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < B.n; u += (int64_t)gridDim.x * blockDim.x) {
        int64_t d = (S.flag[u] & kInT) ? (int64_t)S.trow[S.tidx[u]].T : B.off[u + 1] - B.off[u];
        double r = 0.0;
        if (d >= 2) {
            u128 s = ((u128)S.acc[2 * u + 1] << 64) | S.acc[2 * u];
            if (s && W > 0.0) r = u128_to_double(s, -kAccFrac) * W * B.RD[d];
        }
        S.scores[u] = r;
    }
}

// ---- base preparation: 2-hop degree sums (admission bounds), every row's largest weight ------
__global__ void sv_deg2(BaseView B, int64_t *d2) {
    int lane = threadIdx.x & 31;
    int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = w; v < B.n; v += nw) {
        int64_t s = 0;
        for (int64_t e = B.off[v] + lane; e < B.off[v + 1]; e += 32) {
            int32_t u = B.col[e];
            s += B.off[u + 1] - B.off[u];
        }
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
        if (lane == 0) d2[v] = s;
    }
}

// Every row recounted once: its largest weight, and its aggregates and cross list
// written where the incremental kernels read them.  (The scoring path's hub rows
// keep their aggregates and cross lists elsewhere: they are rewritten here for
// every row, with the same values for the other rows.)
__global__ void __launch_bounds__(kSvThreads) sv_rowmax_all(BaseView B, int32_t *tkey, uint32_t *tcnt,
                                                            int64_t per_cta, unsigned long long *rowmax,
                                                            RowSum *rsum, int32_t *cl_col, int32_t *cl_lab,
                                                            int *err) {
    __shared__ uint32_t sh_u32[kSvThreads / 32];
    __shared__ u128 sh_u128[kSvThreads / 32];
    __shared__ df sh_df[kSvThreads / 32];
    __shared__ int sh_n;
    int64_t o = (int64_t)blockIdx.x * per_cta;
    for (int64_t x = blockIdx.x; x < B.n; x += gridDim.x) {
        int64_t b = B.off[x];
        int64_t d = B.off[x + 1] - b;
        int32_t cv = B.lab[x];
        uint32_t cap = table_cap(d, B.k);
        Tab t{tkey + o, tcnt + o, nullptr, nullptr, cap - 1};
        __syncthreads();
        if (threadIdx.x == 0) sh_n = 0;
        for (uint32_t j = threadIdx.x; j < cap; j += blockDim.x) { t.key[j] = kEmpty; t.cnt[j] = 0; }
        __syncthreads();
        uint32_t own = 0;
        for (int64_t e = threadIdx.x; e < d; e += blockDim.x) {
            int32_t u = B.col[b + e];
            int32_t c = B.lab[u];
            if (c == cv) { own++; continue; }
            tab_insert(t, c, 1, err);
            int p = atomicAdd(&sh_n, 1);
            cl_col[b + p] = u;
            cl_lab[b + p] = c;
        }
        own = blk_sum_u32(own, sh_u32);
        RowAgg a;
        NodeRec rec;
        df m;
        finish_row(t, cap, own, (uint32_t)d, cv, B.k, B.LG, a, rec, m, sh_u32, sh_u128, sh_df);
        if (threadIdx.x == 0) {
            rowmax[x] = m.hi > 0.0f ? double_bits(m) : 0ull;
            RowSum r;
            r.xlo = (uint64_t)a.X;
            r.xhi = (uint64_t)(a.X >> 64);
            r.L = a.L;
            r.pad = 0;
            rsum[x] = r;
            if (rec.s_fix != B.rec[x].s_fix || rec.dx != B.rec[x].dx) atomicOr(err, 2);
        }
    }
}

}  // namespace

// ======================================================================================
// host side: resident bases, slots, the request loop
// ======================================================================================
namespace {

int sm_count() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

template <class T>
cudaError_t dalloc(T **p, size_t count, int64_t &bytes) {
    size_t b = std::max<size_t>(count, 1) * sizeof(T);
    bytes += (int64_t)b;
    return cudaMalloc((void **)p, b);
}

struct Base {
    rs_graph *g = nullptr;            // owned; its scoring state stays frozen
    int64_t n = 0, nnz = 0;
    int32_t k = 0, dmax = 0;
    unsigned long long *acc = nullptr;     // raw sums of the base graph
    double *scores = nullptr;
    unsigned long long *rowmax = nullptr;
    std::vector<int32_t> deg;              // host: degrees
    std::vector<int64_t> d2;               // host: sum of the neighbours' degrees
    BaseView view() const {
        BaseView v;
        v.n = n; v.k = k; v.off = g->off; v.col = g->col; v.lab = g->lab; v.rec = g->rec; v.rsum = g->rsum;
        v.cl_col = g->cl_col; v.cl_lab = g->cl_lab; v.xoff = g->xoff; v.xcol = g->xcol; v.xS = g->xS;
        v.xout = g->xout; v.xin = g->xin; v.LG = g->LG; v.RD = g->RD; v.rowmax = rowmax;
        return v;
    }
};

struct Request {
    int64_t ticket = 0;
    int32_t graph = 0, top_k = 0;
    std::vector<int32_t> nodes, src, dst;
};

struct Slot {
    cudaStream_t s = nullptr;
    cudaEvent_t done = nullptr;
    int64_t bytes = 0;
    // incremental buffers
    SlotView v{};
    int32_t *d_req = nullptr;          // removal lists on the device
    int64_t req_cap = 0;
    int32_t *h_req = nullptr;          // pinned staging
    int32_t *ids = nullptr;
    double *vals = nullptr;
    int32_t *h_ids = nullptr;          // pinned results
    double *h_vals = nullptr;
    int32_t *h_err = nullptr;
    rs_graph *tk = nullptr;            // holds the top-K workspace
    // full path: the copy of the base graph the request in flight uses (index in the pool)
    int32_t copy = -1;
    // the request in flight
    bool busy = false;
    Request req;
    int32_t path = 0;                  // 1 incremental, 0 full
    int32_t status = RS_OK;
};

}  // namespace

// a full copy of a base graph, for the full path
struct Copy {
    rs_graph *g = nullptr;
    int32_t graph = -1;
    int64_t bytes = 0;
    bool busy = false;
    uint64_t last_use = 0;
};

struct rs_server {
    std::vector<Base> bases;
    std::vector<Slot> slots;
    std::vector<Copy> copies;
    uint64_t clock = 0;
    std::deque<Request> queue;
    int32_t mode = RS_SERVE_INCREMENTAL;
    int32_t max_top_k = 0;
    int64_t budget = 0, used = 0;
    int64_t next_ticket = 1;
    int64_t n_max = 0, nnz_max = 0, hub_cap = 0;
    int64_t tcap = 0, xcap = 0;
};

namespace {

int prepare_base(Base &b) {
    rs_graph *g = b.g;
    if (g->n_graphs != 1) return fail(RS_EINVAL, "rs_server_create: batches are not served (build single graphs)");
    if (g->perm) return fail(RS_EINVAL, "rs_server_create: graphs built with RS_REORDER are not served");
    b.n = g->n; b.nnz = g->nnz; b.k = g->k; b.dmax = g->dmax;
    int64_t unused = 0;
    RS_CUDA_TRY(dalloc(&b.acc, 2 * (size_t)b.n, unused));
    RS_CUDA_TRY(dalloc(&b.scores, (size_t)b.n, unused));
    RS_CUDA_TRY(dalloc(&b.rowmax, (size_t)b.n, unused));
    cudaStream_t s = nullptr;
    RS_CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    int rc = 0;
    if (b.n > 0) rc = score_graph(g, b.scores, s);
    int64_t *d2 = nullptr;
    int32_t *ktab = nullptr;
    uint32_t *ctab = nullptr;
    int *err = nullptr;
    if (!rc && b.n > 0) {
        cudaError_t e = cudaMemcpyAsync(b.acc, g->acc, 2 * b.n * sizeof(unsigned long long), cudaMemcpyDeviceToDevice, s);
        int grid = 2 * sm_count();
        int64_t per = 1;
        { int64_t m = std::min<int64_t>(b.dmax, b.k); while (per < 2 * m) per <<= 1; }
        if (!e) e = dalloc(&ktab, (size_t)(grid * per), unused);
        if (!e) e = dalloc(&ctab, (size_t)(grid * per), unused);
        if (!e) e = dalloc(&err, 1, unused);
        if (!e) e = dalloc(&d2, (size_t)b.n, unused);
        if (!e) e = cudaMemsetAsync(err, 0, sizeof(int), s);
        if (!e) {
            BaseView v = b.view();
            sv_rowmax_all<<<grid, kSvThreads, 0, s>>>(v, ktab, ctab, per, b.rowmax, g->rsum, g->cl_col, g->cl_lab,
                                                      err);
            e = cudaGetLastError();
            if (!e) {
                sv_deg2<<<grid_for(b.n * 32, kSvThreads, 8), kSvThreads, 0, s>>>(v, d2);
                e = cudaGetLastError();
            }
        }
        std::vector<int64_t> off(b.n + 1);
        int h_err = 0;
        b.d2.resize(b.n);
        if (!e) e = cudaMemcpyAsync(off.data(), g->off, (b.n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s);
        if (!e) e = cudaMemcpyAsync(b.d2.data(), d2, b.n * sizeof(int64_t), cudaMemcpyDeviceToHost, s);
        if (!e) e = cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (!e) e = cudaStreamSynchronize(s);
        if (e) rc = cuda_fail(e, "rs_server_create: base state");
        else if (h_err) rc = fail(RS_ECUDA, "rs_server_create: base state check failed (internal)");
        b.deg.resize(b.n);
        for (int64_t i = 0; i < b.n; ++i) b.deg[i] = (int32_t)(off[i + 1] - off[i]);
    }
    cudaFree(d2); cudaFree(ktab); cudaFree(ctab); cudaFree(err);
    cudaStreamDestroy(s);
    return rc;
}

void free_slot(Slot &sl) {
    cudaFree(sl.v.dead); cudaFree(sl.v.flag); cudaFree(sl.v.tidx); cudaFree(sl.v.tlist); cudaFree(sl.v.wsmall);
    cudaFree(sl.v.wbig); cudaFree(sl.v.trow); cudaFree(sl.v.tkey); cudaFree(sl.v.tcnt); cudaFree(sl.v.xnew_col);
    cudaFree(sl.v.xnew_lab); cudaFree(sl.v.ctr); cudaFree(sl.v.acc); cudaFree(sl.v.scores); cudaFree(sl.v.hkey);
    cudaFree(sl.v.hcnt); cudaFree(sl.v.hq); cudaFree(sl.v.pairs); cudaFree(sl.v.tris); cudaFree(sl.v.err); cudaFree(sl.d_req); cudaFree(sl.ids); cudaFree(sl.vals);
    cudaFreeHost(sl.h_req); cudaFreeHost(sl.h_ids); cudaFreeHost(sl.h_vals); cudaFreeHost(sl.h_err);
    if (sl.tk) rs_free_graph(sl.tk);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.s) cudaStreamDestroy(sl.s);
    sl = Slot();
}

int alloc_slot(rs_server *srv, Slot &sl) {
    int64_t &b = sl.bytes;
    int64_t n = srv->n_max, nnz = srv->nnz_max;
    SlotView &v = sl.v;
    v.tcap = srv->tcap;
    v.wcap = n;
    v.xpool_cap = srv->xcap;
    v.pool_cap = 4 * srv->xcap + 2 * srv->tcap;
    v.hub_cap = srv->hub_cap;
    RS_CUDA_TRY(cudaStreamCreateWithFlags(&sl.s, cudaStreamNonBlocking));
    RS_CUDA_TRY(cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming));
    RS_CUDA_TRY(dalloc(&v.dead, (size_t)((nnz + 31) / 32), b));
    RS_CUDA_TRY(dalloc(&v.flag, (size_t)n, b));
    RS_CUDA_TRY(dalloc(&v.tidx, (size_t)n, b));
    RS_CUDA_TRY(dalloc(&v.tlist, (size_t)v.tcap, b));
    RS_CUDA_TRY(dalloc(&v.wsmall, (size_t)v.wcap, b));
    RS_CUDA_TRY(dalloc(&v.wbig, (size_t)v.wcap, b));
    RS_CUDA_TRY(dalloc(&v.trow, (size_t)v.tcap, b));
    RS_CUDA_TRY(dalloc(&v.tkey, (size_t)v.pool_cap, b));
    RS_CUDA_TRY(dalloc(&v.tcnt, (size_t)v.pool_cap, b));
    RS_CUDA_TRY(dalloc(&v.xnew_col, (size_t)v.xpool_cap, b));
    RS_CUDA_TRY(dalloc(&v.xnew_lab, (size_t)v.xpool_cap, b));
    RS_CUDA_TRY(dalloc(&v.ctr, (size_t)C_NCTR, b));
    RS_CUDA_TRY(dalloc(&v.acc, 2 * (size_t)n, b));
    RS_CUDA_TRY(dalloc(&v.scores, (size_t)n, b));
    int64_t hub_slots = v.hub_cap > kCtaTab ? v.hub_cap * 4 * sm_count() : 1;
    RS_CUDA_TRY(dalloc(&v.hkey, (size_t)hub_slots, b));
    RS_CUDA_TRY(dalloc(&v.hcnt, (size_t)hub_slots, b));
    RS_CUDA_TRY(dalloc(&v.hq, 2 * (size_t)hub_slots, b));
    v.pair_cap = srv->xcap;
    v.tri_cap = srv->xcap;
    RS_CUDA_TRY(dalloc(&v.pairs, 2 * (size_t)v.pair_cap, b));
    RS_CUDA_TRY(dalloc(&v.tris, 3 * (size_t)v.tri_cap, b));
    RS_CUDA_TRY(dalloc(&v.err, 1, b));
    sl.req_cap = 1 << 16;
    RS_CUDA_TRY(dalloc(&sl.d_req, (size_t)sl.req_cap, b));
    RS_CUDA_TRY(cudaMallocHost((void **)&sl.h_req, sl.req_cap * sizeof(int32_t)));
    int32_t kk = std::max(srv->max_top_k, 1);
    RS_CUDA_TRY(dalloc(&sl.ids, (size_t)kk, b));
    RS_CUDA_TRY(dalloc(&sl.vals, (size_t)kk, b));
    RS_CUDA_TRY(cudaMallocHost((void **)&sl.h_ids, kk * sizeof(int32_t)));
    RS_CUDA_TRY(cudaMallocHost((void **)&sl.h_vals, kk * sizeof(double)));
    RS_CUDA_TRY(cudaMallocHost((void **)&sl.h_err, sizeof(int32_t)));
    sl.tk = new rs_graph();
    sl.tk->n = n;
    if (int rc = topk_prepare(sl.tk, n)) return rc;
    b += (2 * n + 16384) * 12 + 64;
    return 0;
}

// bounds of the touched rows of a request, from degrees and 2-hop degree sums
struct Bounds { int64_t t, dt; };
Bounds request_bounds(const Base &b, const Request &r) {
    Bounds x{0, 0};
    for (int32_t v : r.nodes) { x.t += 1 + b.deg[v]; x.dt += b.deg[v] + b.d2[v]; }
    for (size_t i = 0; i < r.src.size(); ++i) {
        x.t += 2;
        x.dt += (int64_t)b.deg[r.src[i]] + b.deg[r.dst[i]];
    }
    return x;
}

bool fits_buffers(const rs_server *srv, const Base &b, const Request &r) {
    if (b.g->strict) return false;       // the delta kernels follow the default triad reading
    if ((int64_t)(r.nodes.size() + 2 * r.src.size()) > (int64_t)(1 << 16)) return false;
    Bounds x = request_bounds(b, r);
    return x.t <= srv->tcap && x.dt <= srv->xcap;
}

bool fits_incremental(const rs_server *srv, const Base &b, const Request &r) {
    if (!fits_buffers(srv, b, r)) return false;
    Bounds x = request_bounds(b, r);
    // the bound on the touched rows' degree sums is loose (2-hop degree sums), so the delta
    // kernels still beat a full rescoring far above it: on the serving workload, raising the
    // cutoff from nnz/48 to nnz/24, /12, /6 and /4 took the incremental share from 44% to
    // 51, 58, 65 and 69% and the closed-loop rate from 1,335 to 1,410, 1,476, 1,522 and
    // 1,553 requests/s, with lower p99 at every offered rate; nnz/4 is also the slots'
    // buffer size for the largest graph
    return x.dt <= b.nnz / 4;
}

// stage the removal lists on the slot's stream; returns the device pointers
int stage_lists(Slot &sl, const Request &r, const int32_t **nodes, const int32_t **src, const int32_t **dst) {
    int64_t nn = (int64_t)r.nodes.size(), ne = (int64_t)r.src.size();
    std::memcpy(sl.h_req, r.nodes.data(), nn * sizeof(int32_t));
    std::memcpy(sl.h_req + nn, r.src.data(), ne * sizeof(int32_t));
    std::memcpy(sl.h_req + nn + ne, r.dst.data(), ne * sizeof(int32_t));
    if (nn + 2 * ne)
        RS_CUDA_TRY(cudaMemcpyAsync(sl.d_req, sl.h_req, (nn + 2 * ne) * sizeof(int32_t), cudaMemcpyHostToDevice, sl.s));
    *nodes = sl.d_req;
    *src = sl.d_req + nn;
    *dst = sl.d_req + nn + ne;
    return 0;
}

// incremental path: every kernel on the slot's stream, no host synchronisation
int launch_incremental(rs_server *srv, Slot &sl, const Request &r) {
    const Base &b = srv->bases[r.graph];
    BaseView B = b.view();
    SlotView &S = sl.v;
    cudaStream_t s = sl.s;
    const int32_t *dn, *ds, *dd;
    if (int rc = stage_lists(sl, r, &dn, &ds, &dd)) return rc;
    RS_CUDA_TRY(cudaMemsetAsync(S.dead, 0, ((b.nnz + 31) / 32) * sizeof(uint32_t), s));
    RS_CUDA_TRY(cudaMemsetAsync(S.flag, 0, b.n * sizeof(int32_t), s));
    RS_CUDA_TRY(cudaMemsetAsync(S.ctr, 0, C_NCTR * sizeof(unsigned long long), s));
    RS_CUDA_TRY(cudaMemsetAsync(S.err, 0, sizeof(int32_t), s));
    RS_CUDA_TRY(cudaMemcpyAsync(S.acc, b.acc, 2 * b.n * sizeof(unsigned long long), cudaMemcpyDeviceToDevice, s));
    Bounds x = request_bounds(b, r);
    int sms = sm_count();
    int64_t nn = (int64_t)r.nodes.size(), ne = (int64_t)r.src.size();
    auto warps_grid = [&](int64_t items, int per_sm) {
        return (int)std::max<int64_t>(1, std::min<int64_t>((items * 32 + kSvThreads - 1) / kSvThreads, (int64_t)sms * per_sm));
    };
    if (nn) sv_mark_nodes<<<warps_grid(nn, 8), kSvThreads, 0, s>>>(B, S, dn, nn);
    if (ne) sv_mark_edges<<<(int)std::min<int64_t>((ne + 255) / 256, sms * 8), 256, 0, s>>>(B, S, ds, dd, ne);
    int64_t tb = std::max<int64_t>(x.t, 1);
    int64_t wb = std::min<int64_t>(b.n, x.t + x.dt + 1);
    sv_trows<<<(int)std::min<int64_t>(tb, sms * 8), kSvThreads, 0, s>>>(B, S);
    sv_mark_w<<<(int)std::min<int64_t>(tb, sms * 8), kSvThreads, 0, s>>>(B, S);
    sv_type2_warp<<<warps_grid(wb, 4), kSvThreads, 0, s>>>(B, S);
    sv_type2_cta<<<(int)std::min<int64_t>(wb, sms * 4), kSvThreads, 0, s>>>(B, S);
    sv_tri_pairs<<<(int)std::min<int64_t>(tb, sms * 8), kSvThreads, 0, s>>>(B, S);
    sv_tri_find<<<sms * 8, kSvThreads, 0, s>>>(B, S);
    sv_tri_delta<<<sms * 8, kSvThreads, 0, s>>>(B, S);
    sv_wmax<<<grid_for(b.n, kSvThreads, 8), kSvThreads, 0, s>>>(B, S);
    sv_finalize<<<grid_for(b.n, kSvThreads, 8), kSvThreads, 0, s>>>(B, S);
    RS_CUDA_TRY(cudaGetLastError());
    return 0;
}

// device bytes of a full copy of a base graph (CSR twice, cross lists, G_x slots
// with both values, per-node records and workspaces)
int64_t full_bytes_estimate(const Base &b) { return 38 * b.nnz + 170 * b.n + (16 << 20); }

// full path: restore a copy of the base graph, apply the removals, rescore
int launch_full(rs_server *srv, Slot &sl, const Request &r) {
    Base &b = srv->bases[r.graph];
    cudaStream_t s = sl.s;
    Copy &cp = srv->copies[sl.copy];
    if (!cp.g) {
        if (int rc = rs_clone_graph(b.g, &cp.g, s)) return rc;
    }
    rs_graph *g = cp.g;
    RS_CUDA_TRY(cudaMemcpyAsync(g->off, b.g->off, (b.n + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    if (b.nnz) RS_CUDA_TRY(cudaMemcpyAsync(g->col, b.g->col, b.nnz * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    if (b.n) RS_CUDA_TRY(cudaMemsetAsync(g->removed, 0, 4 * b.n, s));
    int64_t applied = 0;
    if (int rc = rs_apply_removals(g, r.nodes.data(), (int64_t)r.nodes.size(), r.src.data(), r.dst.data(),
                                   (int64_t)r.src.size(), &applied, s))
        return rc;
    if (int rc = score_graph(g, sl.v.scores, s)) return rc;
    RS_CUDA_TRY(cudaMemsetAsync(sl.v.err, 0, sizeof(int32_t), s));
    return 0;
}

// a copy of graph gi for the full path: an idle one, or a new one within the budget
// (idle copies of other graphs are released, least recently used first); -1 if
// none can be had now, -2 if none ever can (nothing else holds memory)
int acquire_copy(rs_server *srv, int32_t gi) {
    for (size_t i = 0; i < srv->copies.size(); ++i) {
        Copy &c = srv->copies[i];
        if (c.graph == gi && !c.busy) { c.busy = true; c.last_use = ++srv->clock; return (int)i; }
    }
    int64_t need = full_bytes_estimate(srv->bases[gi]);
    while (srv->used + need > srv->budget) {
        int victim = -1;
        for (size_t i = 0; i < srv->copies.size(); ++i) {
            Copy &c = srv->copies[i];
            if (c.g && !c.busy && (victim < 0 || c.last_use < srv->copies[victim].last_use)) victim = (int)i;
        }
        if (victim < 0) break;
        Copy &v = srv->copies[victim];
        rs_free_graph(v.g);
        srv->used -= v.bytes;
        v = Copy();
    }
    if (srv->used + need > srv->budget) {
        bool any = false;
        for (auto &c : srv->copies) any |= c.busy;
        for (auto &sl : srv->slots) any |= sl.busy;
        return any ? -1 : -2;
    }
    int idx = -1;
    for (size_t i = 0; i < srv->copies.size(); ++i)
        if (!srv->copies[i].g && srv->copies[i].graph < 0) { idx = (int)i; break; }
    if (idx < 0) { srv->copies.push_back(Copy()); idx = (int)srv->copies.size() - 1; }
    Copy &c = srv->copies[idx];
    c.graph = gi;
    c.bytes = need;
    c.busy = true;
    c.last_use = ++srv->clock;
    srv->used += need;
    return idx;                    // the copy itself is made on the slot's stream
}

int start_request(rs_server *srv, Slot &sl, Request &&r, int refuse = 0) {
    const Base &b = srv->bases[r.graph];
    bool inc = sl.copy < 0;
    int rc = refuse ? refuse : inc ? launch_incremental(srv, sl, r) : launch_full(srv, sl, r);
    if (!rc && b.n > 0) rc = topk_scores(sl.tk, sl.v.scores, b.n, r.top_k, sl.ids, sl.vals, sl.s);
    if (!rc) {
        cudaError_t e = cudaMemcpyAsync(sl.h_ids, sl.ids, r.top_k * sizeof(int32_t), cudaMemcpyDeviceToHost, sl.s);
        if (!e) e = cudaMemcpyAsync(sl.h_vals, sl.vals, r.top_k * sizeof(double), cudaMemcpyDeviceToHost, sl.s);
        if (!e) e = cudaMemcpyAsync(sl.h_err, sl.v.err, sizeof(int32_t), cudaMemcpyDeviceToHost, sl.s);
        if (!e) e = cudaEventRecord(sl.done, sl.s);
        if (e) rc = cuda_fail(e, "rs_server: request");
    }
    sl.req = std::move(r);
    sl.path = inc ? 1 : 0;
    sl.status = rc;
    sl.busy = true;
    if (rc) cudaEventRecord(sl.done, sl.s);   // completes at once, with its error
    return 0;
}

}  // namespace

extern "C" rs_status rs_server_create(rs_graph *const *graphs, int32_t n_graphs, int32_t max_slots,
                                      int64_t budget_bytes, int32_t max_top_k, int32_t mode, rs_server **out) {
    if (!graphs || n_graphs < 1 || !out || max_slots < 1 || budget_bytes < 0)
        return (rs_status)fail(RS_EINVAL, "rs_server_create: bad arguments");
    if (mode != RS_SERVE_INCREMENTAL && mode != RS_SERVE_FULL)
        return (rs_status)fail(RS_EINVAL, "rs_server_create: unknown mode");
    if (max_top_k < 1 || max_top_k > 16384) return (rs_status)fail(RS_EINVAL, "rs_server_create: max_top_k in [1, 16384]");
    for (int32_t i = 0; i < n_graphs; ++i)
        if (!graphs[i]) return (rs_status)fail(RS_EINVAL, "rs_server_create: NULL graph");
    rs_server *srv = new rs_server();
    srv->mode = mode;
    srv->budget = budget_bytes;
    srv->max_top_k = max_top_k;
    srv->bases.resize(n_graphs);
    auto bail = [&](int rc) {
        for (auto &sl : srv->slots) free_slot(sl);
        for (auto &b : srv->bases) { cudaFree(b.acc); cudaFree(b.scores); cudaFree(b.rowmax); }
        delete srv;
        return (rs_status)rc;
    };
    for (int32_t i = 0; i < n_graphs; ++i) {
        srv->bases[i].g = graphs[i];
        if (int rc = prepare_base(srv->bases[i])) return bail(rc);
        srv->n_max = std::max(srv->n_max, srv->bases[i].n);
        srv->nnz_max = std::max(srv->nnz_max, srv->bases[i].nnz);
        int64_t m = std::min<int64_t>(srv->bases[i].dmax, srv->bases[i].k), c = 1;
        while (c < 2 * m) c <<= 1;
        srv->hub_cap = std::max(srv->hub_cap, c);
    }
    srv->tcap = std::max<int64_t>(1, std::min<int64_t>(srv->n_max, std::max<int64_t>(1 << 16, srv->n_max / 4)));
    srv->xcap = std::max<int64_t>(1, std::min<int64_t>(srv->nnz_max, std::max<int64_t>(1 << 20, srv->nnz_max / 4)));
    for (int32_t i = 0; i < max_slots; ++i) {
        Slot sl;
        int rc = alloc_slot(srv, sl);
        if (rc || srv->used + sl.bytes > srv->budget) {
            free_slot(sl);
            if (i == 0) return bail(rc ? rc : fail(RS_EBUDGET, "rs_server_create: one request slot does not fit the budget"));
            break;
        }
        srv->used += sl.bytes;
        srv->slots.push_back(std::move(sl));
    }
    *out = srv;
    return RS_OK;
}

extern "C" rs_status rs_server_submit(rs_server *srv, int32_t graph, const int32_t *nodes, int64_t n_nodes,
                                      const int32_t *edge_src, const int32_t *edge_dst, int64_t n_edges,
                                      int32_t top_k, int64_t *ticket_out) {
    if (!srv || !ticket_out) return (rs_status)fail(RS_EINVAL, "rs_server_submit: NULL argument");
    if (graph < 0 || graph >= (int32_t)srv->bases.size()) return (rs_status)fail(RS_EINVAL, "rs_server_submit: bad graph");
    const Base &b = srv->bases[graph];
    if (top_k < 1 || top_k > srv->max_top_k || (int64_t)top_k > b.n)
        return (rs_status)fail(RS_EINVAL, "rs_server_submit: top_k must be in [1, min(n, max_top_k)]");
    if (n_nodes < 0 || n_edges < 0 || (n_nodes && !nodes) || (n_edges && (!edge_src || !edge_dst)))
        return (rs_status)fail(RS_EINVAL, "rs_server_submit: bad arrays");
    Request r;
    r.graph = graph;
    r.top_k = top_k;
    r.nodes.assign(nodes, nodes + n_nodes);
    r.src.assign(edge_src, edge_src + n_edges);
    r.dst.assign(edge_dst, edge_dst + n_edges);
    for (int32_t v : r.nodes)
        if (v < 0 || v >= b.n) return (rs_status)fail(RS_EINVAL, "rs_server_submit: node id out of range");
    for (int64_t i = 0; i < n_edges; ++i)
        if (r.src[i] < 0 || r.src[i] >= b.n || r.dst[i] < 0 || r.dst[i] >= b.n)
            return (rs_status)fail(RS_EINVAL, "rs_server_submit: edge endpoint out of range");
    r.ticket = srv->next_ticket++;
    *ticket_out = r.ticket;
    srv->queue.push_back(std::move(r));
    return RS_OK;
}

extern "C" rs_status rs_server_poll(rs_server *srv, int32_t max, int32_t kmax, int64_t *tickets, int32_t *status,
                                    int32_t *path, int32_t *ids, double *scores, int32_t *n_done, int32_t block) {
    if (!srv || !n_done || max < 0 || (max > 0 && (!tickets || !status)) || kmax < 0)
        return (rs_status)fail(RS_EINVAL, "rs_server_poll: bad arguments");
    int32_t done = 0;
    while (true) {
        // collect finished requests
        for (auto &sl : srv->slots) {
            if (!sl.busy || done >= max) continue;
            cudaError_t q = cudaEventQuery(sl.done);
            if (q == cudaErrorNotReady) continue;
            int32_t st = sl.status;
            if (q != cudaSuccess && !st) st = cuda_fail(q, "rs_server: request");
            if (!st && *sl.h_err) st = RS_EBUDGET;
            tickets[done] = sl.req.ticket;
            status[done] = st;
            if (path) path[done] = sl.path;
            int32_t k = std::min(kmax, sl.req.top_k);
            if (ids) for (int32_t j = 0; j < k; ++j) ids[(int64_t)done * kmax + j] = st ? -1 : sl.h_ids[j];
            if (scores) for (int32_t j = 0; j < k; ++j) scores[(int64_t)done * kmax + j] = st ? 0.0 : sl.h_vals[j];
            sl.busy = false;
            if (sl.copy >= 0) { srv->copies[sl.copy].busy = false; sl.copy = -1; }
            ++done;
        }
        // admit queued requests, in order, into free slots within the memory budget
        for (auto &sl : srv->slots) {
            if (srv->queue.empty()) break;
            if (sl.busy) continue;
            const Request &front = srv->queue.front();
            const Base &b = srv->bases[front.graph];
            bool need_full = srv->mode == RS_SERVE_FULL || !fits_incremental(srv, b, front);
            int refuse = 0;
            sl.copy = -1;
            if (need_full) {
                int c = acquire_copy(srv, front.graph);
                if (c == -1) break;                          // wait for memory to free up
                if (c == -2) refuse = fail(RS_EBUDGET, "rs_server: the request does not fit the memory budget");
                else sl.copy = c;
            }
            Request r = std::move(srv->queue.front());
            srv->queue.pop_front();
            start_request(srv, sl, std::move(r), refuse);
        }
        bool in_flight = false;
        for (auto &sl : srv->slots) in_flight |= sl.busy;
        if (!block || done > 0 || (!in_flight && srv->queue.empty()) || done >= max) break;
    }
    *n_done = done;
    return RS_OK;
}

extern "C" rs_status rs_server_info(const rs_server *srv, int32_t *slots, int64_t *bytes_used, int64_t *queued,
                                    int32_t *in_flight) {
    if (!srv) return (rs_status)fail(RS_EINVAL, "rs_server_info: NULL server");
    if (slots) *slots = (int32_t)srv->slots.size();
    if (bytes_used) *bytes_used = srv->used;
    if (queued) *queued = (int64_t)srv->queue.size();
    if (in_flight) {
        int32_t c = 0;
        for (auto &sl : srv->slots) c += sl.busy;
        *in_flight = c;
    }
    return RS_OK;
}

extern "C" rs_status rs_server_whatif(rs_server *srv, int32_t graph, const int32_t *nodes, int64_t n_nodes,
                                      const int32_t *edge_src, const int32_t *edge_dst, int64_t n_edges,
                                      int32_t full, double *scores_out, int32_t *path_out, void *stream) {
    if (!srv || !scores_out) return (rs_status)fail(RS_EINVAL, "rs_server_whatif: NULL argument");
    if (graph < 0 || graph >= (int32_t)srv->bases.size()) return (rs_status)fail(RS_EINVAL, "rs_server_whatif: bad graph");
    for (auto &sl : srv->slots)
        if (sl.busy) return (rs_status)fail(RS_EINVAL, "rs_server_whatif: requests are in flight");
    const Base &b = srv->bases[graph];
    if (n_nodes < 0 || n_edges < 0 || (n_nodes && !nodes) || (n_edges && (!edge_src || !edge_dst)))
        return (rs_status)fail(RS_EINVAL, "rs_server_whatif: bad arrays");
    Request r;
    r.graph = graph;
    r.top_k = 1;
    r.nodes.assign(nodes, nodes + n_nodes);
    r.src.assign(edge_src, edge_src + n_edges);
    r.dst.assign(edge_dst, edge_dst + n_edges);
    for (int32_t v : r.nodes)
        if (v < 0 || v >= b.n) return (rs_status)fail(RS_EINVAL, "rs_server_whatif: node id out of range");
    for (int64_t i = 0; i < n_edges; ++i)
        if (r.src[i] < 0 || r.src[i] >= b.n || r.dst[i] < 0 || r.dst[i] >= b.n)
            return (rs_status)fail(RS_EINVAL, "rs_server_whatif: edge endpoint out of range");
    Slot &sl = srv->slots[0];
    bool inc = full == 2 ? fits_buffers(srv, b, r) : (!full && fits_incremental(srv, b, r));
    sl.copy = -1;
    if (!inc) {
        int c = acquire_copy(srv, graph);
        if (c < 0) return (rs_status)fail(RS_EBUDGET, "rs_server_whatif: a full copy does not fit the memory budget");
        sl.copy = c;
    }
    int rc = inc ? launch_incremental(srv, sl, r) : launch_full(srv, sl, r);
    if (sl.copy >= 0) { srv->copies[sl.copy].busy = false; sl.copy = -1; }
    if (rc) return (rs_status)rc;
    int32_t err = 0;
    cudaError_t e = cudaMemcpyAsync(&err, sl.v.err, sizeof(int32_t), cudaMemcpyDeviceToHost, sl.s);
    if (!e) e = cudaStreamSynchronize(sl.s);
    if (!e && b.n) e = cudaMemcpyAsync(scores_out, sl.v.scores, b.n * sizeof(double), cudaMemcpyDeviceToDevice,
                                       (cudaStream_t)stream);
    if (!e) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e) return (rs_status)cuda_fail(e, "rs_server_whatif");
    if (err) return (rs_status)fail(RS_EBUDGET, "rs_server_whatif: a slot buffer overflowed");
    if (path_out) *path_out = inc ? 1 : 0;
    return RS_OK;
}

extern "C" rs_status rs_server_base_scores(rs_server *srv, int32_t graph, double *scores_out, void *stream) {
    if (!srv || !scores_out || graph < 0 || graph >= (int32_t)srv->bases.size())
        return (rs_status)fail(RS_EINVAL, "rs_server_base_scores: bad arguments");
    const Base &b = srv->bases[graph];
    if (b.n)
        if (cudaError_t e = cudaMemcpyAsync(scores_out, b.scores, b.n * sizeof(double), cudaMemcpyDeviceToDevice,
                                            (cudaStream_t)stream))
            return (rs_status)cuda_fail(e, "rs_server_base_scores");
    return RS_OK;
}

extern "C" void rs_server_free(rs_server *srv) {
    if (!srv) return;
    for (auto &sl : srv->slots) {
        if (sl.busy) cudaEventSynchronize(sl.done);
        free_slot(sl);
    }
    for (auto &c : srv->copies)
        if (c.g) rs_free_graph(c.g);
    for (auto &b : srv->bases) {
        cudaFree(b.acc); cudaFree(b.scores); cudaFree(b.rowmax);
        rs_free_graph(b.g);
    }
    delete srv;
}
