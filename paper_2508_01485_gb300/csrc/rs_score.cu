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
//   P3  per node a: oriented triangle listing on G_x (pairs of out-neighbours,
//       closing edge by binary search), the Type-I terms of the three apexes;
//   FIN R(u) = acc(u) / (w_max d(u)(d(u)-1)), 0 when d(u) < 2 or w_max = 0.
// All terms are added into 128-bit fixed-point accumulators, so the scores do
// not depend on the order in which threads run.
#include "rs.h"
#include "rs_internal.cuh"
#include "rs_device.cuh"

using namespace rs;

#define FULL 0xFFFFFFFFu

namespace {

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

// sum of the staged values over the lanes of `grp` (exact, fixed order)
__device__ __forceinline__ u128 group_sum_all(const uint64_t *stage, unsigned grp) {
    u128 q = 0;
    while (grp) {
        int j = __ffs(grp) - 1;
        q += stage[j];
        grp &= grp - 1;
    }
    return q;
}

// Every weight of a row with L distinct neighbour communities is at most
// L log2 L (an entropy over at most L categories is at most log2 L); a row
// whose bound cannot exceed the w_max found so far needs no column maximum.
__device__ __forceinline__ bool row_may_raise_max(uint32_t L, float wcur) {
    if (L < 2) return false;
    float fl = (float)L;
    return fl * __log2f(fl) * 1.001f + 1e-6f > wcur;
}
// w_max found so far, rounded down to a float (read once per warp)
__device__ __forceinline__ float current_wmax(const unsigned long long *wmax_bits) {
    unsigned long long b = *(volatile const unsigned long long *)wmax_bits;
    return __double2float_rd(__longlong_as_double((long long)b));
}

// publish a row's largest weight when it may raise its graph's w_max (wcur is
// the w_max read earlier, rounded down: any m above w_max has m.hi >= wcur)
__device__ __forceinline__ void publish_max(const Batch &B, int32_t gi, df m, float wcur) {
    if (m.hi > 0.0f && m.hi >= wcur) atomicMax(&B.wmax[gi], double_bits(m));
}

// ======================================================================================
// P1
// ======================================================================================

// Row kernels take their next row from a per-launch counter (zeroed at the start of
// every scoring pass), so warps or CTAs that drew short rows take more and no long
// tail is left on a few of them.
__device__ __forceinline__ int64_t warp_next(unsigned long long *ctr) {
    unsigned long long t = 0;
    if ((threadIdx.x & 31) == 0) t = atomicAdd(ctr, 1ull);
    return (int64_t)__shfl_sync(FULL, t, 0);
}
__device__ __forceinline__ int64_t cta_next(unsigned long long *ctr, long long *sh) {
    __syncthreads();
    if (threadIdx.x == 0) *sh = (long long)atomicAdd(ctr, 1ull);
    __syncthreads();
    return *sh;
}

constexpr int kSlots = kSmallMax;

__device__ __forceinline__ void store_rowsum(RowSum *rsum, int32_t v, const RowAgg &a) {
    RowSum r;
    r.xlo = (uint64_t)a.X;
    r.xhi = (uint64_t)(a.X >> 64);
    r.L = a.L;
    r.pad = 0;
    rsum[v] = r;
}

// Small rows, tiles of 32 consecutive rows (id order) per warp: the union of
// their CSR segments is streamed with one neighbour per lane (coalesced
// columns, one label gather per lane), (row, community) groups come from warp
// matching, and lane l then finishes row l of the tile.  A row of degree
// <= 32 spans at most two chunks, so its foreign list holds at most 32
// entries (a community seen in two chunks appears twice and is merged).
struct SmallTile {
    int32_t flab[kSlots][32];       // foreign (community, count) entries, entry-major
    uint8_t fcnt[kSlots][32];
    int32_t pre[33];                // prefix sums of the tile's degrees
    int64_t rb[32];                 // row starts
    int32_t cv[32];                 // row labels
    uint32_t own[32], nf[32];
    int32_t nx[32];                 // cross list fill
};

// one chunk of up to 32 tile entries, entry e0 + lane in this lane (act): its row r, its
// neighbour x and x's label c; the own-community counts, the cross lists and the
// (row, community) groups are updated
__device__ __forceinline__ void p1_small_chunk(SmallTile &T, bool act, int32_t r, int32_t x, int32_t c,
                                               int32_t *__restrict__ cl_col, int32_t *__restrict__ cl_lab, int lane) {
    bool own = act && c == T.cv[r];
    bool foreign = act && !own;
    unsigned om = __ballot_sync(FULL, own), fm = __ballot_sync(FULL, foreign);
    unsigned gown = 0, grow = 0;
    if (own) gown = __match_any_sync(om, r);
    if (foreign) grow = __match_any_sync(fm, r);
    int32_t xbase = foreign ? T.nx[r] : 0;
    __syncwarp();
    if (own && lane == __ffs(gown) - 1) T.own[r] += __popc(gown);
    if (foreign) {
        int64_t p = T.rb[r] + xbase + __popc(grow & lanemask_lt());
        cl_col[p] = x;
        cl_lab[p] = c;
        if (lane == __ffs(grow) - 1) T.nx[r] = xbase + __popc(grow);
        unsigned long long key = ((unsigned long long)(uint32_t)r << 32) | (uint32_t)c;
        unsigned gc = __match_any_sync(fm, key);
        if (lane == __ffs(gc) - 1) {
            uint32_t slot = atomicAdd(&T.nf[r], 1u);
            T.flab[slot][r] = c;
            T.fcnt[slot][r] = (uint8_t)__popc(gc);
        }
    }
    __syncwarp();
}

// lane `lane` finishes row v (degree d, label cv) of the tile: aggregates, weights, s_v
__device__ __forceinline__ void p1_small_finish(SmallTile &T, int32_t v, int32_t d, int32_t cv, const Batch &B,
                                                const uint64_t *__restrict__ LG, NodeRec *__restrict__ rec,
                                                int32_t *__restrict__ Lall, RowSum *__restrict__ rsum, int lane) {
    int32_t gi = graph_of(B, v);
    float wcur = current_wmax(&B.wmax[gi]);
    uint32_t own = T.own[lane];
    int nf = (int)T.nf[lane];
    // merge a community listed from two chunks
    for (int j = 1; j < nf; ++j)
        for (int j2 = 0; j2 < j; ++j2)
            if (T.fcnt[j2][lane] && T.flab[j2][lane] == T.flab[j][lane]) {
                T.fcnt[j2][lane] += T.fcnt[j][lane];
                T.fcnt[j][lane] = 0;
                break;
            }
    u128 X = (u128)own * LG[own];
    uint64_t seen = own ? (1ull << own) : 0ull;
    uint32_t L = own > 0 ? 1u : 0u;
    for (int j = 0; j < nf; ++j) {
        uint32_t f = T.fcnt[j][lane];
        if (!f) continue;
        X += (u128)f * LG[f];
        seen |= 1ull << f;
        ++L;
    }
    RowAgg a{(uint32_t)d, L, X};
    store_rowsum(rsum, v, a);
    bool want_max = row_may_raise_max(a.L, wcur);
    df cm{0.0f, 0.0f}, wown{0.0f, 0.0f};
    if (want_max) {
        while (seen) {
            uint32_t f = (uint32_t)(__ffsll((long long)seen) - 1);
            df w = column_weight(a, f, LG);
            if (f == own) wown = w;
            cm = df_max(cm, w);
            seen &= seen - 1;
        }
    } else if (own > 0) {
        wown = column_weight(a, own, LG);
    }
    NodeRec rr;
    df m = p1_row_result(a, own, cm, k_of(B, gi), LG, rr, cv, wown, want_max);
    publish_max(B, gi, m, wcur);
    rec[v] = rr;
    Lall[v] = (int32_t)a.L;
}

// the tile's rows: lane l takes row rows[t0 + l]; prefix sums of the degrees, row starts
// and labels into T; returns the tile's entry count D
__device__ __forceinline__ int32_t p1_small_setup(SmallTile &T, const int64_t *__restrict__ off,
                                                  const int32_t *__restrict__ lab, const int32_t *__restrict__ rows,
                                                  int64_t nrows, int64_t t0, int lane, bool &have, int32_t &v,
                                                  int32_t &d, int32_t &cv) {
    int64_t i = t0 + lane;
    have = i < nrows;
    v = have ? rows[i] : 0;
    int64_t b = have ? off[v] : 0;
    d = have ? (int32_t)(off[v + 1] - b) : 0;
    cv = have ? lab[v] : -1;
    int32_t incl = d;
    for (int o = 1; o < 32; o <<= 1) {
        int32_t y = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += y;
    }
    T.pre[lane + 1] = incl;
    if (lane == 0) T.pre[0] = 0;
    T.rb[lane] = b;
    T.cv[lane] = cv;
    T.own[lane] = 0;
    T.nf[lane] = 0;
    T.nx[lane] = 0;
    __syncwarp();
    return __shfl_sync(FULL, incl, 31);
}

__global__ void __launch_bounds__(kThreads) p1_small_kernel(
    const int64_t *__restrict__ off, const int32_t *__restrict__ col, const int32_t *__restrict__ lab,
    const int32_t *__restrict__ rows, int64_t nrows, Batch B, const uint64_t *__restrict__ LG,
    NodeRec *__restrict__ rec, int32_t *__restrict__ Lall,
    RowSum *__restrict__ rsum, int32_t *__restrict__ cl_col, int32_t *__restrict__ cl_lab) {
    __shared__ SmallTile tiles[kThreads / 32];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    SmallTile &T = tiles[wid];
    int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t t0 = warp * 32; t0 < nrows; t0 += nwarps * 32) {
        bool have;
        int32_t v, d, cv;
        const int32_t D = p1_small_setup(T, off, lab, rows, nrows, t0, lane, have, v, d, cv);
        // entry e of the tile: its row (last r with pre[r] <= e) and its CSR column
        auto locate = [&](int32_t e, int32_t &r, int32_t &x) {
            int32_t lo = 0, hi = 32;
            while (hi - lo > 1) {
                int32_t mid = (lo + hi) >> 1;
                if (T.pre[mid] <= e) lo = mid; else hi = mid;
            }
            r = lo;
            x = col[T.rb[r] + (e - T.pre[r])];
        };
        // software pipeline: the label of the next chunk and the column of the one
        // after it are loaded while the current chunk is matched
        int32_t rA = 0, xA = -1, cA = -1, rB = 0, xB = -1;
        if (lane < D) { locate(lane, rA, xA); cA = lab[xA]; }
        if (32 + lane < D) locate(32 + lane, rB, xB);
        for (int32_t e0 = 0; e0 < D; e0 += 32) {
            const int32_t r = rA, x = xA, c = cA;
            const bool act = e0 + lane < D;
            int32_t cB = -1, rC = 0, xC = -1;
            if (e0 + 32 + lane < D) cB = lab[xB];
            if (e0 + 64 + lane < D) locate(e0 + 64 + lane, rC, xC);
            rA = rB; xA = xB; cA = cB; rB = rC; xB = xC;
            p1_small_chunk(T, act, r, x, c, cl_col, cl_lab, lane);
        }
        // lane `lane` finishes row `lane` of the tile
        if (have) p1_small_finish(T, v, d, cv, B, LG, rec, Lall, rsum, lane);
        __syncwarp();
    }
}

// The same tiles with the loads staged in shared memory by asynchronous copies
// (p1_stage = 1): lane l copies its row's columns (cp.async, 4 bytes each) to the tile's
// entry range [pre[l], pre[l+1]) and writes the entries' row number; after the wait the
// lanes copy the labels of those neighbours in the same way (a gather by cp.async);
// the chunks then read row, column and label from shared memory.  A warp keeps its
// tile's entries (at most 32 x 32) and their labels in flight at once instead of two
// chunks ahead.  Dynamic shared memory: kStageWarps x (SmallTile + SmallStage).
constexpr int kStageWarps = 4;
struct SmallStage {
    int32_t col[kSmallMax * 32];
    int32_t lab[kSmallMax * 32];
    uint8_t row[kSmallMax * 32];
};

__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

__global__ void __launch_bounds__(kStageWarps * 32) p1_small_staged_kernel(
    const int64_t *__restrict__ off, const int32_t *__restrict__ col, const int32_t *__restrict__ lab,
    const int32_t *__restrict__ rows, int64_t nrows, Batch B, const uint64_t *__restrict__ LG,
    NodeRec *__restrict__ rec, int32_t *__restrict__ Lall,
    RowSum *__restrict__ rsum, int32_t *__restrict__ cl_col, int32_t *__restrict__ cl_lab) {
    extern __shared__ __align__(16) unsigned char st_smem[];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    SmallTile &T = reinterpret_cast<SmallTile *>(st_smem)[wid];
    SmallStage &S = reinterpret_cast<SmallStage *>(st_smem + kStageWarps * sizeof(SmallTile))[wid];
    int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t t0 = warp * 32; t0 < nrows; t0 += nwarps * 32) {
        bool have;
        int32_t v, d, cv;
        const int32_t D = p1_small_setup(T, off, lab, rows, nrows, t0, lane, have, v, d, cv);
        {
            const int32_t p0 = T.pre[lane];
            const int32_t *src = col + T.rb[lane];
            for (int32_t j = 0; j < d; ++j) {
                cp_async4(&S.col[p0 + j], src + j);
                S.row[p0 + j] = (uint8_t)lane;
            }
            cp_async_wait_all();
            __syncwarp();
            for (int32_t e = lane; e < D; e += 32) cp_async4(&S.lab[e], lab + S.col[e]);
            cp_async_wait_all();
            __syncwarp();
        }
        for (int32_t e0 = 0; e0 < D; e0 += 32) {
            const int32_t e = e0 + lane;
            const bool act = e < D;
            const int32_t r = act ? S.row[e] : 0, x = act ? S.col[e] : -1, c = act ? S.lab[e] : -1;
            p1_small_chunk(T, act, r, x, c, cl_col, cl_lab, lane);
        }
        if (have) p1_small_finish(T, v, d, cv, B, LG, rec, Lall, rsum, lane);
        __syncwarp();
    }
}

// Mid rows, one warp per row, a per-warp shared-memory table of kWarpCap slots.
constexpr int kMidWarps = kThreads / 32;

__global__ void __launch_bounds__(kThreads) p1_mid_kernel(
    const int64_t *__restrict__ off, const int32_t *__restrict__ col, const int32_t *__restrict__ lab,
    const int32_t *__restrict__ rows, int64_t nrows, Batch B, const uint64_t *__restrict__ LG,
    NodeRec *__restrict__ rec, int32_t *__restrict__ Lall, int *err,
    RowSum *__restrict__ rsum, int32_t *__restrict__ cl_col, int32_t *__restrict__ cl_lab,
    unsigned long long *wq) {
    __shared__ int32_t skey[kMidWarps][kWarpCap];
    __shared__ uint32_t scnt[kMidWarps][kWarpCap];
    __shared__ int16_t sused[kMidWarps][kWarpCap];    // slots taken by the current row
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (uint32_t j = lane; j < kWarpCap; j += 32) { skey[wid][j] = kEmpty; scnt[wid][j] = 0; }
    __syncwarp();
    for (int64_t i = warp_next(wq); i < nrows; i = warp_next(wq)) {
        int32_t v = rows[i];
        int64_t b = off[v];
        int d = (int)(off[v + 1] - b);
        int32_t cv = lab[v];
        int32_t gi = graph_of(B, v);
        uint32_t cap = dev_pow2_at_least(2u * (uint32_t)min(d, k_of(B, gi)));
        Tab t{skey[wid], scnt[wid], nullptr, nullptr, cap - 1};
        uint32_t own = 0, nused = 0;
        int32_t nx = 0;
        u128 X = 0;                       // foreign part, from count deltas at insert time
        // software pipeline: the next chunk's labels and the columns of the one after
        // it are loaded while the current chunk is inserted
        int32_t xA = lane < d ? col[b + lane] : -1;
        int32_t cA = lane < d ? lab[xA] : -1;
        int32_t xB = 32 + lane < d ? col[b + 32 + lane] : -1;
        for (int base = 0; base < d; base += 32) {
            int e = base + lane;
            bool act = e < d;
            const int32_t x = xA, c = cA;
            const int32_t cB = e + 32 < d ? lab[xB] : -1;
            const int32_t xC = e + 64 < d ? col[b + e + 64] : -1;
            xA = xB; cA = cB; xB = xC;
            own += (act && c == cv);
            bool foreign = act && c != cv;
            unsigned fm = __ballot_sync(FULL, foreign);
            bool lead = false, fresh = false;
            int sl = -1;
            if (foreign) {
                int64_t p = b + nx + __popc(fm & lanemask_lt());
                cl_col[p] = x;
                cl_lab[p] = c;
                unsigned grp = __match_any_sync(fm, c);
                lead = lane == __ffs(grp) - 1;
                if (lead) {
                    uint32_t old, g = __popc(grp);
                    sl = tab_insert_old(t, c, g, old, fresh, err);
                    X += (u128)(old + g) * LG[old + g] - (u128)old * LG[old];
                }
            }
            unsigned nm = __ballot_sync(FULL, fresh);
            if (fresh) sused[wid][nused + __popc(nm & lanemask_lt())] = (int16_t)sl;
            nused += __popc(nm);
            nx += __popc(fm);
        }
        __syncwarp();
        for (int o = 16; o; o >>= 1) own += __shfl_xor_sync(FULL, own, o);
        RowAgg a{(uint32_t)d, nused + (own > 0 ? 1u : 0u), warp_sum_u128(X) + (u128)own * LG[own]};
        float wcur = 0.0f;
        if (lane == 0) wcur = current_wmax(&B.wmax[gi]);
        wcur = __shfl_sync(FULL, wcur, 0);
        bool want_max = row_may_raise_max(a.L, wcur);
        df cm{0.0f, 0.0f}, wown{0.0f, 0.0f};
        if (want_max)
            for (uint32_t j = lane; j < nused; j += 32) cm = df_max(cm, column_weight(a, t.cnt[sused[wid][j]], LG));
        if (own > 0 && lane == 0) { wown = column_weight(a, own, LG); cm = df_max(cm, wown); }
        cm = warp_max_df(cm);
        if (lane == 0) {
            NodeRec r;
            df m = p1_row_result(a, own, cm, k_of(B, gi), LG, r, cv, wown, want_max);
            publish_max(B, gi, m, wcur);
            rec[v] = r;
            Lall[v] = (int32_t)a.L;
            store_rowsum(rsum, v, a);
        }
        __syncwarp();
        for (uint32_t j = lane; j < nused; j += 32) { int sl = sused[wid][j]; t.key[sl] = kEmpty; t.cnt[sl] = 0; }
        __syncwarp();
    }
}

// Large rows, one CTA per row, a per-CTA table of up to kMidCap slots
// CTA-ordered position of the flagged threads of one round; every thread calls
template <int NT>
__device__ __forceinline__ int32_t cta_rank(bool flag, int32_t &base, int32_t *sh_cnt) {
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned m = __ballot_sync(FULL, flag);
    if (lane == 0) sh_cnt[wid] = __popc(m);
    __syncthreads();
    int32_t p = base, tot = 0;
    for (int j = 0; j < NT / 32; ++j) {
        if (j < wid) p += sh_cnt[j];
        tot += sh_cnt[j];
    }
    p += __popc(m & lanemask_lt());
    base += tot;
    __syncthreads();
    return p;
}

template <int NT>
__global__ void __launch_bounds__(NT) p1_large_kernel(
    const int64_t *__restrict__ off, const int32_t *__restrict__ col, const int32_t *__restrict__ lab,
    const int32_t *__restrict__ rows, int64_t nrows, Batch B, const uint64_t *__restrict__ LG,
    NodeRec *__restrict__ rec, int32_t *__restrict__ Lall, int *err,
    RowSum *__restrict__ rsum, int32_t *__restrict__ cl_col, int32_t *__restrict__ cl_lab,
    unsigned long long *wq) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint32_t sh_u32[NT / 32];
    __shared__ u128 sh_u128[NT / 32];
    __shared__ df sh_df[NT / 32];
    __shared__ int32_t sh_cnt[NT / 32];
    int tid = threadIdx.x, lane = tid & 31;
    __shared__ long long sh_next;
    for (int64_t i = cta_next(wq, &sh_next); i < nrows; i = cta_next(wq, &sh_next)) {
        int32_t v = rows[i];
        int64_t b = off[v];
        int d = (int)(off[v + 1] - b);
        int32_t cv = lab[v];
        int32_t gi = graph_of(B, v);
        uint32_t cap = dev_pow2_at_least(2u * (uint32_t)min(d, k_of(B, gi)));
        Tab t{(int32_t *)smem, (uint32_t *)(smem + 4 * cap), nullptr, nullptr, cap - 1};
        for (uint32_t j = tid; j < cap; j += NT) { t.key[j] = kEmpty; t.cnt[j] = 0; }
        __syncthreads();
        uint32_t own = 0;
        int32_t nx = 0;
        int32_t xA = tid < d ? col[b + tid] : -1;
        int32_t cA = tid < d ? lab[xA] : -1;
        int32_t xB = NT + tid < d ? col[b + NT + tid] : -1;
        for (int base = 0; base < d; base += NT) {
            int e = base + tid;
            bool act = e < d;
            const int32_t x = xA, c = cA;
            const int32_t cB = e + NT < d ? lab[xB] : -1;
            const int32_t xC = e + 2 * NT < d ? col[b + e + 2 * NT] : -1;
            xA = xB; cA = cB; xB = xC;
            own += (act && c == cv);
            bool foreign = act && c != cv;
            unsigned fm = __ballot_sync(FULL, foreign);
            if (foreign) {
                unsigned grp = __match_any_sync(fm, c);
                if (lane == __ffs(grp) - 1) tab_insert(t, c, __popc(grp), err);
            }
            int32_t p = cta_rank<NT>(foreign, nx, sh_cnt);
            if (foreign) { cl_col[b + p] = x; cl_lab[b + p] = c; }
        }
        own = block_sum_u32<NT>(own, sh_u32);      // syncs: the table is complete
        uint32_t Lf = 0;
        u128 X = 0;
        for (uint32_t j = tid; j < cap; j += NT)
            if (t.key[j] != kEmpty) { Lf++; X += (u128)t.cnt[j] * LG[t.cnt[j]]; }
        Lf = block_sum_u32<NT>(Lf, sh_u32);
        X = block_sum_u128<NT>(X, sh_u128);
        RowAgg a{(uint32_t)d, Lf + (own > 0 ? 1u : 0u), X + (u128)own * LG[own]};
        float wcur = current_wmax(&B.wmax[gi]);
        bool want_max = __syncthreads_or(row_may_raise_max(a.L, wcur));
        df cm{0.0f, 0.0f}, wown{0.0f, 0.0f};
        if (want_max)
            for (uint32_t j = tid; j < cap; j += NT)
                if (t.key[j] != kEmpty) cm = df_max(cm, column_weight(a, t.cnt[j], LG));
        if (own > 0) { wown = column_weight(a, own, LG); cm = df_max(cm, wown); }
        cm = block_max_df<NT>(cm, sh_df);
        if (tid == 0) {
            NodeRec r;
            df m = p1_row_result(a, own, cm, k_of(B, gi), LG, r, cv, wown, want_max);
            publish_max(B, gi, m, wcur);
            rec[v] = r;
            Lall[v] = (int32_t)a.L;
            store_rowsum(rsum, v, a);
        }
        __syncthreads();                              // table reuse
    }
}

// hub rows: chunks insert foreign communities into the row's global table
template <int NT>
__global__ void __launch_bounds__(NT) hub_p1_insert_kernel(
    const int64_t *__restrict__ off, const int32_t *__restrict__ col, const int32_t *__restrict__ lab,
    const HubInfo *__restrict__ hubs, const int32_t *__restrict__ items, const int32_t *__restrict__ chunks,
    int64_t nitems, int32_t chunk_len, int32_t *hkey, uint32_t *hcnt, HubAgg *hagg, int *err) {
    __shared__ uint32_t sh_u32[NT / 32];
    int tid = threadIdx.x, lane = tid & 31;
    for (int64_t it = blockIdx.x; it < nitems; it += gridDim.x) {
        HubInfo h = hubs[items[it]];
        int64_t b = off[h.row];
        int64_t d = off[h.row + 1] - b;
        int64_t lo = (int64_t)chunks[it] * chunk_len;
        int64_t hi = min(d, lo + chunk_len);
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

// hub rows, P1 step 2: each slot range of a hub's table adds its foreign groups and
// their sum f LG[f] to the hub's aggregates (exact integer sums, so any order gives the
// same bits)
template <int NT>
__global__ void __launch_bounds__(NT) hub_p1_sums_kernel(
    const HubInfo *__restrict__ hubs, const int32_t *__restrict__ sitem, const int32_t *__restrict__ srange,
    int64_t nsitems, const uint64_t *__restrict__ LG, const int32_t *hkey, const uint32_t *hcnt, HubAgg *hagg) {
    __shared__ uint32_t sh_u32[NT / 32];
    __shared__ u128 sh_u128[NT / 32];
    for (int64_t it = blockIdx.x; it < nsitems; it += gridDim.x) {
        const int32_t hi = sitem[it];
        const HubInfo h = hubs[hi];
        const int64_t j0 = (int64_t)srange[it] * kHubSlotRange, j1 = min((int64_t)h.cap, j0 + (int64_t)kHubSlotRange);
        uint32_t Lf = 0;
        u128 X = 0;
        for (int64_t j = j0 + threadIdx.x; j < j1; j += NT) {
            const int64_t s = h.tab + j;
            if (hkey[s] != kEmpty) {
                const uint32_t c = hcnt[s];
                Lf++;
                X += (u128)c * LG[c];
            }
        }
        Lf = block_sum_u32<NT>(Lf, sh_u32);
        X = block_sum_u128<NT>(X, sh_u128);
        if (threadIdx.x == 0) {
            if (Lf) atomicAdd(&hagg[hi].L, Lf);
            if (X) atomic_add_u128(reinterpret_cast<unsigned long long *>(&hagg[hi].X), X);
        }
        __syncthreads();                               // the reductions' words are reused
    }
}

// hub rows, P1 step 3, a thread per hub: the row aggregates with the own community, the
// own and absent columns' weights (published to w_max), the node record
template <int NT>
__global__ void __launch_bounds__(NT) hub_p1_finish_kernel(
    const int64_t *__restrict__ off, const int32_t *__restrict__ lab, const HubInfo *__restrict__ hubs,
    int64_t nhubs, Batch B, const uint64_t *__restrict__ LG, HubAgg *hagg, NodeRec *__restrict__ rec,
    int32_t *__restrict__ Lall) {
    for (int64_t hi = (int64_t)blockIdx.x * NT + threadIdx.x; hi < nhubs; hi += (int64_t)gridDim.x * NT) {
        const HubInfo h = hubs[hi];
        const int32_t gi = graph_of(B, h.row);
        const int64_t d = off[h.row + 1] - off[h.row];
        HubAgg g = hagg[hi];
        const uint32_t own = g.own;
        const RowAgg a{(uint32_t)d, g.L + (own > 0 ? 1u : 0u), g.X + (u128)own * LG[own]};
        df wown{0.0f, 0.0f};
        if (own > 0) wown = column_weight(a, own, LG);
        NodeRec r;
        const df m = p1_row_result(a, own, wown, k_of(B, gi), LG, r, lab[h.row], wown, true);
        publish_max(B, gi, m, current_wmax(&B.wmax[gi]));
        rec[h.row] = r;
        Lall[h.row] = (int32_t)a.L;
        g.X = a.X;
        g.L = a.L;
        hagg[hi] = g;
    }
}

// hub rows, P1 step 4: the weight of every foreign column of each slot range, its cube root
// sigma kept for P2 (a column's weight depends only on the row's aggregates and its count,
// both final here), and the range's largest weight to w_max (a maximum, so the order of
// the ranges does not matter).  A positive sigma is stored negated when the column has a
// single member (no Type-II push to make), so that P2 reads one word instead of two; the
// sign change is exact, and a zero sigma (no push either) stays +0.
template <int NT>
__global__ void __launch_bounds__(NT) hub_p1_colmax_kernel(
    const int64_t *__restrict__ off, const HubInfo *__restrict__ hubs, const int32_t *__restrict__ sitem,
    const int32_t *__restrict__ srange, int64_t nsitems, Batch B, const uint64_t *__restrict__ LG,
    const int32_t *hkey, const uint32_t *hcnt, const HubAgg *__restrict__ hagg, df *hsig) {
    __shared__ df sh_df[NT / 32];
    for (int64_t it = blockIdx.x; it < nsitems; it += gridDim.x) {
        const int32_t hi = sitem[it];
        const HubInfo h = hubs[hi];
        const HubAgg g = hagg[hi];
        const RowAgg a{(uint32_t)(off[h.row + 1] - off[h.row]), g.L, g.X};
        const int64_t j0 = (int64_t)srange[it] * kHubSlotRange, j1 = min((int64_t)h.cap, j0 + (int64_t)kHubSlotRange);
        df cm{0.0f, 0.0f};
        for (int64_t j = j0 + threadIdx.x; j < j1; j += NT) {
            const int64_t s = h.tab + j;
            if (hkey[s] != kEmpty) {
                const df w = column_weight(a, hcnt[s], LG);
                cm = df_max(cm, w);
                const df sg = df_cbrt(w);
                hsig[s] = (hcnt[s] > 1 || !(sg.hi > 0.0f)) ? sg : df{-sg.hi, -sg.lo};
            }
        }
        cm = block_max_df<NT>(cm, sh_df);
        if (threadIdx.x == 0) {
            const int32_t gi = graph_of(B, h.row);
            publish_max(B, gi, cm, current_wmax(&B.wmax[gi]));
        }
        __syncthreads();                               // the reduction's words are reused
    }
}

// ======================================================================================
// G_x row offsets: nodes with dx >= 2 keep dx slots; xoff is the exclusive scan of
// those capacities, in one pass (decoupled look-back).  Tiles of kGxTile nodes are
// taken in ticket order; a tile publishes its own total at once and its inclusive
// prefix as soon as the tiles before it have, and its first warp sums the published
// words of its predecessors back to the nearest inclusive one, 32 tiles per step.  A predecessor has
// always started (its ticket is smaller), so every wait ends; the wait is bounded
// all the same (spin_limit reads of a word).  If the bound is ever reached, the tile
// flags err (bit 32, reported by rs_score as RS_ETIMEOUT) and takes its prefix from a
// direct sum of the capacities of every node before it instead, so the offsets stay
// exact.  withhold_tile >= 0 (a test hook, -1 otherwise) keeps that tile from
// publishing its words, so that the waits of the tiles after it run out.
// ======================================================================================
constexpr int kGxThreads = 256;
constexpr int kGxPer = kGxTile / kGxThreads;
constexpr unsigned long long kGxAgg = 1ull << 62, kGxIncl = 2ull << 62, kGxMask = (1ull << 62) - 1;

// status: one word per tile (flag in the top two bits), zeroed before the launch;
// ticket: zeroed before the launch.  Warp w of a tile scans its kGxPer runs of 32
// consecutive nodes (coalesced loads and stores), carrying its running total.
__global__ void __launch_bounds__(kGxThreads) gx_offsets_kernel(
    const NodeRec *__restrict__ rec, int64_t n, int64_t *__restrict__ xoff, unsigned long long *status,
    unsigned long long *ticket, int *err, long spin_limit, int64_t withhold_tile) {
    __shared__ int64_t warp_tot[kGxThreads / 32];
    __shared__ unsigned long long sh_tile;
    __shared__ int64_t sh_prefix;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) sh_tile = atomicAdd(ticket, 1ull);
    __syncthreads();
    const int64_t t = (int64_t)sh_tile;
    const int64_t base = t * kGxTile + (int64_t)wid * (32 * kGxPer);
    int32_t cap[kGxPer];
#pragma unroll
    for (int k = 0; k < kGxPer; ++k) {
        int64_t v = base + k * 32 + lane;
        int32_t dx = v < n ? rec[v].dx : 0;
        cap[k] = dx >= 2 ? dx : 0;
    }
    int64_t val[kGxPer];
    int64_t carry = 0;
#pragma unroll
    for (int k = 0; k < kGxPer; ++k) {
        int64_t x = cap[k];
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(FULL, x, o);
            if (lane >= o) x += y;
        }
        val[k] = carry + x;                           // inclusive within the warp's nodes
        carry += __shfl_sync(FULL, x, 31);
    }
    if (lane == 0) warp_tot[wid] = carry;
    __syncthreads();
    if (wid == 0) {
        // exclusive prefixes of the warps inside the tile, and the tile's total
        int64_t c = lane < kGxThreads / 32 ? warp_tot[lane] : 0, x = c;
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(FULL, x, o);
            if (lane >= o) x += y;
        }
        const int64_t total = __shfl_sync(FULL, x, 31);
        if (lane < kGxThreads / 32) warp_tot[lane] = x - c;
        int64_t excl = 0;
        const bool publish = t != withhold_tile;
        if (t == 0) {
            if (lane == 0 && publish) *(volatile unsigned long long *)&status[0] = kGxIncl | (unsigned long long)total;
        } else {
            if (lane == 0 && publish) *(volatile unsigned long long *)&status[t] = kGxAgg | (unsigned long long)total;
            // look back 32 tiles at a time: lane l reads tile hi - l; the nearest
            // inclusive word ends the walk, the aggregates after it are added
            bool gave_up = false;
            for (int64_t hi = t - 1;; hi -= 32) {
                const int64_t j = hi - lane;
                unsigned long long w = kGxIncl;          // before tile 0: an inclusive zero
                if (j >= 0) {
                    long spins = 0;
                    do {
                        w = *(volatile unsigned long long *)&status[j];
                    } while (!(w >> 62) && ++spins < spin_limit);
                }
                if (__any_sync(FULL, !(w >> 62))) {     // a wait ran out
                    gave_up = true;
                    break;
                }
                const unsigned inc = __ballot_sync(FULL, (w >> 62) == 2);
                const int stop = inc ? __ffs(inc) - 1 : 31;
                int64_t add = lane <= stop ? (int64_t)(w & kGxMask) : 0;
                for (int o = 16; o; o >>= 1) add += __shfl_xor_sync(FULL, add, o);
                excl += add;
                if (inc) break;
            }
            if (gave_up) {
                // the exact prefix from the node records themselves
                if (lane == 0) atomicOr(err, 32);
                int64_t sum = 0;
                for (int64_t v = lane; v < t * kGxTile; v += 32) {
                    const int32_t dx = rec[v].dx;
                    sum += dx >= 2 ? dx : 0;
                }
                for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(FULL, sum, o);
                excl = sum;
            }
            if (lane == 0 && publish)
                *(volatile unsigned long long *)&status[t] = kGxIncl | (unsigned long long)(excl + total);
        }
        if (lane == 0) sh_prefix = excl;
    }
    __syncthreads();
    const int64_t before = sh_prefix + warp_tot[wid];
    if (t == 0 && threadIdx.x == 0) xoff[0] = 0;
#pragma unroll
    for (int k = 0; k < kGxPer; ++k) {
        int64_t v = base + k * 32 + lane;
        if (v < n) xoff[v + 1] = before + val[k];
    }
}

// ======================================================================================
// P2
// ======================================================================================
// P2 for small and mid rows walks the cross list P1 wrote (the neighbours of
// another community, in id order) and the row aggregates; own-community
// neighbours are never touched again.

constexpr int kNarrowRows = 8;                 // rows per tile of the narrow mid and large rows

// Rows with at most 32 cross neighbours, tiles of R <= 32 consecutive rows of a list
// per warp (the small rows, R = 32, and the mid and large rows with dx <= 32, whose
// longer cross lists take smaller tiles so that more warps share them).  The
// union of the tile's cross lists is processed in chunks of whole rows, one
// entry per lane (a chunk ends before the first row that would not fit its 32
// lanes); lane l prepares and closes row l.  As no row spans two chunks, a
// community's count f and Type-II sum come from one warp match on
// (row, community).
// one G_x slot p of a row: its id and value, and for the first slot of an 8-slot sector of
// the slot space also the packed index entry xsk[p / 8] (searches of long out-lists read it;
// every slot inside a row is written once here, so the entries of sectors starting inside
// rows are complete when P2 ends)
__device__ __forceinline__ void gx_put(int32_t *xcol, df *xS, int32_t *xsk, int64_t p, int32_t u, df sig) {
    xcol[p] = u;
    xS[p] = sig;
    if ((p & 7) == 0) xsk[p >> 3] = u;
}

struct P2Tile {
    int32_t pre[33];            // prefix sums of dx over the tile
    int64_t rb[32], xb[32];     // cross list start (= CSR start), G_x row start
    int32_t dx[32], w[32];
    uint32_t d[32], L[32];
    uint64_t xlo[32], xhi[32];
    df sig1[32];
    int32_t no[32], ni[32];
    uint64_t st[32];
};

template <int R>
__global__ void __launch_bounds__(kThreads) p2_small_kernel(
    const int64_t *__restrict__ off, const int32_t *__restrict__ rows, int64_t nrows_host,
    const int32_t *__restrict__ nrows_dev, const uint64_t *__restrict__ LG, const NodeRec *__restrict__ rec, const RowSum *__restrict__ rsum,
    const int32_t *__restrict__ cl_col, const int32_t *__restrict__ cl_lab, unsigned long long *acc,
    const int64_t *__restrict__ xoff, int32_t *__restrict__ xcol, df *__restrict__ xS, int32_t *__restrict__ xsk,
    int32_t *__restrict__ xout, int32_t *__restrict__ xin, Strict SX) {
    __shared__ P2Tile tiles[kThreads / 32];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    P2Tile &T = tiles[wid];
    int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nrows = nrows_dev ? *nrows_dev : nrows_host;   // a list counted by p2_split, or the small rows
    for (int64_t t0 = warp * R; t0 < nrows; t0 += nwarps * R) {
        int64_t i = t0 + lane;
        bool have = lane < R && i < nrows;
        int32_t w = have ? rows[i] : 0;
        int32_t dx = 0;
        if (have) {
            int64_t b = off[w];
            NodeRec rw = rec[w];
            dx = rw.dx;
            T.rb[lane] = b;
            T.d[lane] = (uint32_t)(off[w + 1] - b);
            T.w[lane] = w;
            if (dx > 0) {
                RowSum rs = rsum[w];
                T.xlo[lane] = rs.xlo; T.xhi[lane] = rs.xhi; T.L[lane] = rs.L;
                RowAgg a{T.d[lane], rs.L, ((u128)rs.xhi << 64) | rs.xlo};
                T.sig1[lane] = df_cbrt(column_weight(a, 1, LG));
                T.xb[lane] = xoff[w];
            }
        }
        T.dx[lane] = dx;
        T.no[lane] = 0;
        T.ni[lane] = 0;
        int32_t incl = dx;
        for (int o = 1; o < 32; o <<= 1) {
            int32_t y = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += y;
        }
        int32_t DX = __shfl_sync(FULL, incl, 31);
        T.pre[lane + 1] = incl;
        if (lane == 0) T.pre[0] = 0;
        __syncwarp();
        for (int32_t e0 = 0; e0 < DX;) {
            // rows [.., rb) end within e0 + 32: the chunk is [e0, pre[rb])
            unsigned fit = __ballot_sync(FULL, incl <= e0 + 32);
            int32_t rb = 32 - __clz(fit);
            int32_t E = __shfl_sync(FULL, incl, rb - 1);
            int32_t e = e0 + lane;
            bool act = e < E;
            int32_t r = 0, u = -1, c = -1, j = 0;
            NodeRec ru{0, -1, 0};
            if (act) {
                int32_t lo = 0, hi = 32;
                while (hi - lo > 1) {
                    int32_t mid = (lo + hi) >> 1;
                    if (T.pre[mid] <= e) lo = mid; else hi = mid;
                }
                r = lo;
                j = e - T.pre[r];
                u = cl_col[T.rb[r] + j];
                c = cl_lab[T.rb[r] + j];
                ru = rec[u];
            }
            T.st[lane] = ru.s_fix;
            __syncwarp();
            unsigned am = __ballot_sync(FULL, act);
            unsigned long long key = ((unsigned long long)(uint32_t)r << 32) | (uint32_t)c;
            unsigned gc = 0;
            if (act) gc = __match_any_sync(am, key);
            df sig{0.0f, 0.0f};
            if (act) {
                uint32_t f = __popc(gc);
                u128 rest = 0;
                if (f > 1) {
                    unsigned m = gc & ~(1u << lane);
                    while (m) { rest += T.st[__ffs(m) - 1]; m &= m - 1; }
                }
                if (f == 1) sig = T.sig1[r];
                else {
                    RowAgg a{T.d[r], T.L[r], ((u128)T.xhi[r] << 64) | T.xlo[r]};
                    sig = df_cbrt(column_weight(a, f, LG));
                    push_type2(acc, u, sig, strict_rest(SX, off, T.w[r], u, rest));
                }
            }
            // G_x entries of this chunk, in id order within each row
            bool gx = act && T.dx[r] >= 2 && ru.dx >= 2;
            bool o = gx && rank_after(ru.dx, u, T.dx[r], T.w[r]);
            bool in = gx && !o;
            unsigned om = __ballot_sync(FULL, o), im = __ballot_sync(FULL, in);
            unsigned go = 0, gi = 0;
            if (o) go = __match_any_sync(om, r);
            if (in) gi = __match_any_sync(im, r);
            int32_t bo = o ? T.no[r] : 0, bi = in ? T.ni[r] : 0;
            __syncwarp();
            if (o) {
                int64_t p = T.xb[r] + bo + __popc(go & lanemask_lt());
                gx_put(xcol, xS, xsk, p, u, sig);
                if (lane == __ffs(go) - 1) T.no[r] = bo + __popc(go);
            }
            if (in) {
                int64_t p = T.xb[r] + T.dx[r] - 1 - (bi + __popc(gi & lanemask_lt()));
                gx_put(xcol, xS, xsk, p, u, sig);
                if (lane == __ffs(gi) - 1) T.ni[r] = bi + __popc(gi);
            }
            __syncwarp();
            e0 = E;
        }
        if (have) { xout[w] = T.no[lane]; xin[w] = T.ni[lane]; }
        __syncwarp();
    }
}

// Mid rows, one warp per row: a per-warp table (community -> count, Type-II
// sum) over the cross list, then the terms and the G_x entries in id order.
constexpr int kMidSlotBytes = 4 + 4 + 16;   // key, count, 2-word sum

__global__ void __launch_bounds__(kThreads) p2_mid_kernel(
    const int64_t *__restrict__ off, const int32_t *__restrict__ rows, const int32_t *__restrict__ nrows_dev, Batch B, int32_t dx_max, int32_t wslots,
    const uint64_t *__restrict__ LG, const NodeRec *__restrict__ rec, const RowSum *__restrict__ rsum,
    const int32_t *__restrict__ cl_col, const int32_t *__restrict__ cl_lab, unsigned long long *acc,
    const int64_t *__restrict__ xoff, int32_t *__restrict__ xcol, df *__restrict__ xS, int32_t *__restrict__ xsk,
    int32_t *__restrict__ xout, int32_t *__restrict__ xin, int *err, Strict SX, unsigned long long *wq) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint64_t stage[kThreads];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint64_t *st = stage + (threadIdx.x & ~31);
    unsigned char *base_w = smem + (size_t)wid * wslots * kMidSlotBytes;   // wslots >= every row's table
    const int64_t nrows = *nrows_dev;               // rows of this kernel, counted by p2_split
    for (int64_t i = warp_next(wq); i < nrows; i = warp_next(wq)) {
        int32_t w = rows[i];
        int64_t b = off[w];
        int d = (int)(off[w + 1] - b);
        NodeRec rw = rec[w];
        int dx = rw.dx;
        if (dx > dx_max || dx <= 32) continue;     // the CTA-per-row kernel / the tile kernel
        int32_t bo = 0, bi = 0;
        {
            uint32_t cap = dev_pow2_at_least(2u * (uint32_t)min(dx, k_of(B, graph_of(B, w))));
            Tab t;
            t.q = (unsigned long long *)base_w;
            t.key = (int32_t *)(base_w + 16 * wslots);
            t.cnt = (uint32_t *)(base_w + 20 * wslots);
            t.sig = nullptr;
            t.mask = cap - 1;
            for (uint32_t j = lane; j < cap; j += 32) { t.key[j] = kEmpty; t.cnt[j] = 0; t.q[2 * j] = 0; t.q[2 * j + 1] = 0; }
            __syncwarp();
            for (int base = 0; base < dx; base += 32) {
                int e = base + lane;
                bool act = e < dx;
                int32_t c = act ? cl_lab[b + e] : -1;
                st[lane] = act ? rec[cl_col[b + e]].s_fix : 0;
                __syncwarp();
                unsigned am = __ballot_sync(FULL, act);
                if (act) {
                    unsigned grp = __match_any_sync(am, c);
                    if (lane == __ffs(grp) - 1) {
                        int sl = tab_insert(t, c, __popc(grp), err);
                        if (sl >= 0) atomic_add_u128(t.q + 2 * sl, group_sum_all(st, grp));
                    }
                }
                __syncwarp();
            }
            RowSum rs = rsum[w];
            RowAgg a{(uint32_t)d, rs.L, ((u128)rs.xhi << 64) | rs.xlo};
            df sig1 = df_cbrt(column_weight(a, 1, LG));   // the usual count of a foreign community
            int64_t xb = xoff[w];
            for (int base = 0; base < dx; base += 32) {
                int e = base + lane;
                bool act = e < dx;
                int32_t u = act ? cl_col[b + e] : -1;
                int32_t c = act ? cl_lab[b + e] : -1;
                NodeRec ru{0, -1, 0};
                if (act) ru = rec[u];
                df sig{0.0f, 0.0f};
                bool ok = act;
                if (act) {
                    int sl = tab_find(t, c);
                    if (sl < 0) { atomicOr(err, 2); ok = false; }
                    else {
                        uint32_t f = t.cnt[sl];
                        sig = f == 1 ? sig1 : df_cbrt(column_weight(a, f, LG));
                        if (f > 1) {
                            u128 q = ((u128)t.q[2 * sl + 1] << 64) | t.q[2 * sl];
                            push_type2(acc, u, sig, strict_rest(SX, off, w, u, q - ru.s_fix));
                        }
                    }
                }
                if (dx >= 2) {
                    bool inx = ok && ru.dx >= 2;
                    bool o = inx && rank_after(ru.dx, u, dx, w);
                    bool in = inx && !o;
                    unsigned mo = __ballot_sync(FULL, o), mi = __ballot_sync(FULL, in);
                    if (o) gx_put(xcol, xS, xsk, xb + bo + __popc(mo & lanemask_lt()), u, sig);
                    if (in) gx_put(xcol, xS, xsk, xb + dx - 1 - (bi + __popc(mi & lanemask_lt())), u, sig);
                    bo += __popc(mo); bi += __popc(mi);
                }
            }
        }
        if (lane == 0) { xout[w] = bo; xin[w] = bi; }
        __syncwarp();
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
                                         int32_t *xsk, int32_t *sh_cnt /* 2 * NT/32 */) {
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned mo = __ballot_sync(FULL, out), mi = __ballot_sync(FULL, in);
    if (lane == 0) { sh_cnt[wid] = __popc(mo); sh_cnt[NT / 32 + wid] = __popc(mi); }
    __syncthreads();
    int32_t po = base_out, pi = base_in, to = 0, ti = 0;
    for (int j = 0; j < NT / 32; ++j) {
        if (j < wid) { po += sh_cnt[j]; pi += sh_cnt[NT / 32 + j]; }
        to += sh_cnt[j]; ti += sh_cnt[NT / 32 + j];
    }
    if (out) gx_put(xcol, xS, xsk, xb + po + __popc(mo & lanemask_lt()), u, sig);
    if (in) gx_put(xcol, xS, xsk, xb + dxw - 1 - (pi + __popc(mi & lanemask_lt())), u, sig);
    base_out += to; base_in += ti;
    __syncthreads();
}

template <int NT>
__global__ void __launch_bounds__(NT) p2_large_kernel(
    const int64_t *__restrict__ off, const int32_t *__restrict__ rows, const int32_t *__restrict__ nrows_dev, Batch B, int32_t dx_min,
    const uint64_t *__restrict__ LG, const NodeRec *__restrict__ rec, const RowSum *__restrict__ rsum,
    const int32_t *__restrict__ cl_col, const int32_t *__restrict__ cl_lab, unsigned long long *acc,
    const int64_t *__restrict__ xoff, int32_t *__restrict__ xcol, df *__restrict__ xS, int32_t *__restrict__ xsk,
    int32_t *__restrict__ xout, int32_t *__restrict__ xin, int *err, Strict SX, unsigned long long *wq) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int32_t sh_cnt[2 * NT / 32];
    __shared__ uint64_t stage[NT];
    int tid = threadIdx.x, lane = tid & 31;
    uint64_t *st = stage + (tid & ~31);
    const int64_t nrows = *nrows_dev;               // rows of this kernel, counted by p2_split
    __shared__ long long sh_next;
    for (int64_t i = cta_next(wq, &sh_next); i < nrows; i = cta_next(wq, &sh_next)) {
        int32_t w = rows[i];
        int64_t b = off[w];
        int d = (int)(off[w + 1] - b);
        NodeRec rw = rec[w];
        int dx = rw.dx;
        if (dx < dx_min) continue;                  // done by the warp-per-row kernel
        if (dx == 0) {
            if (tid == 0) { xout[w] = 0; xin[w] = 0; }
            continue;
        }
        uint32_t cap = dev_pow2_at_least(2u * (uint32_t)min(dx, k_of(B, graph_of(B, w))));
        Tab t = p2_table(smem, cap);
        for (uint32_t j = tid; j < cap; j += NT) {
            t.key[j] = kEmpty; t.cnt[j] = 0; t.q[2 * j] = 0; t.q[2 * j + 1] = 0;
        }
        __syncthreads();
        for (int base = 0; base < dx; base += NT) {
            int e = base + tid;
            bool act = e < dx;
            int32_t c = act ? cl_lab[b + e] : -1;
            st[lane] = act ? rec[cl_col[b + e]].s_fix : 0;
            __syncwarp();
            unsigned am = __ballot_sync(FULL, act);
            if (act) {
                unsigned grp = __match_any_sync(am, c);
                if (lane == __ffs(grp) - 1) {
                    int sl = tab_insert(t, c, __popc(grp), err);
                    if (sl >= 0) atomic_add_u128(t.q + 2 * sl, group_sum_all(st, grp));
                }
            }
            __syncwarp();
        }
        __syncthreads();
        RowSum rs = rsum[w];
        RowAgg a{(uint32_t)d, rs.L, ((u128)rs.xhi << 64) | rs.xlo};
        for (uint32_t j = tid; j < cap; j += NT)
            if (t.key[j] != kEmpty) t.sig[j] = df_cbrt(column_weight(a, t.cnt[j], LG));
        __syncthreads();
        int64_t xb = xoff[w];
        int32_t bo = 0, bi = 0;
        for (int base = 0; base < dx; base += NT) {
            int e = base + tid;
            bool act = e < dx;
            int32_t u = act ? cl_col[b + e] : -1;
            NodeRec ru{0, -1, 0};
            if (act) ru = rec[u];
            bool ok = act;
            df sig{0.0f, 0.0f};
            if (act) {
                int sl = tab_find(t, cl_lab[b + e]);
                if (sl < 0) { atomicOr(err, 2); ok = false; }
                else {
                    sig = t.sig[sl];
                    if (t.cnt[sl] > 1) {
                        u128 q = ((u128)t.q[2 * sl + 1] << 64) | t.q[2 * sl];
                        push_type2(acc, u, sig, strict_rest(SX, off, w, u, q - ru.s_fix));
                    }
                }
            }
            if (dx >= 2) {
                bool inx = ok && ru.dx >= 2;
                bool o = inx && rank_after(ru.dx, u, dx, w);
                gx_round<NT>(o, inx && !o, xb, dx, u, sig, bo, bi, xcol, xS, xsk, sh_cnt);
            }
        }
        if (tid == 0) { xout[w] = bo; xin[w] = bi; }
        __syncthreads();
    }
}

// hub rows, P2 step 1: Type-II group sums and per-chunk G_x counts; every entry's table slot
// (found once per group of lanes with the same community) is kept for step 3
template <int NT>
__global__ void __launch_bounds__(NT) hub_p2_insert_kernel(
    const int64_t *__restrict__ off, const int32_t *__restrict__ col, const HubInfo *__restrict__ hubs,
    const int32_t *__restrict__ items, const int32_t *__restrict__ chunks, int64_t nitems, int32_t chunk_len,
    const NodeRec *__restrict__ rec, const int32_t *hkey, unsigned long long *hq,
    int32_t *hitem_out, int32_t *hitem_in, int32_t *__restrict__ hslot, int *err) {
    __shared__ uint32_t sh_u32[NT / 32];
    __shared__ uint64_t stage[NT];
    int tid = threadIdx.x, lane = tid & 31;
    uint64_t *st = stage + (tid & ~31);
    for (int64_t it = blockIdx.x; it < nitems; it += gridDim.x) {
        HubInfo h = hubs[items[it]];
        int64_t b = off[h.row];
        int64_t d = off[h.row + 1] - b;
        int64_t lo = (int64_t)chunks[it] * chunk_len;
        int64_t hi = min(d, lo + chunk_len);
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
                const int leader = __ffs(grp) - 1;
                int s = -1;
                if (lane == leader) {
                    s = tab_find(t, ru.label);
                    if (s < 0) atomicOr(err, 4);
                    else atomic_add_u128(t.q + 2 * s, group_sum_all(st, grp));
                }
                hslot[h.ent + e] = __shfl_sync(grp, s, leader);
            } else if (act) {
                hslot[h.ent + e] = -1;
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

// hub rows, P2 step 2, a thread per hub: the row's G_x out and in counts, summed over its chunks
template <int NT>
__global__ void __launch_bounds__(NT) hub_p2_counts_kernel(
    const HubInfo *__restrict__ hubs, int64_t nhubs, const int32_t *hitem_out, const int32_t *hitem_in,
    int32_t *xout, int32_t *xin) {
    for (int64_t hi = (int64_t)blockIdx.x * NT + threadIdx.x; hi < nhubs; hi += (int64_t)gridDim.x * NT) {
        const HubInfo h = hubs[hi];
        int32_t so = 0, si = 0;
        for (int j = 0; j < h.n_items; ++j) {
            so += hitem_out[h.first_item + j];
            si += hitem_in[h.first_item + j];
        }
        xout[h.row] = so;
        xin[h.row] = si;
    }
}

// hub rows, P2 step 3: Type-II terms and the G_x entries of each chunk
template <int NT>
__global__ void __launch_bounds__(NT) hub_p2_emit_kernel(
    const int64_t *__restrict__ off, const int32_t *__restrict__ col, const HubInfo *__restrict__ hubs,
    const int32_t *__restrict__ items, const int32_t *__restrict__ chunks, int64_t nitems, int32_t chunk_len,
    const NodeRec *__restrict__ rec, const int32_t *__restrict__ hslot,
    const unsigned long long *hq, const df *hsig, const int32_t *hitem_out, const int32_t *hitem_in,
    unsigned long long *acc, const int64_t *__restrict__ xoff, int32_t *__restrict__ xcol,
    df *__restrict__ xS, int32_t *__restrict__ xsk, int *err, Strict SX) {
    __shared__ int32_t sh_cnt[2 * NT / 32];
    int tid = threadIdx.x;
    for (int64_t it = blockIdx.x; it < nitems; it += gridDim.x) {
        int32_t hidx = items[it];
        HubInfo h = hubs[hidx];
        int64_t b = off[h.row];
        int64_t d = off[h.row + 1] - b;
        int32_t ch = chunks[it];
        int64_t lo = (int64_t)ch * chunk_len;
        int64_t hi = min(d, lo + chunk_len);
        NodeRec rw = rec[h.row];
        int32_t bo = 0, bi = 0;
        for (int j = 0; j < ch; ++j) { bo += hitem_out[h.first_item + j]; bi += hitem_in[h.first_item + j]; }
        int64_t xb = xoff[h.row];
        for (int64_t base = lo; base < hi; base += NT) {
            int64_t e = base + tid;
            bool act = e < hi;
            int32_t u = act ? col[b + e] : -1;
            NodeRec ru{0, -1, 0};
            if (act) ru = rec[u];
            // the slot step 1 found (-1: own community, or a miss step 1 flagged)
            const int s = act ? hslot[h.ent + e] : -1;
            bool cross = s >= 0;
            df sig{0.0f, 0.0f};
            if (cross) {
                int64_t gs = h.tab + s;
                const df st = hsig[gs];                // negative: a single member, no push
                sig = st.hi < 0.0f ? df{-st.hi, -st.lo} : st;
                if (st.hi > 0.0f) {
                    u128 q = ((u128)hq[2 * gs + 1] << 64) | hq[2 * gs];
                    push_type2(acc, u, sig, strict_rest(SX, off, h.row, u, q - ru.s_fix, b + e));
                }
            }
            if (rw.dx >= 2) {
                bool inx = cross && ru.dx >= 2;
                bool o = inx && rank_after(ru.dx, u, rw.dx, h.row);
                gx_round<NT>(o, inx && !o, xb, rw.dx, u, sig, bo, bi, xcol, xS, xsk, sh_cnt);
            }
        }
    }
}

// ======================================================================================
// P3: Type-I triads from G_x triangles
// ======================================================================================
// The reverse value of a G_x edge.  Row x writes its in-neighbours (the G_x
// neighbours of lower rank) from the back of its G_x row in increasing id
// order, so its in-list read backwards from the row's last slot is sorted and
// S(x -> y) for an in-neighbour y is found by binary search there.  P3 needs
// the reverse values only of the edges of triangles.  It either looks them up
// per triangle (three searches in in-lists), or reads them from xR, which the
// mirror pass below fills for every G_x edge beforehand (one search per edge,
// in a short out-list).  The first wins when triangles are few per G_x edge
// (0.11 on the 1M-node DC-SBM graph), the second when they are many; the
// choice is a launch parameter (p3_mirror).
__device__ __forceinline__ df in_value(int32_t x, int32_t y, const int64_t *xoff, const int32_t *xcol,
                                       const df *xS, const int32_t *xin, int *err) {
    const int64_t last = xoff[x + 1] - 1;
    const int32_t len = xin[x];
    int32_t l = 0, h = len;
    while (l < h) {
        int32_t mid = (l + h) >> 1;
        if (xcol[last - mid] < y) l = mid + 1; else h = mid;
    }
    if (l < len && xcol[last - l] == y) return xS[last - l];
    atomicOr(err, 16);
    return df{0.0f, 0.0f};
}

// where P3 takes a reverse value: xR at the out-slot (mirror pass), or the
// in-list of the higher-ranked end
struct Rev {
    const df *xR;                   // null: look the values up
    const int64_t *xoff;
    const int32_t *xcol;
    const df *xS;
    const int32_t *xin;
    int *err;
    // S(hi -> lo) for the G_x edge whose out-slot (lo -> hi) is `slot`
    __device__ __forceinline__ df get(int64_t slot, int32_t hi, int32_t lo) const {
        return xR ? xR[slot] : in_value(hi, lo, xoff, xcol, xS, xin, err);
    }
};

// position of key in the sorted list xcol[lo, lo + len), or -1
__device__ __forceinline__ int64_t find_in_list(const int32_t *xcol, int64_t lo, int32_t len, int32_t key) {
    int32_t l = 0, h = len;
    while (l < h) {
        int32_t mid = (l + h) >> 1;
        if (xcol[lo + mid] < key) l = mid + 1; else h = mid;
    }
    return (l < len && xcol[lo + l] == key) ? lo + l : -1;
}

// lists of at most this many ids are binary-searched directly (they span at most 9 sectors)
constexpr int32_t kSkipMin = 64;

// position of key in the sorted list xcol[lo, lo + len), or -1.  A list of more than
// kSkipMin ids is searched first in xsk (xsk[t] = xcol[8 t], the first id of every 8-slot
// sector of the slot space, written by P2 with the slots), over the sectors that start
// inside the list, for the one sector that can hold key (the last whose first id is <= key;
// before them, the sector holding the list's head, when the list does not start a sector);
// that sector is then read with two 16-byte loads and its slots inside the list compared
// with key.  The chain of dependent loads of a long list thus runs over the packed index (8
// times denser than the list) and ends with one sector.  xcol is padded to whole sectors,
// so the last sector is readable.
__device__ __forceinline__ int64_t find_in_list_sk(const int32_t *xcol, const int32_t *xsk, int64_t lo, int32_t len,
                                                   int32_t key) {
    if (len <= kSkipMin) return find_in_list(xcol, lo, len, key);
    const int64_t end = lo + len;
    const int64_t t0 = (lo + 7) >> 3;                // first sector starting inside the list
    const int32_t ns = (int32_t)(((end - 1) >> 3) - t0 + 1);
    int32_t l = 0, h = ns;                           // first of them whose first id exceeds key
    while (l < h) {
        const int32_t mid = (l + h) >> 1;
        if (__ldg(xsk + t0 + mid) <= key) l = mid + 1; else h = mid;
    }
    const int64_t t = t0 + l - 1;
    if (t < (lo >> 3)) return -1;                    // key is below the first id, which starts a sector
    const int4 *v = reinterpret_cast<const int4 *>(xcol + 8 * t);
    const int4 x = __ldg(v), y = __ldg(v + 1);
    const int32_t e[8] = {x.x, x.y, x.z, x.w, y.x, y.y, y.z, y.w};
    const int64_t b = 8 * t;
    int64_t pos = -1;
#pragma unroll
    for (int j = 0; j < 8; ++j)
        if (e[j] == key && b + j >= lo && b + j < end) pos = b + j;
    return pos;
}

// P3m (mirror, when p3_mirror is set): every G_x out-slot (w -> u) receives the reverse value
// S(u -> w), which row u wrote at its in-slot for w.  Node u's slots are
// [xoff[u], xoff[u] + dx(u)), its in-slots the last xin(u) of them.  The slot
// space [0, xoff[n]) is cut into tiles of kMirTile consecutive slots, one
// tile per CTA trip, so the work per CTA does not depend on the in-degrees.
// The nodes a tile spans run from the node holding its first slot to the one
// holding the next tile's first slot (a table filled during P2, so no tile
// searches the offsets).  A tile stages their offsets in shared memory, counts
// their in-slots inside the tile and spreads only those over the threads; a
// slot's out-slot twin is found in w's out-list (w has the lower rank), by
// find_in_list_sk: a binary search, or for a list of more than kSkipMin ids one
// through the packed sector index.  A tile spanning more than kMirNodes nodes
// (long runs of nodes outside G_x) searches the offsets in global memory.
constexpr int kMirNodes = 1024;

// cover[t] = the node whose G_x row holds slot t kMirTile (t < tiles), and
// cover[tiles] = the node holding the last slot; every slot lies in exactly
// one non-empty row, so each entry is written once
__global__ void mirror_tiles_kernel(int64_t n, const int64_t *__restrict__ xoff, int32_t *__restrict__ cover) {
    const int64_t S = xoff[n];
    const int64_t tiles = (S + kMirTile - 1) / kMirTile;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = xoff[u], hi = xoff[u + 1];
        if (hi <= lo) continue;
        for (int64_t t = (lo + kMirTile - 1) / kMirTile; t * kMirTile < hi; ++t) cover[t] = (int32_t)u;
        if (hi == S) cover[tiles] = (int32_t)u;
    }
}

__device__ __forceinline__ int64_t last_leq(const int64_t *xoff, int64_t lo, int64_t hi, int64_t key) {
    // last index i in [lo, hi) with xoff[i] <= key (xoff[lo] <= key)
    while (hi - lo > 1) {
        int64_t mid = lo + ((hi - lo) >> 1);
        if (xoff[mid] <= key) lo = mid; else hi = mid;
    }
    return lo;
}

// copy S(u -> w) from u's in-slot sl to w's out-slot for u (found in w's out-list, through
// the packed index when the list is long)
__device__ __forceinline__ void mirror_one(int64_t sl, int32_t u, const int64_t *xoff, const int32_t *xcol,
                                           const int32_t *xsk, const df *xS, const int32_t *xout, df *xR, int *err) {
    const int32_t w = xcol[sl];
    const int64_t pos = find_in_list_sk(xcol, xsk, xoff[w], xout[w], u);
    if (pos >= 0) xR[pos] = xS[sl];
    else atomicOr(err, 16);
}

__global__ void __launch_bounds__(kThreads) gx_mirror_kernel(
    int64_t n, const int64_t *__restrict__ xoff, const int32_t *__restrict__ xcol, const df *__restrict__ xS,
    const int32_t *__restrict__ xout, const int32_t *__restrict__ xin, const int32_t *__restrict__ cover,
    df *__restrict__ xR, const int32_t *__restrict__ xsk, int *err) {
    __shared__ int64_t s_lo[kMirNodes];          // first in-slot of each staged node inside the tile
    __shared__ int32_t s_pre[kMirNodes + 1];     // prefix sums of the staged nodes' in-slots in the tile
    __shared__ int32_t s_wsum[kThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t S = xoff[n];
    const int64_t tiles = (S + kMirTile - 1) / kMirTile;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        int64_t s0 = t * kMirTile, s1 = min(S, s0 + kMirTile);
        // nodes [ulo, uhi): from the one holding s0 to the one holding s1 (or the last slot)
        int64_t ulo = cover[t], uhi = (int64_t)cover[t + 1] + 1;
        __syncthreads();                             // the previous tile's stage is free
        int32_t nn = (int32_t)(uhi - ulo);
        if (nn > kMirNodes) {
            for (int64_t sl = s0 + tid; sl < s1; sl += blockDim.x) {
                int64_t u = last_leq(xoff, ulo, uhi, sl);
                if (sl >= xoff[u + 1] - xin[u]) mirror_one(sl, (int32_t)u, xoff, xcol, xsk, xS, xout, xR, err);
            }
            continue;
        }
        // in-slots of each staged node inside [s0, s1): four consecutive nodes per thread
        constexpr int kPer = kMirNodes / kThreads;
        int32_t cnt[kPer];
        int32_t mine = 0;
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            int32_t i = tid * kPer + j;
            cnt[j] = 0;
            if (i < nn) {
                int64_t end = xoff[ulo + i + 1];
                int64_t lo = max(end - (int64_t)xin[ulo + i], s0);
                int64_t hi = min(end, s1);
                s_lo[i] = lo;
                cnt[j] = hi > lo ? (int32_t)(hi - lo) : 0;
            }
            mine += cnt[j];
        }
        int32_t incl = mine;
        for (int o = 1; o < 32; o <<= 1) {
            int32_t y = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) s_wsum[wid] = incl;
        __syncthreads();
        int32_t before = 0, total = 0;
        for (int j = 0; j < kThreads / 32; ++j) {
            if (j < wid) before += s_wsum[j];
            total += s_wsum[j];
        }
        int32_t run = before + incl - mine;
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            int32_t i = tid * kPer + j;
            if (i < nn) s_pre[i] = run;
            run += cnt[j];
        }
        if (tid == 0) s_pre[nn] = total;
        __syncthreads();
        for (int32_t q = tid; q < total; q += blockDim.x) {
            int32_t lo = 0, hi = nn;                    // last staged node with s_pre <= q
            while (hi - lo > 1) {
                int32_t mid = (lo + hi) >> 1;
                if (s_pre[mid] <= q) lo = mid; else hi = mid;
            }
            mirror_one(s_lo[lo] + (q - s_pre[lo]), (int32_t)(ulo + lo), xoff, xcol, xsk, xS, xout, xR, err);
        }
    }
}

// the three apex terms of triangle (a, b, c), rank a < b < c, added to the accumulators
__device__ __forceinline__ void triangle_terms(int32_t a, int32_t b, int32_t c, df Sab, df Sba, df Sac, df Sca,
                                               df Sbc, df Scb, unsigned long long *acc) {
    add_triangle(acc, a, b, c, triangle_term_values(Sab, Sba, Sac, Sca, Sbc, Scb));
}

// P3 lists the triangles of G_x once each, from their lowest-ranked node a
// (rank = (dx, id); a node's out-list holds its higher-ranked G_x neighbours,
// sorted by id).  Every pair {b, c} of a's out-neighbours is a candidate, and
// it closes a triangle iff the higher-ranked of the two is in the out-list of
// the lower-ranked one.  There are sum_a d+(a)(d+(a)-1)/2 candidates, several
// times fewer than the wedges a -> b -> c on these graphs.
//
// A warp takes 32 consecutive nodes and stages their out-lists (with each
// entry's G_x offset, out-degree and rank) in shared memory, window by window
// of at most kWinCap entries.  All candidate pairs of a window form one flat
// index space that the lanes share evenly (two per lane per trip): entry e
// owns the pairs (e, f > e) of its node.  The closing edge is looked up in the
// lower-ranked node's out-list in global memory by find_in_list_sk (a binary
// search, or for a long list one through the packed sector index).  Found
// triangles are queued in shared memory and finished a warp at a time, one per
// lane: the three forward values
// sit at the out-slots, the three reverse ones in xR (the mirror pass) or, with
// p3_mirror = 0, in the in-lists of the two higher-ranked nodes, and the terms
// of the three apexes are added.  Nodes with more than kWinCap out-neighbours
// (heavy nodes) are walked by wedges instead (p3_heavy_kernel).
constexpr int kP3Warps = kThreads / 32;

struct P3Stage {
    int64_t boff[kWinCap];          // xoff[b]
    int32_t nb[kWinCap];            // b
    int32_t bdeg[kWinCap];          // d+(b)
    int32_t bdx[kWinCap];           // dx(b): rank(b) = (dx(b), b)
    uint16_t ppre[kWinCap + 1];     // prefix sums of the pairs (e, f > e) owned by the entries
    uint8_t owner[kWinCap];         // lane (node) of the entry
    int32_t seg[33];                // first entry of each lane's node in the window
    int64_t aoff[32];               // xoff[a]
    // triangles found and not yet finished: the closing slot, the owner lane
    // and the window entries of the lower- and higher-ranked neighbours
    int64_t qpos[64];
    uint8_t qow[64], qlo[64], qhi[64];
};

// finish the first m (<= 32) queued triangles of the window, one per lane: the
// forward values are at the three out-slots
// the node of owner lane ow: base + ow, or (scrambled groups) the staged id anode[ow]
template <bool kScr>
__device__ __forceinline__ void p3_flush(const P3Stage &S, const int32_t *anode, int m, int64_t base, const df *xS,
                                         const Rev &R,
                                         unsigned long long *acc, int lane) {
    if (lane < m) {
        int ow = S.qow[lane], el = S.qlo[lane], eh = S.qhi[lane];
        int64_t ao = S.aoff[ow] - S.seg[ow];
        int64_t il = ao + el, ih = ao + eh, pc = S.qpos[lane];
        int32_t a = kScr ? anode[ow] : (int32_t)(base + ow), b = S.nb[el], c = S.nb[eh];
        df Sba = R.get(il, b, a), Sca = R.get(ih, c, a), Scb = R.get(pc, c, b);
        triangle_terms(a, b, c, xS[il], Sba, xS[ih], Sca, xS[pc], Scb, acc);
    }
}

__device__ __forceinline__ bool rank_less(int32_t dx1, int32_t id1, int32_t dx2, int32_t id2) {
    return dx1 < dx2 || (dx1 == dx2 && id1 < id2);
}

// Heavy nodes: a wedge walk, one CTA per task.  A task is a heavy node a with a block
// of kHvBlock of its out-neighbours b.  The CTA stages a's out-list A (sorted by id),
// kHvIds ids at a time, as a shared-memory hash table of 4-slot buckets (id -> position
// in the chunk, at most a quarter of the slots used) beside the value S(c->a) and the sum S(a->c) + S(c->a) for
// every c of the chunk.  Its warps then take the task's out-neighbours b one at a time: a warp
// streams b's out-list (the nodes c ranked above b), coalesced, and looks every c up in
// the table; a hit closes the triangle {a, b, c}, which is met once, at its
// middle-ranked node b.  When A takes several chunks, b's out-list is first cut to the
// chunk's id range.  There are several times more wedges than pairs on such nodes, but
// a wedge costs a coalesced load and a probe or two in shared memory where a pair
// costs a binary search in global memory.
//
// A third of the heavy wedges close on the 8M-node graph, so finishing the triangles
// dominates, and its atomics are cut down: hits are queued and finished a warp at a
// time (one triangle per lane); a's terms are summed in registers over the task, b's
// over the warp's walk of b (every queued triangle has the same b), and c's in two
// 64-bit words per staged position in shared memory (the term's low 48 bits and the
// rest, each added without reading the old value back), added to the accumulators once
// per chunk.  The integer sums are exact, so the bits do not depend on how they are split.
//
// The warp whose group holds a heavy node does not walk it: it appends the node's
// tasks to the task list (slots taken with an atomic counter), and p3_heavy_kernel,
// launched next on the same stream, runs them, a CTA per task.
constexpr int kHvIds = 1024;                  // ids of A staged per chunk
constexpr int kHvSlots = 4 * kHvIds;          // hash slots: the table is at most a quarter full
constexpr int kHvUnroll = 4;                  // 32-entry rows of b's out-list per trip
constexpr int kHvQ = 32 * kHvUnroll + 32;     // queued triangles per warp: < 32 left + one trip
constexpr int kHvWarps = kThreads / 32;

struct HvQueue {
    int32_t k[kHvQ];                          // c's entry in b's out-list
    int32_t c[kHvQ];
    int32_t pos[kHvQ];                        // c's position in the chunk of A
};
struct P3Heavy {
    int4 key[kHvSlots / 4];                   // the chunk's ids, 4 slots per bucket (-1: empty slot)
    uint16_t slot_pos[kHvSlots];              // their positions in the chunk
    df sca[kHvIds], pac[kHvIds];              // S(c->a), S(a->c) + S(c->a)
    unsigned long long clo[kHvIds], chi[kHvIds];   // c's terms of the chunk: bits [0, 48) and [48, 112)
    HvQueue q[kHvWarps];
    int64_t a, bA;
    int32_t dA, eb0, nb, next_b, stop;
};

// first position of the sorted p[0, cnt) (cnt >= 1) holding an id >= key, or cnt;
// the trip count depends on cnt alone
__device__ __forceinline__ int32_t lower_pos(const int32_t *p, int32_t cnt, int32_t key) {
    int32_t base = 0, len = cnt;
    while (len > 1) {
        const int32_t half = len >> 1;
        base = p[base + half] < key ? base + half : base;
        len -= half;
    }
    return base + (p[base] < key ? 1 : 0);
}

__device__ __forceinline__ uint32_t hv_hash(int32_t c, uint32_t mask) {
    return (((uint32_t)c * 0x9E3779B1u) >> 16) & mask;
}

// position of id c in the staged chunk, or -1.  The table is buckets of 4 slots, filled
// in slot order, at most a quarter of the slots used: one 16-byte load of the home bucket
// settles nearly every lookup (a key is there, or the bucket has an empty slot); a full
// home bucket (under 1% of them) sends the probe on to the next buckets.
__device__ __forceinline__ int32_t hv_find(const P3Heavy &H, int32_t c, uint32_t bmask) {
    uint32_t bk = hv_hash(c, bmask);
    for (uint32_t it = 0; it <= bmask; ++it) {
        const int4 q = H.key[bk];
        const int j = q.x == c ? 0 : q.y == c ? 1 : q.z == c ? 2 : q.w == c ? 3 : -1;
        if (j >= 0) return H.slot_pos[4 * bk + j];
        if (q.w < 0) return -1;
        bk = (bk + 1) & bmask;
    }
    return -1;
}

// c's term t added to its chunk sums in shared memory: bits [0, 48) of t to lo_w, bits
// [48, 112) to hi_w, each by an atomic add whose old value is not needed (no carry to
// propagate).  A position receives at most kHvBlock terms per chunk (one per out-neighbour
// b of the task), and every term is below 2^101 (at most 2^37 in value: each S(x->y) is
// the cube root of a weight below 31 * 2^31, so below 2^12, and a term is S * S * (S + S)),
// so the low word stays below 2^55 and the high one below 2^60; the chunk's sum is
// lo + hi * 2^48, exactly.
__device__ __forceinline__ void shared_add_split(unsigned long long *lo_w, unsigned long long *hi_w, u128 t) {
    atomicAdd(lo_w, (unsigned long long)((uint64_t)t & ((1ull << 48) - 1)));
    atomicAdd(hi_w, (unsigned long long)(uint64_t)(t >> 48));
}

// finish the m (<= 32) queued triangles {a, b, c} at queue entries [f, f + m) of the
// warp's current b, one per lane (all lanes call); the chunk of A starts at slot aslot0
__device__ __forceinline__ void hv_finish(P3Heavy &H, const HvQueue &Q, int f, int m, int32_t b, int64_t ob,
                                          int64_t aslot0, df Sab, df Sba, df Pab, const df *xS, const Rev &R,
                                          int lane, u128 &acc_a, u128 &acc_b) {
    if (lane < m) {
        const int32_t c = Q.c[f + lane], p = Q.pos[f + lane];
        const int64_t pc = ob + Q.k[f + lane];
        const df Sbc = xS[pc], Scb = R.get(pc, c, b), Sac = xS[aslot0 + p];
        const TriTerms t = triangle_term_values_p(Sab, Sba, Sac, H.sca[p], Sbc, Scb, H.pac[p], Pab);
        acc_a += t.a;
        acc_b += t.b;
        shared_add_split(&H.clo[p], &H.chi[p], t.c);
    }
}

// an out-neighbour b of the task (entry eb of A): its out-list [ob + s, ob + e) cut to
// the chunk's id range [lo_id, hi_id] when A takes several chunks, and the values of
// the edge a -> b
struct HvB {
    int32_t b, s, e;
    int64_t ob;
    df Sab, Sba;
};
__device__ __forceinline__ HvB hv_load_b(int32_t a, int64_t eb, bool cut, int32_t lo_id, int32_t hi_id,
                                         const int64_t *xoff, const int32_t *xcol, const df *xS, const Rev &R,
                                         const int32_t *xout) {
    HvB B;
    B.b = xcol[eb];
    B.ob = xoff[B.b];
    const int32_t db = xout[B.b];
    B.s = 0;
    B.e = db;
    if (cut && db > 0) {
        B.s = lower_pos(xcol + B.ob, db, lo_id);
        B.e = lower_pos(xcol + B.ob, db, hi_id + 1);
    }
    B.Sab = xS[eb];
    B.Sba = R.get(eb, B.b, a);
    return B;
}

// one warp's walk of out-neighbour b over the staged chunk (starting at slot aslot0):
// each trip loads and looks up kHvUnroll rows of 32 entries of b's out-list, queues the
// hits, and finishes the queued triangles 32 at a time (at the end of the list, the
// rest too); the finishing code is inlined once
__device__ __forceinline__ void hv_walk_b(P3Heavy &H, HvQueue &Q, const HvB &B, int64_t aslot0, uint32_t mask,
                                          const int32_t *xcol, const df *xS, const Rev &R,
                                          unsigned long long *acc, int lane, u128 &acc_a) {
    if (B.s >= B.e) return;
    const df Pab = df_add(B.Sab, B.Sba);
    int qn = 0;                                        // queued triangles (warp-uniform)
    u128 acc_b = 0;
    for (int32_t j0 = B.s; j0 < B.e; j0 += 32 * kHvUnroll) {
        int32_t c[kHvUnroll], pos[kHvUnroll];
#pragma unroll
        for (int u = 0; u < kHvUnroll; ++u) {
            const int32_t k = j0 + u * 32 + lane;
            c[u] = k < B.e ? xcol[B.ob + k] : -1;
        }
        // every row's home bucket is probed with no loop (b's out-list is already cut to
        // the chunk's id range, so an id outside it simply misses); the rare lanes whose
        // home bucket is full without their id probe on, in a branch the warp takes together
        bool more = false;
#pragma unroll
        for (int u = 0; u < kHvUnroll; ++u) {
            const uint32_t bk = hv_hash(c[u], mask);
            const int4 q = H.key[bk];
            const int j = q.x == c[u] ? 0 : q.y == c[u] ? 1 : q.z == c[u] ? 2 : q.w == c[u] ? 3 : -1;
            const bool valid = j0 + u * 32 + lane < B.e;
            pos[u] = valid && j >= 0 ? (int32_t)H.slot_pos[4 * bk + j] : -1;
            more |= valid && j < 0 && q.w >= 0;
        }
        if (__any_sync(FULL, more)) {
#pragma unroll
            for (int u = 0; u < kHvUnroll; ++u)
                if (pos[u] < 0 && j0 + u * 32 + lane < B.e) pos[u] = hv_find(H, c[u], mask);
        }
#pragma unroll
        for (int u = 0; u < kHvUnroll; ++u) {
            const bool hit = pos[u] >= 0;
            const unsigned hm = __ballot_sync(FULL, hit);
            if (hit) {
                const int slot = qn + __popc(hm & lanemask_lt());
                Q.k[slot] = j0 + u * 32 + lane;
                Q.c[slot] = c[u];
                Q.pos[slot] = pos[u];
            }
            qn += __popc(hm);
        }
        const bool last = j0 + 32 * kHvUnroll >= B.e;
        int f = 0;
        while (qn - f >= 32 || (last && qn > f)) {
            const int m = min(32, qn - f);
            __syncwarp();
            hv_finish(H, Q, f, m, B.b, B.ob, aslot0, B.Sab, B.Sba, Pab, xS, R, lane, acc_a, acc_b);
            f += m;
        }
        if (f > 0) {                                   // the rest (< 32) to the front
            __syncwarp();
            int32_t k = 0, cc = 0, pp = 0;
            if (lane < qn - f) { k = Q.k[f + lane]; cc = Q.c[f + lane]; pp = Q.pos[f + lane]; }
            __syncwarp();
            if (lane < qn - f) { Q.k[lane] = k; Q.c[lane] = cc; Q.pos[lane] = pp; }
            qn -= f;
        }
        __syncwarp();
    }
    acc_b = warp_sum_u128(acc_b);
    if (lane == 0 && acc_b) atomic_add_u128(acc + 2 * (int64_t)B.b, acc_b);
}

// groups of 32 nodes are handed out by an atomic counter (next_group, zeroed before
// the launch), so warps that drew light groups take more and no tail is left waiting.
// kScr (graphs built with RS_REORDER): lane j of group g takes node
// (32 g + j) * stride mod n (stride coprime to n), because consecutive ids then hold a
// community's heaviest nodes together and one group of them would be a long tail for
// its warp; otherwise lane j takes node 32 g + j and stride is unused.
template <bool kScr>
__global__ void __launch_bounds__(kThreads, 5) p3_list_kernel(
    int64_t n, const int64_t *__restrict__ xoff, const int32_t *__restrict__ xcol, const int32_t *__restrict__ xsk,
    const df *__restrict__ xS, Rev R, const int32_t *__restrict__ xout, const NodeRec *__restrict__ rec,
    unsigned long long *acc, unsigned long long *next_group, int64_t stride, unsigned long long *hvl, int64_t hvcap,
    unsigned long long *hv_count) {
    __shared__ P3Stage stage[kP3Warps];
    __shared__ int32_t s_anode[kScr ? kP3Warps * 32 : 1];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    P3Stage &S = stage[wid];
    int32_t *anode = s_anode + (kScr ? wid * 32 : 0);
    while (true) {
        unsigned long long ticket = 0;
        if (lane == 0) ticket = atomicAdd(next_group, 1ull);
        const int64_t base = (int64_t)__shfl_sync(FULL, ticket, 0) * 32;
        if (base >= n) break;
        int64_t av = base + lane;
        if (kScr && av < n) av = (int64_t)(((unsigned __int128)av * (uint64_t)stride) % (uint64_t)n);
        int32_t da = av < n ? xout[av] : 0;
        bool grp = da >= 2 && da <= kWinCap;
        int32_t mine = grp ? da : 0;
        int32_t incl = mine;
        for (int o = 1; o < 32; o <<= 1) {
            int32_t y = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += y;
        }
        int64_t ba = grp ? xoff[av] : 0;
        // windows of consecutive nodes whose entries fit kWinCap
        int32_t start = 0;
        while (true) {
            int32_t excl0 = start > 0 ? __shfl_sync(FULL, incl, start - 1) : 0;
            unsigned fitm = __ballot_sync(FULL, lane >= start && incl - excl0 <= kWinCap);
            if (start >= 32 || fitm == 0) break;
            int32_t end = 32 - __clz(fitm);               // lanes [start, end) fit
            int32_t Ew = __shfl_sync(FULL, incl, end - 1) - excl0;
            bool inwin = lane >= start && lane < end;
            int32_t e0 = incl - mine - excl0;              // this lane's first entry in the window
            if (Ew > 0) {
                // seg is nondecreasing over all 32 lanes: the entry j belongs to the
                // last lane o with seg[o] <= j (lanes without entries share the next seg)
                S.seg[lane] = lane < start ? 0 : (inwin ? e0 : Ew);
                if (lane == 0) S.seg[32] = Ew;
                S.aoff[lane] = ba;
                if (kScr) anode[lane] = (int32_t)av;
                __syncwarp();
                // entries, their data and the pair prefix sums, lanes over entries
                uint32_t carry = 0;
                if (lane == 0) S.ppre[0] = 0;
                for (int32_t j0 = 0; j0 < Ew; j0 += 32) {
                    int32_t j = j0 + lane;
                    uint32_t x = 0;
                    if (j < Ew) {
                        int32_t lo = 0, hi = 32;
                        while (hi - lo > 1) {
                            int32_t mid = (lo + hi) >> 1;
                            if (S.seg[mid] <= j) lo = mid; else hi = mid;
                        }
                        int32_t loc = j - S.seg[lo];
                        int32_t b = xcol[S.aoff[lo] + loc];
                        S.nb[j] = b;
                        S.owner[j] = (uint8_t)lo;
                        S.boff[j] = xoff[b];
                        S.bdeg[j] = xout[b];
                        S.bdx[j] = rec[b].dx;
                        x = (uint32_t)(S.seg[lo + 1] - S.seg[lo] - 1 - loc);   // pairs (j, f > j) of the node
                    }
                    for (int o = 1; o < 32; o <<= 1) {
                        uint32_t y = __shfl_up_sync(FULL, x, o);
                        if (lane >= o) x += y;
                    }
                    if (j < Ew) S.ppre[j + 1] = (uint16_t)(carry + x);
                    carry += __shfl_sync(FULL, x, 31);
                }
                __syncwarp();
                int32_t P = S.ppre[Ew];
                int qn = 0;                                // queued triangles (warp-uniform)
                // pairs per lane per trip: each search and the finishing code are inlined U
                // times, and the searches run one after another anyway, so a short unroll
                // keeps the code in the instruction cache (4 measured 10.07 against 9.10 ms
                // on the 8M-node graph)
                constexpr int U = 2;
                for (int32_t p0 = 0; p0 < P; p0 += 32 * U) {
                    int32_t lo_e[U], hi_e[U];
                    int64_t pos[U];
#pragma unroll
                    for (int q = 0; q < U; ++q) {
                        int32_t pv = p0 + q * 32 + lane;
                        lo_e[q] = -1;
                        hi_e[q] = 0;
                        if (pv < P) {
                            int32_t lo = 0, hi = Ew;        // last entry with ppre[e] <= pv
                            while (hi - lo > 1) {
                                int32_t mid = (lo + hi) >> 1;
                                if (S.ppre[mid] <= pv) lo = mid; else hi = mid;
                            }
                            int32_t f = lo + 1 + (pv - S.ppre[lo]);
                            bool e_low = rank_less(S.bdx[lo], S.nb[lo], S.bdx[f], S.nb[f]);
                            lo_e[q] = e_low ? lo : f;
                            hi_e[q] = e_low ? f : lo;
                        }
                    }
#pragma unroll
                    for (int q = 0; q < U; ++q)
                        pos[q] = lo_e[q] >= 0 ? find_in_list_sk(xcol, xsk, S.boff[lo_e[q]], S.bdeg[lo_e[q]], S.nb[hi_e[q]])
                                          : -1;
#pragma unroll
                    for (int q = 0; q < U; ++q) {
                        bool hit = pos[q] >= 0;
                        unsigned hm = __ballot_sync(FULL, hit);
                        if (hit) {
                            int slot = qn + __popc(hm & lanemask_lt());
                            S.qpos[slot] = pos[q];
                            S.qow[slot] = S.owner[lo_e[q]];
                            S.qlo[slot] = (uint8_t)lo_e[q];
                            S.qhi[slot] = (uint8_t)hi_e[q];
                        }
                        qn += __popc(hm);
                        if (qn >= 32) {                        // a full warp of triangles
                            __syncwarp();
                            p3_flush<kScr>(S, anode, 32, base, xS, R, acc, lane);
                            __syncwarp();
                            if (lane < qn - 32) {
                                S.qpos[lane] = S.qpos[32 + lane];
                                S.qow[lane] = S.qow[32 + lane];
                                S.qlo[lane] = S.qlo[32 + lane];
                                S.qhi[lane] = S.qhi[32 + lane];
                            }
                            qn -= 32;
                            __syncwarp();
                        }
                    }
                }
                __syncwarp();
                p3_flush<kScr>(S, anode, qn, base, xS, R, acc, lane);   // the window's stage is reused next
                qn = 0;
                __syncwarp();
            }
            start = end;
        }
        // heavy nodes' tasks go to the list (its capacity bounds their number, so the
        // error branch is not taken)
        if (da > kWinCap) {
            const int32_t nt = (da + kHvBlock - 1) / kHvBlock;
            const unsigned long long h = atomicAdd(hv_count, (unsigned long long)nt);
            if (h + nt <= (unsigned long long)hvcap) {
                for (int32_t i = 0; i < nt; ++i) hvl[h + i] = (unsigned long long)av << 32 | (unsigned)i;
            } else {
                atomicOr(R.err, 64);
            }
        }
    }
}

// the heavy-node tasks listed by p3_list_kernel, a CTA per task, claimed with an atomic
// counter; the CTA's warps claim the task's out-neighbours b from a counter in shared
// memory (dynamic shared memory: sizeof(P3Heavy))
__global__ void __launch_bounds__(kThreads, 3) p3_heavy_kernel(
    int64_t n, const int64_t *__restrict__ xoff, const int32_t *__restrict__ xcol, const df *__restrict__ xS,
    Rev R, const int32_t *__restrict__ xout, unsigned long long *acc, const unsigned long long *__restrict__ hvl,
    int64_t hvcap, const unsigned long long *hv_count, unsigned long long *hv_next) {
    extern __shared__ __align__(16) unsigned char hv_smem[];
    P3Heavy &H = *reinterpret_cast<P3Heavy *>(hv_smem);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, tid = threadIdx.x;
    HvQueue &Q = H.q[wid];
    unsigned long long lim = *hv_count;
    if (lim > (unsigned long long)hvcap) lim = (unsigned long long)hvcap;
    if (lim == 0) return;
    for (int i = tid; i < kHvIds; i += kThreads) {
        H.clo[i] = 0;
        H.chi[i] = 0;
    }
    while (true) {
        __syncthreads();                               // the previous task is flushed
        if (tid == 0) {
            const unsigned long long t = atomicAdd(hv_next, 1ull);
            H.stop = t >= lim;
            H.a = -1;
            if (!H.stop) {
                const unsigned long long w = hvl[t];
                const int64_t a = (int64_t)(w >> 32), blk = (int64_t)(w & 0xffffffffull);
                if (a >= n || xout[a] <= kWinCap || blk * kHvBlock >= xout[a]) {
                    atomicOr(R.err, 64);
                } else {
                    H.a = a;
                    H.bA = xoff[a];
                    H.dA = xout[a];
                    H.eb0 = (int32_t)(blk * kHvBlock);
                    H.nb = min(kHvBlock, H.dA - H.eb0);
                }
            }
        }
        __syncthreads();
        if (H.stop) break;
        if (H.a < 0) continue;
        const int32_t a = (int32_t)H.a, dA = H.dA, eb0 = H.eb0, nb = H.nb;
        const int64_t bA = H.bA;
        u128 acc_a = 0;
        for (int32_t k0 = 0; k0 < dA; k0 += kHvIds) {
            const int32_t cnt = min(kHvIds, dA - k0);
            const uint32_t buckets = max(32u, dev_pow2_at_least((uint32_t)cnt)), mask = buckets - 1;
            for (uint32_t i = tid; i < buckets; i += kThreads) H.key[i] = make_int4(-1, -1, -1, -1);
            if (tid == 0) H.next_b = 0;
            __syncthreads();
            for (int32_t i = tid; i < cnt; i += kThreads) {
                const int64_t sl = bA + k0 + i;
                const int32_t c = xcol[sl];
                // the first free slot of the first bucket with one, from the home bucket on
                // (the ids are distinct and at most a quarter of the slots are used, so one
                // is found); slots fill in order, so a bucket with an empty last slot has
                // room and holds every key that hashes to it
                int32_t *keys = reinterpret_cast<int32_t *>(H.key);
                uint32_t bk = hv_hash(c, mask), slot = 4u * kHvSlots;
                for (uint32_t it = 0; it <= mask && slot >= 4u * kHvSlots; ++it) {
                    for (int j = 0; j < 4; ++j)
                        if (atomicCAS(&keys[4 * bk + j], -1, c) == -1) { slot = 4 * bk + j; break; }
                    bk = (bk + 1) & mask;
                }
                if (slot < 4u * kHvSlots) H.slot_pos[slot] = (uint16_t)i;
                else atomicOr(R.err, 64);
                const df sac = xS[sl], sca = R.get(sl, c, a);
                H.sca[i] = sca;
                H.pac[i] = df_add(sac, sca);
            }
            __syncthreads();
            const int32_t lo_id = xcol[bA + k0], hi_id = xcol[bA + k0 + cnt - 1];
            const bool cut = dA > kHvIds;
            // the warp claims out-neighbours one at a time; the next one's data is loaded
            // while the current one is walked
            auto claim = [&]() {
                int32_t j = 0;
                if (lane == 0) j = atomicAdd(&H.next_b, 1);
                return __shfl_sync(FULL, j, 0);
            };
            int32_t j = claim();
            HvB cur{};
            if (j < nb) cur = hv_load_b(a, bA + eb0 + j, cut, lo_id, hi_id, xoff, xcol, xS, R, xout);
            while (j < nb) {
                const int32_t jn = claim();
                HvB nxt{};
                if (jn < nb) nxt = hv_load_b(a, bA + eb0 + jn, cut, lo_id, hi_id, xoff, xcol, xS, R, xout);
                hv_walk_b(H, Q, cur, bA + k0, mask, xcol, xS, R, acc, lane, acc_a);
                j = jn;
                cur = nxt;
            }
            __syncthreads();
            // c's sums of the chunk to the accumulators, zeroed for the next chunk
            for (int32_t i = tid; i < cnt; i += kThreads) {
                const unsigned long long lo = H.clo[i], hi = H.chi[i];
                if (lo | hi) {
                    atomic_add_u128(acc + 2 * (int64_t)xcol[bA + k0 + i], ((u128)hi << 48) + lo);
                    H.clo[i] = 0;
                    H.chi[i] = 0;
                }
            }
            __syncthreads();
        }
        acc_a = warp_sum_u128(acc_a);
        if (lane == 0 && acc_a) atomic_add_u128(acc + 2 * (int64_t)a, acc_a);
    }
}

// ======================================================================================
// Strict reading: X(w, u) for every pushed pair, from the closed triads (u, w, v)
// with C(v) = C(u) != C(w): for every intra-community edge {u, v} (u < v) and
// every common neighbour w of another community, s_v is added at u's entry in
// w's row and s_u at v's.  The shorter row of u, v is walked; w is looked up in
// the other row and the entries in w's row by binary search (rows are sorted).
// ======================================================================================
__device__ __forceinline__ int64_t csr_find(const int64_t *off, const int32_t *col, int32_t row, int32_t key) {
    int64_t lo = off[row], hi = off[row + 1], end = hi;
    while (lo < hi) {
        int64_t mid = lo + ((hi - lo) >> 1);
        if (col[mid] < key) lo = mid + 1; else hi = mid;
    }
    return (lo < end && col[lo] == key) ? lo : -1;
}

__global__ void __launch_bounds__(kThreads) strict_pairs_kernel(int64_t n, const int64_t *__restrict__ off,
                                                                const int32_t *__restrict__ col,
                                                                const int32_t *__restrict__ lab,
                                                                const NodeRec *__restrict__ rec,
                                                                unsigned long long *sx) {
    int lane = threadIdx.x & 31;
    int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = w0; u < n; u += nw) {                 // a warp per row u, lanes over its entries v
        int32_t cu = lab[u];
        int64_t bu = off[u], du = off[u + 1] - bu;
        for (int64_t e = lane; e < du; e += 32) {
            int32_t v = col[bu + e];
            if (v <= u || lab[v] != cu) continue;
            int64_t bv = off[v], dv = off[v + 1] - bv;
            bool walk_u = du <= dv;
            int32_t o = walk_u ? v : (int32_t)u;
            int64_t ba = walk_u ? bu : bv, da = walk_u ? du : dv;
            uint64_t su = rec[u].s_fix, sv = rec[v].s_fix;
            for (int64_t j = 0; j < da; ++j) {
                int32_t w = col[ba + j];
                if (w == o || lab[w] == cu) continue;
                if (csr_find(off, col, o, w) < 0) continue;
                int64_t pu = csr_find(off, col, w, (int32_t)u), pv = csr_find(off, col, w, v);
                if (sv && pu >= 0) atomic_add_u128(sx + 2 * pu, (u128)sv);
                if (su && pv >= 0) atomic_add_u128(sx + 2 * pv, (u128)su);
            }
        }
    }
}

// ======================================================================================
// P2 row lists by cross degree (known after P1): each P2 kernel then walks only its rows
//   0 mid and large rows, dx <= 32 (tiles)   1 mid rows, 32 < dx <= 128 (p2_mid, 256 slots)
//   2 unused                                 3 large rows, 32 < dx <= min(128, dx_cta) (p2_mid, 256)
//   4 large rows, dx > dx_cta (p2_large)     5 mid rows, dx > 128 (p2_mid, 512 slots)
//   6 large rows, 128 < dx <= dx_cta (p2_mid, 512 slots)
// ======================================================================================
constexpr int kP2Lists = 7;
constexpr int32_t kSmallTableDx = 128;        // rows up to this cross degree fit 256-slot tables

__device__ __forceinline__ void append_row(int32_t *list, int32_t *cnt, bool take, int32_t v) {
    unsigned m = __ballot_sync(FULL, take);
    int lane = threadIdx.x & 31;
    int32_t base = 0;
    if (m && lane == __ffs(m) - 1) base = atomicAdd(cnt, __popc(m));
    base = __shfl_sync(FULL, base, __ffs(m ? m : 1u) - 1);
    if (take) list[base + __popc(m & lanemask_lt())] = v;
}

// list 0 has room for n_mid + n_large rows, the other mid lists for n_mid, the large ones for n_large
__host__ __device__ __forceinline__ int64_t p2_list_start(int c, int64_t n_mid, int64_t n_large) {
    const int mids_before[kP2Lists] = {0, 1, 2, 2, 2, 2, 3};
    const int larges_before[kP2Lists] = {0, 1, 1, 1, 2, 3, 3};
    return mids_before[c] * n_mid + larges_before[c] * n_large;
}

__global__ void p2_split_kernel(const int32_t *__restrict__ rows_mid, int64_t n_mid,
                                const int32_t *__restrict__ rows_large, int64_t n_large,
                                const NodeRec *__restrict__ rec, int32_t dx_cta, int32_t *lists, int32_t *cnt) {
    int64_t total = n_mid + n_large;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x; i0 < total; i0 += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = i0 + threadIdx.x;
        bool act = i < total;
        bool mid = i < n_mid;
        int32_t v = act ? (mid ? rows_mid[i] : rows_large[i - n_mid]) : 0;
        int32_t dx = act ? rec[v].dx : 0;
        int cls = -1;
        if (act) {
            if (dx <= 32) cls = 0;                              // the tile kernel, either class
            else if (mid) cls = dx <= kSmallTableDx ? 1 : 5;
            else cls = dx > dx_cta ? 4 : dx <= kSmallTableDx ? 3 : 6;
        }
        for (int c = 0; c < kP2Lists; ++c)
            append_row(lists + p2_list_start(c, n_mid, n_large), cnt + c, cls == c, v);
    }
}

// ======================================================================================
// finalize: R(u) = acc(u) / (w_max d (d - 1))
// ======================================================================================
__global__ void graph_scale_kernel(const unsigned long long *__restrict__ wmax_bits, int32_t ng, double *winv) {
    int32_t gi = blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= ng) return;
    double wm = __longlong_as_double((long long)wmax_bits[gi]);
    winv[gi] = wm > 0.0 ? 1.0 / wm : 0.0;
}

// one graph (gid null): every CTA takes 1 / w_max itself; a batch reads the
// per-graph reciprocals graph_scale_kernel wrote.  A reordered graph (perm) writes
// each score at the caller's id of its node.
__global__ void __launch_bounds__(kThreads) finalize_kernel(
    int64_t n, const int64_t *__restrict__ off, const unsigned long long *__restrict__ acc,
    const int32_t *__restrict__ gid, const double *__restrict__ winv, const unsigned long long *__restrict__ wmax_bits,
    const double *__restrict__ RD, const int32_t *__restrict__ perm, double *scores) {
    __shared__ double sh_w;
    if (!gid) {
        if (threadIdx.x == 0) {
            double wm = __longlong_as_double((long long)wmax_bits[0]);
            sh_w = wm > 0.0 ? 1.0 / wm : 0.0;
        }
        __syncthreads();
    }
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
        int64_t d = off[u + 1] - off[u];
        double r = 0.0;
        if (d >= 2) {
            double W = gid ? winv[gid[u]] : sh_w;
            u128 s = ((u128)acc[2 * u + 1] << 64) | acc[2 * u];
            if (s && W > 0.0) r = u128_to_double(s, -kAccFrac) * W * RD[d];
        }
        scores[perm ? (int64_t)perm[u] : u] = r;
    }
}

}  // namespace

// ======================================================================================
// host orchestration
// ======================================================================================
// dynamic shared memory limits of the table kernels, set once per process
int rs::prepare_score_kernels() {
    static int done = 0;
    if (done) return 0;
    const int p2_mid_smem = kMidWarps * kWarpCap * kMidSlotBytes;
    RS_CUDA_TRY(cudaFuncSetAttribute(p1_large_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, 8 * kMidCap));
    RS_CUDA_TRY(cudaFuncSetAttribute(p1_large_kernel<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, 8 * kMidCap));
    RS_CUDA_TRY(cudaFuncSetAttribute(p1_large_kernel<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, 8 * kMidCap));
    RS_CUDA_TRY(cudaFuncSetAttribute(p2_large_kernel<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, 32 * kMidCap));
    RS_CUDA_TRY(cudaFuncSetAttribute(p2_large_kernel<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, 32 * kMidCap));
    RS_CUDA_TRY(cudaFuncSetAttribute(p2_large_kernel<1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, 32 * kMidCap));
    RS_CUDA_TRY(cudaFuncSetAttribute(p2_mid_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, p2_mid_smem));
    RS_CUDA_TRY(cudaFuncSetAttribute(p3_heavy_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)sizeof(P3Heavy)));
    RS_CUDA_TRY(cudaFuncSetAttribute(p1_small_staged_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(kStageWarps * (sizeof(SmallTile) + sizeof(SmallStage)))));
    done = 1;
    return 0;
}

// the CTA-per-row kernels at the tuned CTA size
template <int NT>
static void launch_p1_large(rs_graph *g, const Batch &B, int *err, size_t smem, cudaStream_t st) {
    p1_large_kernel<NT><<<grid_for(g->n_large, 1, 4), NT, smem, st>>>(
        g->off, g->col, g->lab, g->rows_large, g->n_large, B, g->LG, g->rec, g->Lall, err,
        g->rsum, g->cl_col, g->cl_lab, g->wq + 1);
}
template <int NT>
static void launch_p2_large(rs_graph *g, const Batch &B, int *err, size_t smem, cudaStream_t st) {
    int32_t *L4 = g->p2rows + p2_list_start(4, g->n_mid, g->n_large);
    p2_large_kernel<NT><<<grid_for(g->n_large, 1, 2), NT, smem, st>>>(
        g->off, L4, g->p2cnt + 4, B, g->tune.p2_cta_dx + 1, g->LG, g->rec, g->rsum, g->cl_col,
        g->cl_lab, g->acc, g->xoff, g->xcol, g->xS, g->xsk, g->xout, g->xin, err, Strict{g->col, g->sx}, g->wq + 6);
}

// a stride near n / golden ratio, coprime to n (a bijection of [0, n) by multiplication)
static int64_t p3_stride(int64_t n) {
    if (n < 3) return 1;
    auto gcd = [](int64_t a, int64_t b) { while (b) { int64_t t = a % b; a = b; b = t; } return a; };
    int64_t st = (int64_t)((double)n * 0.6180339887) | 1;
    while (st < n && gcd(st, n) != 1) st += 2;
    return st < n ? st : 1;
}

int rs::score_graph(rs_graph *g, double *scores, cudaStream_t s) {
    int64_t n = g->n;
    g->scored_version = g->version;
    if (n == 0) return 0;
    constexpr int NT = kThreads;
    int *err = g->d_flag + 4;
    const int cps = g->tune.ctas_per_sm;
    if (int rc = prepare_score_kernels()) return rc;
    prof_begin(g, s);
    RS_CUDA_TRY(cudaMemsetAsync(g->wmax_bits, 0, g->n_graphs * sizeof(unsigned long long), s));
    Batch B{g->gid, g->gk, g->k, g->wmax_bits};
    RS_CUDA_TRY(cudaMemsetAsync(g->acc, 0, 2 * n * sizeof(unsigned long long), s));
    RS_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), s));
    // row counters and the G_x scan's ticket and tile words
    RS_CUDA_TRY(cudaMemsetAsync(g->wq, 0, wq_hv_word(n) * sizeof(unsigned long long), s));
    if (g->n_hubs) {
        RS_CUDA_TRY(cudaMemsetAsync(g->hkey, 0xFF, g->hub_slots * sizeof(int32_t), s));
        RS_CUDA_TRY(cudaMemsetAsync(g->hcnt, 0, g->hub_slots * sizeof(uint32_t), s));
        RS_CUDA_TRY(cudaMemsetAsync(g->hq, 0, 2 * g->hub_slots * sizeof(unsigned long long), s));
        RS_CUDA_TRY(cudaMemsetAsync(g->hagg, 0, g->n_hubs * sizeof(HubAgg), s));
    }
    prof_mark(g, s, "memset", false);
    size_t p1_smem = 8 * (size_t)g->large_cap, p2_smem = 32 * (size_t)g->large_cap;
    // streams of the row kernels (rows_streams): every class on its own stream (0); the hub
    // chain on stream 3 and every other class in turn on stream 0 (1); every kernel in turn
    // on the step's stream (2).  On large graphs with hub rows each class fills the GPU alone,
    // and the classes spread over six streams held the hub chain back (8M-node hub-skewed
    // graph: step 65.7 ms against 63.9 with two streams; a batch of 1,024 graphs: 46.5 against
    // 42.1 ms); on smaller graphs the classes' long per-row chains overlap best on separate
    // streams (1M-node graph without hubs: 0.901 against 1.039 ms; a 1.2M-node graph with 489
    // hubs: 1.095 against 1.189 ms).  The automatic choice (-1) takes two streams for graphs
    // with hub rows and at least kRowsTwoStreamNnz CSR entries.
    constexpr int64_t kRowsTwoStreamNnz = 32000000;
    const int rmode = g->tune.rows_streams >= 0 ? g->tune.rows_streams
                                                : (g->n_hubs && g->nnz >= kRowsTwoStreamNnz ? 1 : 0);
    auto AX = [&](int i) -> cudaStream_t {
        if (rmode == 2) return s;
        if (rmode == 1) return i == 3 ? g->aux[3] : g->aux[0];
        return g->aux[i];
    };
    // ---- P1: the larger classes are launched first (with per-class streams, on
    //      high-priority ones), so their maxima seed w_max early and most small rows skip
    //      theirs (the small rows fill in at the lowest priority)
    if (rmode != 2)
        if (int rc = fork_aux(g, s)) return rc;
    if (g->n_hubs) {
        hub_p1_insert_kernel<NT><<<grid_for(g->n_hub_items, 1, 8), NT, 0, AX(3)>>>(
            g->off, g->col, g->lab, g->hubs, g->hub_items, g->hub_item_chunk, g->n_hub_items,
            g->tune.hub_chunk, g->hkey, g->hcnt, g->hagg, err);
        RS_LAUNCHED(g, AX(3), "hub_p1_insert");
        hub_p1_sums_kernel<NT><<<grid_for(g->n_hub_sitems, 1, 8), NT, 0, AX(3)>>>(
            g->hubs, g->hub_sitem, g->hub_srange, g->n_hub_sitems, g->LG, g->hkey, g->hcnt, g->hagg);
        RS_LAUNCHED(g, AX(3), "hub_p1_sums");
        hub_p1_finish_kernel<NT><<<(unsigned)((g->n_hubs + NT - 1) / NT), NT, 0, AX(3)>>>(
            g->off, g->lab, g->hubs, g->n_hubs, B, g->LG, g->hagg, g->rec, g->Lall);
        RS_LAUNCHED(g, AX(3), "hub_p1_finish");
        hub_p1_colmax_kernel<NT><<<grid_for(g->n_hub_sitems, 1, 8), NT, 0, AX(3)>>>(
            g->off, g->hubs, g->hub_sitem, g->hub_srange, g->n_hub_sitems, B, g->LG, g->hkey, g->hcnt, g->hagg,
            g->hsig);
        RS_LAUNCHED(g, AX(3), "hub_p1_colmax");
    }
    if (g->n_large) {
        switch (g->tune.p1_cta_threads) {
        case 128: launch_p1_large<128>(g, B, err, p1_smem, AX(2)); break;
        case 512: launch_p1_large<512>(g, B, err, p1_smem, AX(2)); break;
        default: launch_p1_large<256>(g, B, err, p1_smem, AX(2)); break;
        }
        RS_LAUNCHED(g, AX(2), "p1_large");
    }
    if (g->n_mid) {
        p1_mid_kernel<<<grid_for(g->n_mid * 32, NT, cps), NT, 0, AX(4)>>>(
            g->off, g->col, g->lab, g->rows_mid, g->n_mid, B, g->LG, g->rec, g->Lall, err,
            g->rsum, g->cl_col, g->cl_lab, g->wq + 0);
        RS_LAUNCHED(g, AX(4), "p1_mid");
    }
    if (g->n_small) {
        if (g->tune.p1_stage)
            p1_small_staged_kernel<<<grid_for(g->n_small, kStageWarps * 32, cps), kStageWarps * 32,
                                     kStageWarps * (sizeof(SmallTile) + sizeof(SmallStage)), AX(0)>>>(
                g->off, g->col, g->lab, g->rows_small, g->n_small, B, g->LG, g->rec, g->Lall,
                g->rsum, g->cl_col, g->cl_lab);
        else
            p1_small_kernel<<<grid_for(g->n_small, NT, cps), NT, 0, AX(0)>>>(
                g->off, g->col, g->lab, g->rows_small, g->n_small, B, g->LG, g->rec, g->Lall,
                g->rsum, g->cl_col, g->cl_lab);
        RS_LAUNCHED(g, AX(0), "p1_small");
    }
    if (rmode != 2)
        if (int rc = join_aux(g, s, rs_graph::kAux)) return rc;
    // ---- P2 row lists (on stream 5) beside the G_x offsets (on the step's stream)
    const int64_t nm = g->n_mid, nl = g->n_large;
    auto Lst = [&](int c) { return g->p2rows + p2_list_start(c, nm, nl); };
    if (nm + nl) {
        RS_CUDA_TRY(cudaMemsetAsync(g->p2cnt, 0, kP2Lists * sizeof(int32_t), s));
        p2_split_kernel<<<grid_for(nm + nl, 256, 8), 256, 0, s>>>(g->rows_mid, nm, g->rows_large, nl, g->rec,
                                                                   g->tune.p2_cta_dx, g->p2rows, g->p2cnt);
        RS_LAUNCHED(g, s, "p2_split");
    }
    const int64_t gx_tiles = (n + kGxTile - 1) / kGxTile;
    gx_offsets_kernel<<<(unsigned)gx_tiles, kGxThreads, 0, s>>>(g->rec, n, g->xoff, g->wq + kWqGxStatus,
                                                              g->wq + kWqGxTicket, err, g->gx_spin,
                                                              g->gx_withhold);
    RS_LAUNCHED(g, s, "gx_offsets");
    const Strict SX{g->col, g->strict ? g->sx : nullptr};
    if (g->strict) {
        RS_CUDA_TRY(cudaMemsetAsync(g->sx, 0, 2 * g->nnz * sizeof(unsigned long long), s));
        strict_pairs_kernel<<<grid_for(n * 32, NT, cps), NT, 0, s>>>(n, g->off, g->col, g->lab, g->rec, g->sx);
        RS_LAUNCHED(g, s, "strict_pairs");
    }
    // ---- P2: with per-class streams, the many-short-rows kernels on the low-priority
    //      streams 0 and 1, the rows with long chains on the others.  The hub
    //      chain (three dependent kernels, the longest of the phase on hub-skewed graphs)
    //      is issued first, so that its blocks are dispatched ahead of the other classes'
    if (rmode != 2)
        if (int rc = fork_aux(g, s)) return rc;
    if (g->n_hubs) {
        hub_p2_insert_kernel<NT><<<grid_for(g->n_hub_items, 1, 8), NT, 0, AX(3)>>>(
            g->off, g->col, g->hubs, g->hub_items, g->hub_item_chunk, g->n_hub_items, g->tune.hub_chunk, g->rec,
            g->hkey, g->hq,
            g->hitem_out, g->hitem_in, g->hslot, err);
        RS_LAUNCHED(g, AX(3), "hub_p2_insert");
        hub_p2_counts_kernel<NT><<<(unsigned)((g->n_hubs + NT - 1) / NT), NT, 0, AX(3)>>>(
            g->hubs, g->n_hubs, g->hitem_out, g->hitem_in, g->xout, g->xin);
        RS_LAUNCHED(g, AX(3), "hub_p2_counts");
        hub_p2_emit_kernel<NT><<<grid_for(g->n_hub_items, 1, 8), NT, 0, AX(3)>>>(
            g->off, g->col, g->hubs, g->hub_items, g->hub_item_chunk, g->n_hub_items, g->tune.hub_chunk, g->rec,
            g->hslot,
            g->hq, g->hsig, g->hitem_out, g->hitem_in, g->acc, g->xoff, g->xcol, g->xS, g->xsk, err, SX);
        RS_LAUNCHED(g, AX(3), "hub_p2_emit");
    }
    if (g->n_small) {
        p2_small_kernel<32><<<grid_for(g->n_small, NT, cps), NT, 0, AX(0)>>>(
            g->off, g->rows_small, g->n_small, nullptr, g->LG, g->rec, g->rsum, g->cl_col, g->cl_lab, g->acc,
            g->xoff, g->xcol, g->xS, g->xsk, g->xout, g->xin, SX);
        RS_LAUNCHED(g, AX(0), "p2_small");
    }
    if (g->tune.p3_mirror) {                         // the mirror's tile table, beside P2
        if (!g->xR || !g->xtile) return fail(RS_EINVAL, "rs_score: p3_mirror is set but its buffers are missing");
        mirror_tiles_kernel<<<grid_for(n, NT, cps), NT, 0, AX(0)>>>(n, g->xoff, g->xtile);
        RS_LAUNCHED(g, AX(0), "mirror_tiles");
    }
    const size_t smem256 = (size_t)kMidWarps * 256 * kMidSlotBytes, smem512 = (size_t)kMidWarps * 512 * kMidSlotBytes;
    if (nm + nl) {
        // the mid and large rows with at most 32 cross neighbours, in the tile kernel
        p2_small_kernel<kNarrowRows><<<grid_for((nm + nl) * (32 / kNarrowRows), NT, cps), NT, 0, AX(1)>>>(
            g->off, Lst(0), 0, g->p2cnt + 0, g->LG, g->rec, g->rsum, g->cl_col, g->cl_lab, g->acc, g->xoff,
            g->xcol, g->xS, g->xsk, g->xout, g->xin, SX);
        RS_LAUNCHED(g, AX(1), "p2_narrow");
    }
    if (g->n_mid) {
        p2_mid_kernel<<<grid_for(g->n_mid * 32, NT, 4), NT, smem256, AX(5)>>>(
            g->off, Lst(1), g->p2cnt + 1, B, 1 << 30, 256, g->LG, g->rec, g->rsum, g->cl_col, g->cl_lab, g->acc,
            g->xoff, g->xcol, g->xS, g->xsk, g->xout, g->xin, err, SX, g->wq + 2);
        RS_LAUNCHED(g, AX(5), "p2_mid");
        // few rows, each a long single-warp chain: on the lightly loaded stream
        p2_mid_kernel<<<grid_for(g->n_mid * 32, NT, 2), NT, smem512, AX(2)>>>(
            g->off, Lst(5), g->p2cnt + 5, B, 1 << 30, 512, g->LG, g->rec, g->rsum, g->cl_col, g->cl_lab, g->acc,
            g->xoff, g->xcol, g->xS, g->xsk, g->xout, g->xin, err, SX, g->wq + 3);
        RS_LAUNCHED(g, AX(2), "p2_mid_wide");
    }
    if (g->n_large) {
        // large rows whose cross list fits a per-warp table go warp-per-row too
        p2_mid_kernel<<<grid_for(g->n_large * 32, NT, 4), NT, smem256, AX(2)>>>(
            g->off, Lst(3), g->p2cnt + 3, B, g->tune.p2_cta_dx, 256, g->LG, g->rec, g->rsum, g->cl_col,
            g->cl_lab, g->acc, g->xoff, g->xcol, g->xS, g->xsk, g->xout, g->xin, err, SX, g->wq + 4);
        RS_LAUNCHED(g, AX(2), "p2_large_warp");
        // (with hubs, stream 3 carries the hub chain: these rows go beside p2_mid instead)
        cudaStream_t sw = g->n_hubs || rmode == 1 ? AX(5) : AX(3);
        p2_mid_kernel<<<grid_for(g->n_large * 32, NT, 2), NT, smem512, sw>>>(
            g->off, Lst(6), g->p2cnt + 6, B, g->tune.p2_cta_dx, 512, g->LG, g->rec, g->rsum, g->cl_col,
            g->cl_lab, g->acc, g->xoff, g->xcol, g->xS, g->xsk, g->xout, g->xin, err, SX, g->wq + 5);
        RS_LAUNCHED(g, sw, "p2_large_warp_wide");
        switch (g->tune.p2_cta_threads) {
        case 256: launch_p2_large<256>(g, B, err, p2_smem, AX(4)); break;
        case 512: launch_p2_large<512>(g, B, err, p2_smem, AX(4)); break;
        default: launch_p2_large<1024>(g, B, err, p2_smem, AX(4)); break;
        }
        RS_LAUNCHED(g, AX(4), "p2_large");
    }
    if (rmode != 2)
        if (int rc = join_aux(g, s, rs_graph::kAux)) return rc;
    // ---- P3: reverse values (mirror mode), then triangles
    if (g->tune.p3_mirror) {
        gx_mirror_kernel<<<grid_for(g->nnz, kMirTile, cps), NT, 0, s>>>(n, g->xoff, g->xcol, g->xS, g->xout,
                                                                       g->xin, g->xtile, g->xR, g->xsk, err);
        RS_LAUNCHED(g, s, "gx_mirror");
    }
    const Rev R{g->tune.p3_mirror ? g->xR : nullptr, g->xoff, g->xcol, g->xS, g->xin, err};
    unsigned long long *next_group = g->wq + 7;
    unsigned long long *hvl = g->wq + wq_hv_word(n);
    const int64_t hvcap = hv_cap(g->nnz);
    if (g->perm)                                     // a graph numbered by community: scrambled groups
        p3_list_kernel<true><<<grid_for(n, NT, cps), NT, 0, s>>>(n, g->xoff, g->xcol, g->xsk, g->xS, R, g->xout,
                                                                  g->rec, g->acc, next_group, p3_stride(n), hvl,
                                                                  hvcap, g->wq + kWqHvCount);
    else
        p3_list_kernel<false><<<grid_for(n, NT, cps), NT, 0, s>>>(n, g->xoff, g->xcol, g->xsk, g->xS, R, g->xout,
                                                                   g->rec, g->acc, next_group, 1, hvl, hvcap,
                                                                   g->wq + kWqHvCount);
    RS_LAUNCHED(g, s, "p3_list");
    p3_heavy_kernel<<<grid_for(hvcap, 1, 3), NT, sizeof(P3Heavy), s>>>(n, g->xoff, g->xcol, g->xS, R, g->xout,
                                                                       g->acc, hvl, hvcap, g->wq + kWqHvCount,
                                                                       g->wq + kWqHvNext);
    RS_LAUNCHED(g, s, "p3_heavy");
    // ---- finalize
    if (g->gid) {
        graph_scale_kernel<<<(g->n_graphs + 255) / 256, 256, 0, s>>>(g->wmax_bits, g->n_graphs, g->winv);
        RS_LAUNCHED(g, s, "graph_scale");
    }
    finalize_kernel<<<grid_for(n, NT, cps), NT, 0, s>>>(n, g->off, g->acc, g->gid, g->winv, g->wmax_bits, g->RD,
                                                         g->perm, scores);
    RS_LAUNCHED(g, s, "finalize");
    return 0;
}
