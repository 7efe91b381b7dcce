// rs_topk.cu -- top-K nodes by (score descending, node id ascending)
// (Alg. 1 Step 4).
//
// Each node is a unique 96-bit key (bits(score) << 32 | ~id): for scores >= 0
// the IEEE bit pattern orders like the value, and ~id makes smaller ids rank
// higher among equal scores.  One cooperative launch (one 1024-thread CTA per
// SM, grid-wide barriers from cooperative groups) runs a most-significant-digit
// radix select with 12-bit digits:
//   per level (three grid-wide barriers): privatised shared-memory histograms
//   of the digit over the current candidates, merged into a global histogram;
//   CTA 0 finds the bucket that holds the K-th key; keys of higher buckets are
//   final ("sure"), keys of that bucket stay candidates, both appended with one
//   atomic per warp, while the global histogram is cleared for the next level.
// As soon as the sure keys and the candidates fit a small shared-memory sort
// (about 2K keys), CTA 0 sorts them (bitonic) and writes the first K.
#include <algorithm>
#include <cooperative_groups.h>

#include "rs.h"
#include "rs_internal.cuh"

namespace cg = cooperative_groups;
using namespace rs;

namespace {

constexpr int kTkThreads = 1024;
constexpr int kBits = 12;
constexpr int kBins = 1 << kBits;
constexpr int kLevels = 96 / kBits;
constexpr int kSortMax = 16384;   // largest K, and the size of the final sort
constexpr size_t kTkSmem = (size_t)kSortMax * (8 + 4);

enum { C_NEED = 0, C_SURE = 1, C_SEL = 2, C_NEXT = 3 /* and 4: candidate counters of even / odd levels */ };

// keys left when the selection stops and sorts: a bitonic sort costs log^2 of its
// size in barriers, so another radix level is cheaper than sorting much more than K
__host__ __device__ __forceinline__ int sort_target(int k) {
    int p = 2048;
    while (p < 2 * k && p < kSortMax) p <<= 1;
    return p;
}

// digit `level` (0 = most significant) of the 96-bit key (key64 : ~id)
__device__ __forceinline__ uint32_t digit_of(unsigned long long key, uint32_t nid, int level) {
    int hi = 95 - kBits * level;                 // top bit of the digit
    int lo = hi - kBits + 1;
    if (lo >= 32) return (uint32_t)(key >> (lo - 32)) & (kBins - 1);
    if (hi < 32) return (nid >> lo) & (kBins - 1);
    // straddles the two words: bits [hi-32 .. 0] of key, then bits [31 .. lo] of nid
    uint32_t top = (uint32_t)(key & ((1ull << (hi - 31)) - 1));
    return ((top << (32 - lo)) | (nid >> lo)) & (kBins - 1);
}

struct TkArgs {
    const double *scores;
    int64_t n;
    int32_t k;
    int32_t *ids_out;
    double *scores_out;
    uint32_t *hist;                 // kBins
    int *ctrl;
    unsigned long long *key[2];     // candidate buffers (n each)
    uint32_t *nid[2];
    unsigned long long *skey;       // sure keys (kSortMax)
    uint32_t *snid;
};

__device__ __forceinline__ void load_item(const TkArgs &A, int level, int src, int64_t i,
                                          unsigned long long &key, uint32_t &nid) {
    if (level == 0) {
        key = (unsigned long long)__double_as_longlong(A.scores[i]);
        nid = ~(uint32_t)i;
    } else {
        key = A.key[src][i];
        nid = A.nid[src][i];
    }
}

// descending bitonic sort of (key, nid) pairs in shared memory, P a power of two;
// the pair of each compare-exchange comes from shifts and masks (st is a power of two)
__device__ void block_sort_desc(unsigned long long *key, uint32_t *nid, int P) {
    for (int size = 2; size <= P; size <<= 1)
        for (int st = size >> 1; st; st >>= 1) {
            const int lst = __ffs(st) - 1;
            const bool flip = st == (size >> 1);
            for (int i = threadIdx.x; i < P / 2; i += blockDim.x) {
                int base = (i >> lst) << (lst + 1), o = i & (st - 1);
                int lo = base + o;
                int hi = flip ? base + 2 * st - 1 - o : lo + st;
                unsigned long long kl = key[lo], kh = key[hi];
                uint32_t nl = nid[lo], nh = nid[hi];
                if (kl < kh || (kl == kh && nl < nh)) {
                    key[lo] = kh; key[hi] = kl;
                    nid[lo] = nh; nid[hi] = nl;
                }
            }
            __syncthreads();
        }
}

// append the flagged items of a warp to buf at a position drawn with one atomic
// per warp (every lane of the warp calls; order inside the buffer is free)
__device__ __forceinline__ void warp_append(bool flag, unsigned long long key, uint32_t nid, int *counter,
                                            unsigned long long *kbuf, uint32_t *ibuf) {
    unsigned m = __ballot_sync(0xFFFFFFFFu, flag);
    if (!m) return;
    int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(counter, __popc(m));
    base = __shfl_sync(0xFFFFFFFFu, base, leader);
    if (flag) {
        int p = base + __popc(m & ((1u << lane) - 1u));
        kbuf[p] = key; ibuf[p] = nid;
    }
}

__global__ void __launch_bounds__(kTkThreads) tk_select_kernel(TkArgs A) {
    cg::grid_group grid = cg::this_grid();
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t *sh_hist = (uint32_t *)smem;                      // kBins (levels)
    __shared__ uint32_t part[32];
    __shared__ int sh_sel;
    __shared__ int64_t sh_above;
    int tid = threadIdx.x;
    int64_t gtid = (int64_t)blockIdx.x * blockDim.x + tid;
    int64_t gsize = (int64_t)gridDim.x * blockDim.x;
    // every warp walks the same trip count, so warp-wide ballots see whole warps
    int64_t wbase = gtid & ~31ll;
    int *ctrl = A.ctrl;
    if (gtid == 0) {
        ctrl[C_SURE] = 0; ctrl[C_NEXT] = 0; ctrl[C_NEXT + 1] = 0;
    }
    for (int64_t b = gtid; b < kBins; b += gsize) A.hist[b] = 0;
    // the state every thread derives alike: candidates m in buffer src, rank need among them
    int src = 0;
    int64_t m = A.n;
    int64_t need = A.k;
    bool done = A.n <= sort_target(A.k);                        // everything fits the final sort
    grid.sync();
    int level = 0;
    for (; level < kLevels && !done; ++level) {
        // histogram of this level's digit (the global one was cleared before)
        for (int b = tid; b < kBins; b += blockDim.x) sh_hist[b] = 0;
        __syncthreads();
        // lanes with the same digit add once (the top digits of real scores crowd a
        // few bins, where per-lane shared atomics would serialise)
        for (int64_t i0 = wbase; i0 < m; i0 += gsize) {
            int64_t i = i0 + (tid & 31);
            bool in = i < m;
            uint32_t dg = kBins;                                // no bin: lanes past the end
            if (in) {
                unsigned long long key; uint32_t nid;
                load_item(A, level, src, i, key, nid);
                dg = digit_of(key, nid, level);
            }
            unsigned same = __match_any_sync(0xFFFFFFFFu, dg);
            if (in && (tid & 31) == __ffs(same) - 1) atomicAdd(&sh_hist[dg], (uint32_t)__popc(same));
        }
        __syncthreads();
        for (int b = tid; b < kBins; b += blockDim.x)
            if (sh_hist[b]) atomicAdd(&A.hist[b], sh_hist[b]);
        grid.sync();
        // CTA 0: the bucket holding the need-th largest key
        if (blockIdx.x == 0) {
            constexpr int per = kBins / kTkThreads;             // 4 bins per thread, from the top
            int top = kBins - per * tid;
            uint32_t sacc = 0;
            for (int j = 1; j <= per; ++j) sacc += A.hist[top - j];
            // inclusive scan over the threads: within warps by shuffles, then over the warp sums
            const int lane = tid & 31, wid = tid >> 5;
            uint32_t incl = sacc;
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                if (lane >= o) incl += v;
            }
            if (lane == 31) part[wid] = incl;
            __syncthreads();
            if (wid == 0) {
                uint32_t w = lane < kTkThreads / 32 ? part[lane] : 0;
                for (int o = 1; o < 32; o <<= 1) {
                    uint32_t v = __shfl_up_sync(0xFFFFFFFFu, w, o);
                    if (lane >= o) w += v;
                }
                part[lane] = w;                                 // inclusive sums of the warp sums
            }
            __syncthreads();
            const uint32_t mine = incl + (wid ? part[wid - 1] : 0u);
            int64_t before = (int64_t)mine - sacc;
            if (before < need && need <= (int64_t)mine) {
                int64_t acc = before;
                for (int j = 1; j <= per; ++j) {
                    int b = top - j;
                    if (acc + A.hist[b] >= need) { sh_sel = b; sh_above = acc; break; }
                    acc += A.hist[b];
                }
            }
            __syncthreads();
            if (tid == 0) {
                ctrl[C_SEL] = sh_sel;
                ctrl[C_NEED] = (int)(need - sh_above);
            }
        }
        grid.sync();
        // compact: higher buckets are sure, the selected bucket stays; the global
        // histogram is cleared for the next level, and the candidate counter of
        // the next level (last read before this level's first barrier) reset
        const uint32_t sel = (uint32_t)ctrl[C_SEL];
        need = ctrl[C_NEED];
        const int dst = src ^ 1;
        int *next = &ctrl[C_NEXT + (level & 1)];
        for (int64_t b = gtid; b < kBins; b += gsize) A.hist[b] = 0;
        if (gtid == 0) ctrl[C_NEXT + ((level + 1) & 1)] = 0;
        for (int64_t i0 = wbase; i0 < m; i0 += gsize) {
            int64_t i = i0 + (tid & 31);
            unsigned long long key = 0; uint32_t nid = 0, dg = 0;
            bool in = i < m;
            if (in) {
                load_item(A, level, src, i, key, nid);
                dg = digit_of(key, nid, level);
            }
            warp_append(in && dg > sel, key, nid, &ctrl[C_SURE], A.skey, A.snid);
            warp_append(in && dg == sel, key, nid, next, A.key[dst], A.nid[dst]);
        }
        grid.sync();
        m = *(volatile int *)next;
        src = dst;
        done = m <= need || *(volatile int *)&ctrl[C_SURE] + m <= sort_target(A.k);
    }
    // CTA 0: sort the sure keys and the candidates left, write the first K
    if (blockIdx.x != 0) return;
    unsigned long long *key = (unsigned long long *)smem;
    uint32_t *nid = (uint32_t *)(key + sort_target(A.k));      // the launch sized the sort for k
    bool from_scores = level == 0;                              // nothing was compacted: n fits the sort
    int ns = ctrl[C_SURE];
    int nc = (int)m;
    int total = ns + nc;
    int P = 1;
    while (P < total) P <<= 1;
    for (int i = tid; i < P; i += blockDim.x) {
        if (i < ns) { key[i] = A.skey[i]; nid[i] = A.snid[i]; }
        else if (i < total) {
            int64_t j = i - ns;
            if (from_scores) { key[i] = (unsigned long long)__double_as_longlong(A.scores[j]); nid[i] = ~(uint32_t)j; }
            else { key[i] = A.key[src][j]; nid[i] = A.nid[src][j]; }
        } else { key[i] = 0; nid[i] = 0; }                     // padding sorts last
    }
    __syncthreads();
    block_sort_desc(key, nid, P);
    for (int i = tid; i < A.k; i += blockDim.x) {
        A.ids_out[i] = (int32_t)~nid[i];
        if (A.scores_out) A.scores_out[i] = __longlong_as_double((long long)key[i]);
    }
}

}  // namespace

static int ensure_topk_workspace(rs_graph *g, int64_t n) {
    if (g->tk_cap >= n && g->tk_hist) return 0;
    void *old[] = {g->tk_hist, g->tk_ctrl, g->tk_keys, g->tk_ids};
    RS_CUDA_TRY(pool_free_many(old, 4));
    g->tk_hist = nullptr; g->tk_ctrl = nullptr; g->tk_keys = nullptr; g->tk_ids = nullptr;
    int64_t cap = n > 1 ? n : 1;
    RS_CUDA_TRY(pool_malloc((void **)&g->tk_hist, kBins * sizeof(uint32_t)));
    RS_CUDA_TRY(pool_malloc((void **)&g->tk_ctrl, 8 * sizeof(int)));
    RS_CUDA_TRY(pool_malloc((void **)&g->tk_keys, (2 * cap + kSortMax) * sizeof(unsigned long long)));
    RS_CUDA_TRY(pool_malloc((void **)&g->tk_ids, (2 * cap + kSortMax) * sizeof(uint32_t)));
    g->tk_cap = cap;
    g->version++;                     // captured steps hold the old buffers
    return 0;
}

static int tk_grid = 0;   // one CTA per SM (or what fits), found once per process

// workspace for n scores and the selection kernel's launch shape
int rs::topk_prepare(rs_graph *g, int64_t n) {
    if (int rc = ensure_topk_workspace(g, n)) return rc;
    if (!tk_grid) {
        RS_CUDA_TRY(cudaFuncSetAttribute(tk_select_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTkSmem));
        int dev = 0, sms = 0, per_sm = 0;
        RS_CUDA_TRY(cudaGetDevice(&dev));
        RS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        RS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tk_select_kernel, kTkThreads, kTkSmem));
        if (per_sm < 1) return fail(RS_ECUDA, "rs_topk: selection kernel does not fit an SM");
        tk_grid = sms * per_sm;
    }
    return 0;
}

int rs::topk_scores(rs_graph *g, const double *scores, int64_t n, int32_t k, int32_t *ids, double *out_scores,
                    cudaStream_t s) {
    if (k > kSortMax) return fail(RS_EINVAL, "rs_topk: k above 16384 is not supported");
    if (n > 2147483647LL) return fail(RS_EINVAL, "rs_topk: n too large");
    if (int rc = topk_prepare(g, n)) return rc;
    const int grid = tk_grid;
    int64_t cap = g->tk_cap;
    TkArgs A;
    A.scores = scores; A.n = n; A.k = k; A.ids_out = ids; A.scores_out = out_scores;
    A.hist = g->tk_hist; A.ctrl = g->tk_ctrl;
    unsigned long long *kb = g->tk_keys;
    uint32_t *ib = (uint32_t *)g->tk_ids;
    A.key[0] = kb; A.key[1] = kb + cap; A.skey = kb + 2 * cap;
    A.nid[0] = ib; A.nid[1] = ib + cap; A.snid = ib + 2 * cap;
    prof_begin(g, s);
    void *args[] = {&A};
    // dynamic shared memory: the level histograms, or the final sort of up to sort_target(k)
    // keys, whichever is larger (24 KB for k <= 1024; the attribute allows kTkSmem)
    const size_t smem = std::max((size_t)kBins * sizeof(uint32_t), (size_t)sort_target(k) * (8 + 4));
    RS_CUDA_TRY(cudaLaunchCooperativeKernel((void *)tk_select_kernel, dim3(grid), dim3(kTkThreads), args, smem, s));
    RS_LAUNCHED(g, s, "tk_select");
    return 0;
}
