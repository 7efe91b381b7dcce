// rs_topk.cu -- top-K nodes by (score descending, node id ascending)
// (Alg. 1 Step 4).
//
// Each node is a unique 96-bit key (bits(score) << 32 | ~id): for scores >= 0
// the IEEE bit pattern orders like the value, and ~id makes smaller ids rank
// higher among equal scores.  One cooperative launch (one 1024-thread CTA per
// SM, grid-wide barriers from cooperative groups) runs a most-significant-digit
// radix select with 12-bit digits:
//   per level: privatised shared-memory histograms of the digit over the
//   current candidates, merged into a global histogram; CTA 0 finds the bucket
//   that holds the K-th key; keys of higher buckets are final ("sure"), keys
//   of that bucket stay candidates.
// As soon as the sure keys and the candidates fit one shared-memory sort
// (kSortMax keys), CTA 0 sorts them (bitonic) and writes the first K.
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

enum { C_CAND = 0, C_NEED = 1, C_SURE = 2, C_SEL = 3, C_DONE = 4, C_NEXT = 5, C_SRC = 6 };

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

// descending bitonic sort of (key, nid) pairs in shared memory, P a power of two
__device__ void block_sort_desc(unsigned long long *key, uint32_t *nid, int P) {
    for (int size = 2; size <= P; size <<= 1)
        for (int st = size >> 1; st; st >>= 1) {
            for (int i = threadIdx.x; i < P / 2; i += blockDim.x) {
                int lo, hi;
                if (st == (size >> 1)) {
                    int blk = i / st, o = i % st;
                    lo = blk * size + o;
                    hi = blk * size + size - 1 - o;
                } else {
                    lo = (i / st) * 2 * st + (i % st);
                    hi = lo + st;
                }
                bool less = key[lo] < key[hi] || (key[lo] == key[hi] && nid[lo] < nid[hi]);
                if (less) {
                    unsigned long long tk = key[lo]; key[lo] = key[hi]; key[hi] = tk;
                    uint32_t ti = nid[lo]; nid[lo] = nid[hi]; nid[hi] = ti;
                }
            }
            __syncthreads();
        }
}

__global__ void __launch_bounds__(kTkThreads) tk_select_kernel(TkArgs A) {
    cg::grid_group grid = cg::this_grid();
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t *sh_hist = (uint32_t *)smem;                      // kBins (levels)
    __shared__ uint32_t part[kTkThreads];
    __shared__ int sh_sel;
    __shared__ int64_t sh_above;
    int tid = threadIdx.x;
    int64_t gtid = (int64_t)blockIdx.x * blockDim.x + tid;
    int64_t gsize = (int64_t)gridDim.x * blockDim.x;
    int *ctrl = A.ctrl;
    if (gtid == 0) {
        ctrl[C_CAND] = (int)A.n; ctrl[C_NEED] = A.k; ctrl[C_SURE] = 0; ctrl[C_SEL] = 0;
        ctrl[C_NEXT] = 0; ctrl[C_SRC] = 0;
        ctrl[C_DONE] = A.n <= kSortMax ? 1 : 0;                 // everything fits the final sort
    }
    grid.sync();
    int level = 0;
    for (; level < kLevels; ++level) {
        if (*(volatile int *)&ctrl[C_DONE]) break;
        int src = ctrl[C_SRC];
        int64_t m = ctrl[C_CAND];
        // histogram of this level's digit
        for (int b = tid; b < kBins; b += blockDim.x) sh_hist[b] = 0;
        for (int64_t b = gtid; b < kBins; b += gsize) A.hist[b] = 0;
        grid.sync();
        for (int64_t i = gtid; i < m; i += gsize) {
            unsigned long long key; uint32_t nid;
            load_item(A, level, src, i, key, nid);
            atomicAdd(&sh_hist[digit_of(key, nid, level)], 1u);
        }
        __syncthreads();
        for (int b = tid; b < kBins; b += blockDim.x)
            if (sh_hist[b]) atomicAdd(&A.hist[b], sh_hist[b]);
        grid.sync();
        // CTA 0: the bucket holding the need-th largest key
        if (blockIdx.x == 0) {
            constexpr int per = kBins / kTkThreads;             // 4 bins per thread, from the top
            int top = kBins - per * tid;
            uint32_t s = 0;
            for (int j = 1; j <= per; ++j) s += A.hist[top - j];
            part[tid] = s;
            __syncthreads();
            for (int o = 1; o < kTkThreads; o <<= 1) {
                uint32_t v = tid >= o ? part[tid - o] : 0;
                __syncthreads();
                part[tid] += v;
                __syncthreads();
            }
            int64_t need = ctrl[C_NEED];
            int64_t before = tid ? part[tid - 1] : 0;
            if (before < need && need <= (int64_t)part[tid]) {
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
                ctrl[C_NEXT] = 0;
            }
        }
        grid.sync();
        // compact: higher buckets are sure, the selected bucket stays
        uint32_t sel = (uint32_t)ctrl[C_SEL];
        int dst = src ^ 1;
        for (int64_t i = gtid; i < m; i += gsize) {
            unsigned long long key; uint32_t nid;
            load_item(A, level, src, i, key, nid);
            uint32_t dg = digit_of(key, nid, level);
            if (dg > sel) {
                int p = atomicAdd(&ctrl[C_SURE], 1);
                A.skey[p] = key; A.snid[p] = nid;
            } else if (dg == sel) {
                int p = atomicAdd(&ctrl[C_NEXT], 1);
                A.key[dst][p] = key; A.nid[dst][p] = nid;
            }
        }
        grid.sync();
        if (gtid == 0) {
            ctrl[C_CAND] = ctrl[C_NEXT];
            ctrl[C_SRC] = dst;
            if (ctrl[C_CAND] <= ctrl[C_NEED] || ctrl[C_SURE] + ctrl[C_CAND] <= sort_target(A.k)) ctrl[C_DONE] = 1;
        }
        grid.sync();
    }
    // CTA 0: sort the sure keys and the candidates left, write the first K
    if (blockIdx.x != 0) return;
    unsigned long long *key = (unsigned long long *)smem;
    uint32_t *nid = (uint32_t *)(key + kSortMax);
    bool from_scores = level == 0;                              // nothing was compacted: n <= kSortMax
    int ns = ctrl[C_SURE];
    int nc = ctrl[C_CAND];
    int src = ctrl[C_SRC];
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
    cudaFree(g->tk_hist); cudaFree(g->tk_ctrl); cudaFree(g->tk_keys); cudaFree(g->tk_ids);
    g->tk_hist = nullptr; g->tk_ctrl = nullptr; g->tk_keys = nullptr; g->tk_ids = nullptr;
    int64_t cap = n > 1 ? n : 1;
    RS_CUDA_TRY(cudaMalloc(&g->tk_hist, kBins * sizeof(uint32_t)));
    RS_CUDA_TRY(cudaMalloc(&g->tk_ctrl, 8 * sizeof(int)));
    RS_CUDA_TRY(cudaMalloc(&g->tk_keys, (2 * cap + kSortMax) * sizeof(unsigned long long)));
    RS_CUDA_TRY(cudaMalloc(&g->tk_ids, (2 * cap + kSortMax) * sizeof(uint32_t)));
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
    RS_CUDA_TRY(cudaLaunchCooperativeKernel((void *)tk_select_kernel, dim3(grid), dim3(kTkThreads), args, kTkSmem, s));
    RS_LAUNCHED(g, s, "tk_select");
    return 0;
}
