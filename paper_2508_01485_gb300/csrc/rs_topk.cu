// rs_topk.cu -- top-K nodes by (score descending, node id ascending)
// (Alg. 1 Step 4).
//
// Each node is a unique 96-bit key (bits(score) << 32 | ~id): for scores >= 0
// the IEEE bit pattern orders like the value, and ~id makes smaller ids rank
// higher among equal scores.  A most-significant-digit radix select with six
// 16-bit digits narrows the candidates: per level, a histogram of the digit
// over the current candidates, one CTA finds the bucket holding the K-th key,
// keys of higher buckets are final ("sure"), keys of that bucket stay
// candidates.  When the candidates left are exactly the ones still needed the
// selection stops; one CTA then sorts the K selected keys (bitonic, shared
// memory) and writes ids and scores.
#include "rs.h"
#include "rs_internal.cuh"

using namespace rs;

namespace {

constexpr int kDigits = 6;
constexpr int kBins = 1 << 16;
constexpr int kSortMax = 16384;   // largest K (shared-memory bitonic sort)

// control words
enum { C_CAND = 0, C_NEED = 1, C_SURE = 2, C_SEL = 3, C_DONE = 4, C_NEXT = 5, C_LEVEL = 6 };

__device__ __forceinline__ uint32_t digit_of(unsigned long long key, int32_t id, int level) {
    uint32_t nid = ~(uint32_t)id;
    switch (level) {
        case 0: return (uint32_t)(key >> 48) & 0xFFFF;
        case 1: return (uint32_t)(key >> 32) & 0xFFFF;
        case 2: return (uint32_t)(key >> 16) & 0xFFFF;
        case 3: return (uint32_t)key & 0xFFFF;
        case 4: return nid >> 16;
        default: return nid & 0xFFFF;
    }
}

__global__ void tk_init_kernel(int *ctrl, int64_t n, int32_t k) {
    ctrl[C_CAND] = (int)n;
    ctrl[C_NEED] = k;
    ctrl[C_SURE] = 0;
    ctrl[C_SEL] = 0;
    ctrl[C_DONE] = 0;
    ctrl[C_NEXT] = 0;
    ctrl[C_LEVEL] = -1;
}

// level 0 reads the scores directly; later levels read the candidate arrays
__global__ void tk_hist_kernel(const double *scores, const unsigned long long *ckey, const int32_t *cid,
                               int level, const int *ctrl, uint32_t *hist) {
    if (ctrl[C_DONE]) return;
    int64_t m = ctrl[C_CAND];
    int lane = threadIdx.x & 31;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < m; base += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = base + threadIdx.x;
        bool act = i < m;
        uint32_t dg = 0;
        if (act) {
            unsigned long long key = level == 0 ? (unsigned long long)__double_as_longlong(scores[i]) : ckey[i];
            int32_t id = level == 0 ? (int32_t)i : cid[i];
            dg = digit_of(key, id, level);
        }
        unsigned am = __ballot_sync(0xFFFFFFFFu, act);
        if (act) {
            unsigned grp = __match_any_sync(am, dg);
            if (lane == __ffs(grp) - 1) atomicAdd(&hist[dg], (uint32_t)__popc(grp));
        }
    }
}

// one CTA of 1024 threads: the bucket holding the need-th largest key
__global__ void __launch_bounds__(1024) tk_select_kernel(const uint32_t *hist, int *ctrl) {
    if (ctrl[C_DONE]) return;
    __shared__ int64_t part[1024];
    __shared__ int64_t above_sh;
    int t = threadIdx.x;
    constexpr int per = kBins / 1024;
    int hi_bin = kBins - per * t;                 // chunk [hi_bin - per, hi_bin), from the top
    int64_t s = 0;
    for (int j = 1; j <= per; ++j) s += hist[hi_bin - j];
    part[t] = s;
    __syncthreads();
    // inclusive scan of chunk totals from the top
    for (int o = 1; o < 1024; o <<= 1) {
        int64_t v = t >= o ? part[t - o] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int64_t need = ctrl[C_NEED];
    int64_t before = t ? part[t - 1] : 0;         // keys in higher chunks
    if (before < need && need <= part[t]) {
        int64_t acc = before;
        for (int j = 1; j <= per; ++j) {
            int b = hi_bin - j;
            if (acc + hist[b] >= need) {
                ctrl[C_SEL] = b;
                above_sh = acc;
                break;
            }
            acc += hist[b];
        }
    }
    __syncthreads();
    if (t == 0) {
        ctrl[C_NEED] = (int)(need - above_sh);
        ctrl[C_NEXT] = 0;
    }
}

__global__ void tk_compact_kernel(const double *scores, const unsigned long long *ckey, const int32_t *cid,
                                  int level, int *ctrl, unsigned long long *nkey, int32_t *nid,
                                  unsigned long long *skey, int32_t *sid) {
    if (ctrl[C_DONE]) return;
    int64_t m = ctrl[C_CAND];
    uint32_t sel = (uint32_t)ctrl[C_SEL];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long key = level == 0 ? (unsigned long long)__double_as_longlong(scores[i]) : ckey[i];
        int32_t id = level == 0 ? (int32_t)i : cid[i];
        uint32_t dg = digit_of(key, id, level);
        if (dg > sel) {
            int p = atomicAdd(&ctrl[C_SURE], 1);
            skey[p] = key; sid[p] = id;
        } else if (dg == sel) {
            int p = atomicAdd(&ctrl[C_NEXT], 1);
            nkey[p] = key; nid[p] = id;
        }
    }
}

__global__ void tk_advance_kernel(int *ctrl, int level) {
    if (ctrl[C_DONE]) return;
    ctrl[C_CAND] = ctrl[C_NEXT];
    if (ctrl[C_CAND] <= ctrl[C_NEED]) {
        ctrl[C_DONE] = 1;
        ctrl[C_LEVEL] = level;     // the candidates left sit in this level's target buffer
    }
}

// sort the K selected keys: sure keys plus the final candidates
__global__ void __launch_bounds__(1024) tk_sort_kernel(const unsigned long long *skey, const int32_t *sid,
                                                       const unsigned long long *key_even, const int32_t *id_even,
                                                       const unsigned long long *key_odd, const int32_t *id_odd,
                                                       const int *ctrl, int32_t k, int32_t *ids_out,
                                                       double *scores_out) {
    extern __shared__ __align__(16) unsigned char smem[];
    // even levels write their candidates to the first buffer, odd levels to the second
    bool odd = ctrl[C_LEVEL] & 1;
    const unsigned long long *ckey = odd ? key_odd : key_even;
    const int32_t *cid = odd ? id_odd : id_even;
    int P = 1;
    while (P < k) P <<= 1;
    unsigned long long *key = (unsigned long long *)smem;
    uint32_t *nid = (uint32_t *)(key + P);
    int ns = ctrl[C_SURE];
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        if (i < ns) { key[i] = skey[i]; nid[i] = ~(uint32_t)sid[i]; }
        else if (i < k) { key[i] = ckey[i - ns]; nid[i] = ~(uint32_t)cid[i - ns]; }
        else { key[i] = 0; nid[i] = 0; }     // padding sorts last (descending order)
    }
    __syncthreads();
    // bitonic sort, descending by (key, ~id)
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
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        ids_out[i] = (int32_t)~nid[i];
        if (scores_out) scores_out[i] = __longlong_as_double((long long)key[i]);
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
    // two candidate buffers plus the sure list
    RS_CUDA_TRY(cudaMalloc(&g->tk_keys, (2 * cap + kSortMax) * sizeof(unsigned long long)));
    RS_CUDA_TRY(cudaMalloc(&g->tk_ids, (2 * cap + kSortMax) * sizeof(int32_t)));
    g->tk_cap = cap;
    return 0;
}

int rs::topk_scores(rs_graph *g, const double *scores, int64_t n, int32_t k, int32_t *ids, double *out_scores,
                    cudaStream_t s) {
    if (k > kSortMax) return fail(RS_EINVAL, "rs_topk: k above 16384 is not supported");
    if (int rc = ensure_topk_workspace(g, n)) return rc;
    static bool attr_done = false;
    if (!attr_done) {
        RS_CUDA_TRY(cudaFuncSetAttribute(tk_sort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kSortMax * (8 + 4)));
        attr_done = true;
    }
    int64_t cap = g->tk_cap;
    unsigned long long *ka = g->tk_keys, *kb = g->tk_keys + cap, *ks = g->tk_keys + 2 * cap;
    int32_t *ia = g->tk_ids, *ib = g->tk_ids + cap, *is = g->tk_ids + 2 * cap;
    int *ctrl = g->tk_ctrl;
    tk_init_kernel<<<1, 1, 0, s>>>(ctrl, n, k);
    RS_CUDA_TRY(cudaGetLastError());
    int grid = grid_for(n, 256, 8);
    for (int level = 0; level < kDigits; ++level) {
        RS_CUDA_TRY(cudaMemsetAsync(g->tk_hist, 0, kBins * sizeof(uint32_t), s));
        const unsigned long long *ck = level == 0 ? nullptr : (level % 2 ? ka : kb);
        const int32_t *ci = level == 0 ? nullptr : (level % 2 ? ia : ib);
        unsigned long long *nk = level % 2 ? kb : ka;
        int32_t *ni = level % 2 ? ib : ia;
        tk_hist_kernel<<<grid, 256, 0, s>>>(scores, ck, ci, level, ctrl, g->tk_hist);
        RS_CUDA_TRY(cudaGetLastError());
        tk_select_kernel<<<1, 1024, 0, s>>>(g->tk_hist, ctrl);
        RS_CUDA_TRY(cudaGetLastError());
        tk_compact_kernel<<<grid, 256, 0, s>>>(scores, ck, ci, level, ctrl, nk, ni, ks, is);
        RS_CUDA_TRY(cudaGetLastError());
        tk_advance_kernel<<<1, 1, 0, s>>>(ctrl, level);
        RS_CUDA_TRY(cudaGetLastError());
    }
    int P = 1;
    while (P < k) P <<= 1;
    size_t smem = (size_t)P * (8 + 4);
    tk_sort_kernel<<<1, 1024, smem, s>>>(ks, is, ka, ia, kb, ib, ctrl, k, ids, out_scores);
    RS_CUDA_TRY(cudaGetLastError());
    return 0;
}
