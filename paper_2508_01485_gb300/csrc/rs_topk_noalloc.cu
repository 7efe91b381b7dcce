// rs_topk_noalloc.cu -- top-K by (score descending, node id ascending) over a
// caller's device array of scores, with no device allocation at all.
//
// For callers that cannot allocate device memory: code whose device memory is
// owned by another allocator (a framework's caching allocator, a fixed memory
// budget), and latency-critical loops that cannot afford cudaMalloc's implicit
// device synchronisation or its possible failure in the middle of a request.
//
// All scratch lives in one file-scope static __device__ array of kNoAllocBytes
// bytes, which every GPU that loads the library holds until the process exits.
// The selection is the same 96-bit key radix select as rs_topk (12-bit digits),
// but it keeps no candidate copies: every level re-reads the scores and keeps
// only keys whose leading digits equal the prefix selected so far, so the
// scratch does not grow with n.  Once the keys above the prefix and the keys on
// it fit kNoAllocSort entries, one pass gathers them and CTA 0 sorts them.
//
// The scratch is shared by every call: the kernel re-initialises the parts
// that must start at zero, and calls whose work overlaps on the GPU (on
// different streams, or from different host threads) race on it.
#include <cooperative_groups.h>

#include <mutex>

#include "rs.h"
#include "rs_internal.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int kNaThreads = 1024;
constexpr int kNaBits = 12;
constexpr int kNaBins = 1 << kNaBits;
constexpr int kNaLevels = 96 / kNaBits;
constexpr int kNoAllocSort = 16384;                 // largest K; size of the final sort
constexpr size_t kNaSmem = (size_t)kNoAllocSort * (8 + 4);

// scratch layout (bytes): histogram | control words | keys | ~ids
constexpr size_t kOffHist = 0;
constexpr size_t kOffCtrl = kOffHist + kNaBins * sizeof(uint32_t);
constexpr size_t kOffKey = kOffCtrl + 256;
constexpr size_t kOffNid = kOffKey + kNoAllocSort * sizeof(unsigned long long);
constexpr size_t kNoAllocBytes = kOffNid + kNoAllocSort * sizeof(uint32_t);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

enum { N_NEED = 0, N_ABOVE = 1, N_CAND = 2, N_DONE = 3, N_LEVEL = 4, N_SEL = 5, N_OUT = 6, N_PHI = 8, N_PLO = 10 };

__device__ __forceinline__ uint32_t na_digit(unsigned long long key, uint32_t nid, int level) {
    int hi = 95 - kNaBits * level;
    int lo = hi - kNaBits + 1;
    if (lo >= 32) return (uint32_t)(key >> (lo - 32)) & (kNaBins - 1);
    if (hi < 32) return (nid >> lo) & (kNaBins - 1);
    uint32_t top = (uint32_t)(key & ((1ull << (hi - 31)) - 1));
    return ((top << (32 - lo)) | (nid >> lo)) & (kNaBins - 1);
}

// the leading `bits` bits of the 96-bit key (key : nid), others cleared
__device__ __forceinline__ void na_prefix(unsigned long long key, uint32_t nid, int bits,
                                          unsigned long long &ph, uint32_t &pl) {
    if (bits >= 64) {
        ph = key;
        int lb = bits - 64;
        pl = lb == 0 ? 0u : (lb >= 32 ? nid : (nid & ~((1u << (32 - lb)) - 1u)));
    } else {
        ph = bits == 0 ? 0ull : (key & ~((1ull << (64 - bits)) - 1ull));
        pl = 0u;
    }
}
// -1, 0, 1: leading `bits` bits of the key below, equal to, above the prefix (ph, pl)
__device__ __forceinline__ int na_cmp(unsigned long long key, uint32_t nid, int bits, unsigned long long ph,
                                      uint32_t pl) {
    unsigned long long kh;
    uint32_t kl;
    na_prefix(key, nid, bits, kh, kl);
    if (kh != ph) return kh < ph ? -1 : 1;
    if (kl != pl) return kl < pl ? -1 : 1;
    return 0;
}

struct NaArgs {
    const double *scores;
    int64_t n;
    int32_t k;
    int32_t *ids_out;
    double *scores_out;
    unsigned char *scratch;
};

__global__ void __launch_bounds__(kNaThreads) na_topk_kernel(NaArgs A) {
    cg::grid_group grid = cg::this_grid();
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t *sh_hist = (uint32_t *)smem;
    __shared__ uint32_t part[kNaThreads];
    __shared__ int sh_sel;
    __shared__ int64_t sh_above;
    uint32_t *hist = (uint32_t *)(A.scratch + kOffHist);
    long long *ctrl = (long long *)(A.scratch + kOffCtrl);
    unsigned long long *gkey = (unsigned long long *)(A.scratch + kOffKey);
    uint32_t *gnid = (uint32_t *)(A.scratch + kOffNid);
    int tid = threadIdx.x;
    int64_t gtid = (int64_t)blockIdx.x * blockDim.x + tid;
    int64_t gsize = (int64_t)gridDim.x * blockDim.x;
    if (gtid == 0) {
        ctrl[N_NEED] = A.k;
        ctrl[N_ABOVE] = 0;
        ctrl[N_CAND] = A.n;
        ctrl[N_DONE] = A.n <= kNoAllocSort ? 1 : 0;
        ctrl[N_LEVEL] = 0;
        ctrl[N_OUT] = 0;
        ctrl[N_PHI] = 0;
        ctrl[N_PLO] = 0;
    }
    grid.sync();
    for (int level = 0; level < kNaLevels; ++level) {
        if (*(volatile long long *)&ctrl[N_DONE]) break;
        int bits = kNaBits * level;
        unsigned long long ph = (unsigned long long)ctrl[N_PHI];
        uint32_t pl = (uint32_t)ctrl[N_PLO];
        for (int b = tid; b < kNaBins; b += blockDim.x) sh_hist[b] = 0;
        for (int64_t b = gtid; b < kNaBins; b += gsize) hist[b] = 0;
        grid.sync();
        for (int64_t i = gtid; i < A.n; i += gsize) {
            unsigned long long key = (unsigned long long)__double_as_longlong(A.scores[i]);
            uint32_t nid = ~(uint32_t)i;
            if (na_cmp(key, nid, bits, ph, pl) == 0) atomicAdd(&sh_hist[na_digit(key, nid, level)], 1u);
        }
        __syncthreads();
        for (int b = tid; b < kNaBins; b += blockDim.x)
            if (sh_hist[b]) atomicAdd(&hist[b], sh_hist[b]);
        grid.sync();
        if (blockIdx.x == 0) {
            constexpr int per = kNaBins / kNaThreads;
            int top = kNaBins - per * tid;
            uint32_t s = 0;
            for (int j = 1; j <= per; ++j) s += hist[top - j];
            part[tid] = s;
            __syncthreads();
            for (int o = 1; o < kNaThreads; o <<= 1) {
                uint32_t v = tid >= o ? part[tid - o] : 0;
                __syncthreads();
                part[tid] += v;
                __syncthreads();
            }
            int64_t need = ctrl[N_NEED];
            int64_t before = tid ? part[tid - 1] : 0;
            if (before < need && need <= (int64_t)part[tid]) {
                int64_t acc = before;
                for (int j = 1; j <= per; ++j) {
                    int b = top - j;
                    if (acc + hist[b] >= need) { sh_sel = b; sh_above = acc; break; }
                    acc += hist[b];
                }
            }
            __syncthreads();
            if (tid == 0) {
                int sel = sh_sel;
                // append the selected digit to the prefix
                int lo = 95 - kNaBits * level - kNaBits + 1;       // lowest bit of the digit
                unsigned long long nph = ph;
                uint32_t npl = pl;
                for (int bb = 0; bb < kNaBits; ++bb) {
                    if (!((sel >> bb) & 1)) continue;
                    int pos = lo + bb;
                    if (pos >= 32) nph |= 1ull << (pos - 32);
                    else npl |= 1u << pos;
                }
                ctrl[N_PHI] = (long long)nph;
                ctrl[N_PLO] = (long long)npl;
                ctrl[N_ABOVE] += sh_above;
                ctrl[N_NEED] = need - sh_above;
                ctrl[N_CAND] = hist[sel];
                ctrl[N_LEVEL] = level + 1;
                if (ctrl[N_CAND] <= ctrl[N_NEED] || ctrl[N_ABOVE] + ctrl[N_CAND] <= kNoAllocSort) ctrl[N_DONE] = 1;
            }
        }
        grid.sync();
    }
    // gather every key at or above the selected prefix (at most kNoAllocSort of them)
    int bits = kNaBits * (int)ctrl[N_LEVEL];
    unsigned long long ph = (unsigned long long)ctrl[N_PHI];
    uint32_t pl = (uint32_t)ctrl[N_PLO];
    for (int64_t i = gtid; i < A.n; i += gsize) {
        unsigned long long key = (unsigned long long)__double_as_longlong(A.scores[i]);
        uint32_t nid = ~(uint32_t)i;
        if (na_cmp(key, nid, bits, ph, pl) >= 0) {
            unsigned long long p = atomicAdd((unsigned long long *)&ctrl[N_OUT], 1ull);
            if (p < (unsigned long long)kNoAllocSort) { gkey[p] = key; gnid[p] = nid; }
        }
    }
    grid.sync();
    if (blockIdx.x != 0) return;
    int total = (int)min((long long)kNoAllocSort, ctrl[N_OUT]);
    unsigned long long *key = (unsigned long long *)smem;
    uint32_t *nid = (uint32_t *)(key + kNoAllocSort);
    int P = 1;
    while (P < total) P <<= 1;
    for (int i = tid; i < P; i += blockDim.x) {
        if (i < total) { key[i] = gkey[i]; nid[i] = gnid[i]; }
        else { key[i] = 0; nid[i] = 0; }
    }
    __syncthreads();
    for (int size = 2; size <= P; size <<= 1)
        for (int st = size >> 1; st; st >>= 1) {
            for (int i = tid; i < P / 2; i += blockDim.x) {
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
    for (int i = tid; i < A.k; i += blockDim.x) {
        A.ids_out[i] = (int32_t)~nid[i];
        if (A.scores_out) A.scores_out[i] = __longlong_as_double((long long)key[i]);
    }
}

// per-device set-up: the scratch array's device address and the launch shape
constexpr int kMaxDevices = 64;
struct NaDevice {
    std::once_flag once;
    cudaError_t status = cudaSuccess;
    unsigned char *scratch = nullptr;
    int grid = 0;
};
NaDevice g_na_dev[kMaxDevices];

void na_setup(NaDevice &d) {
    void *ptr = nullptr;
    d.status = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (d.status != cudaSuccess) return;
    d.scratch = (unsigned char *)ptr;
    d.status = cudaFuncSetAttribute(na_topk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kNaSmem);
    if (d.status != cudaSuccess) return;
    int dev = 0, sms = 0, per_sm = 0;
    if ((d.status = cudaGetDevice(&dev)) != cudaSuccess) return;
    if ((d.status = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return;
    d.status = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, na_topk_kernel, kNaThreads, kNaSmem);
    if (d.status != cudaSuccess) return;
    d.grid = sms * (per_sm > 0 ? per_sm : 0);
}

}  // namespace

extern "C" rs_status rs_topk_noalloc(const double *scores, int64_t n, int32_t k, int32_t *ids_out,
                                     double *scores_out, void *stream) {
    if (!scores || !ids_out) return (rs_status)rs::fail(RS_EINVAL, "rs_topk_noalloc: NULL argument");
    if (n < 1 || n > 2147483647LL) return (rs_status)rs::fail(RS_EINVAL, "rs_topk_noalloc: n must be in [1, 2^31)");
    if (k < 1 || (int64_t)k > n)
        return (rs_status)rs::fail(RS_EINVAL, "rs_topk_noalloc: k must be in [1, n]");
    if (k > kNoAllocSort)
        return (rs_status)rs::fail(RS_EINVAL, "rs_topk_noalloc: k above 16384 exceeds the static scratch");
    int dev = 0;
    if (cudaError_t e = cudaGetDevice(&dev)) return (rs_status)rs::cuda_fail(e, "rs_topk_noalloc");
    if (dev < 0 || dev >= kMaxDevices) return (rs_status)rs::fail(RS_EINVAL, "rs_topk_noalloc: device index too large");
    NaDevice &d = g_na_dev[dev];
    std::call_once(d.once, na_setup, std::ref(d));
    if (d.status != cudaSuccess) return (rs_status)rs::cuda_fail(d.status, "rs_topk_noalloc set-up");
    if (d.grid < 1) return (rs_status)rs::fail(RS_ECUDA, "rs_topk_noalloc: kernel does not fit an SM");
    NaArgs A{scores, n, k, ids_out, scores_out, d.scratch};
    void *args[] = {&A};
    cudaError_t e = cudaLaunchCooperativeKernel((void *)na_topk_kernel, dim3(d.grid), dim3(kNaThreads), args, kNaSmem,
                                                (cudaStream_t)stream);
    if (e != cudaSuccess) return (rs_status)rs::cuda_fail(e, "rs_topk_noalloc launch");
    return RS_OK;
}
