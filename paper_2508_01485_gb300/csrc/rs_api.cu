// rs_api.cu -- C ABI of librs: graph build / validation / removal / cloning,
// row classification, constant tables, scans and the interaction table.
// Scoring kernels live in rs_score.cu, the top-K ranking in rs_topk.cu.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <mutex>
#include <vector>

#include "rs.h"
#include "rs_internal.cuh"

using namespace rs;

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string t_err;

int rs::fail(int status, const std::string &msg) {
    t_err = msg;
    return status;
}
int rs::cuda_fail(cudaError_t e, const char *where) {
    cudaGetLastError();  // clear a sticky launch error from the per-thread slot
    t_err = std::string("CUDA error: ") + cudaGetErrorString(e) + " (" + where + ")";
    return e == cudaErrorMemoryAllocation ? RS_ENOMEM : RS_ECUDA;
}
extern "C" const char *rs_last_error(void) { return t_err.c_str(); }

static cudaStream_t as_stream(void *s) { return (cudaStream_t)s; }

int rs::grid_for(int64_t items, int per_block, int cap_per_sm) {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    int64_t want = (items + per_block - 1) / per_block;
    int64_t cap = (int64_t)sms * cap_per_sm;
    if (want < 1) want = 1;
    return (int)std::min(want, cap);
}

// ---------------------------------------------------------------------------
// inclusive scan of int64 (tiles of 4096, recursive over tile sums)
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 512, kScanPer = 8, kScanTile = kScanThreads * kScanPer;

__device__ __forceinline__ int64_t block_inclusive_scan(int64_t x, int64_t *warp_tot) {
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int nw = blockDim.x >> 5;
        int64_t t = lane < nw ? warp_tot[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xFFFFFFFFu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) warp_tot[lane] = t;
    }
    __syncthreads();
    if (wid > 0) x += warp_tot[wid - 1];
    return x;
}

__global__ void scan_tile_kernel(int64_t *a, int64_t m, int64_t *tile_sums) {
    __shared__ int64_t wt[32];
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
    int64_t v[kScanPer];
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) {
        v[i] = (base + i < m) ? a[base + i] : 0;
        s += v[i];
        v[i] = s;
    }
    int64_t incl = block_inclusive_scan(s, wt);
    int64_t excl = incl - s;
#pragma unroll
    for (int i = 0; i < kScanPer; ++i)
        if (base + i < m) a[base + i] = v[i] + excl;
    if (threadIdx.x == blockDim.x - 1 && tile_sums) tile_sums[blockIdx.x] = incl;
}

__global__ void scan_add_kernel(int64_t *a, int64_t m, const int64_t *tile_sums) {
    if (blockIdx.x == 0) return;
    int64_t add = tile_sums[blockIdx.x - 1];
    int64_t base = (int64_t)blockIdx.x * kScanTile;
    for (int i = threadIdx.x; i < kScanTile; i += blockDim.x)
        if (base + i < m) a[base + i] += add;
}

int64_t rs::scan_tmp_words(int64_t m) {
    int64_t words = 0;
    while (m > kScanTile) {
        m = (m + kScanTile - 1) / kScanTile;
        words += m + 1;
    }
    return words + 1;
}

int rs::inclusive_scan_i64(int64_t *a, int64_t m, int64_t *tmp, cudaStream_t s, int64_t *launches) {
    if (m <= 0) return 0;
    int64_t tiles = (m + kScanTile - 1) / kScanTile;
    if (tiles > 2147483647LL) return fail(RS_EINVAL, "scan too large");
    scan_tile_kernel<<<(unsigned)tiles, kScanThreads, 0, s>>>(a, m, tiles > 1 ? tmp : nullptr);
    RS_CUDA_TRY(cudaGetLastError());
    if (launches) ++*launches;
    if (tiles > 1) {
        int rc = inclusive_scan_i64(tmp, tiles, tmp + tiles + 1, s, launches);
        if (rc) return rc;
        scan_add_kernel<<<(unsigned)tiles, kScanThreads, 0, s>>>(a, m, tmp);
        RS_CUDA_TRY(cudaGetLastError());
        if (launches) ++*launches;
    }
    return 0;
}

// ---------------------------------------------------------------------------
// launch accounting / per-kernel event timing
// ---------------------------------------------------------------------------
static void prof_record(rs_graph *g, cudaStream_t s, const char *name, bool is_kernel) {
    if (g->prof_used == g->prof_ev.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) { g->prof_on = false; return; }
        g->prof_ev.push_back(e);
        g->prof_name.push_back(nullptr);
        g->prof_is_kernel.push_back(0);
        g->prof_prev.push_back(-1);
        g->prof_stream.push_back(nullptr);
    }
    size_t i = g->prof_used;
    int prev = -1;
    for (size_t j = i; j-- > 0;)
        if (g->prof_stream[j] == s) { prev = (int)j; break; }
    cudaEventRecord(g->prof_ev[i], s);
    g->prof_name[i] = name;
    g->prof_is_kernel[i] = is_kernel ? 1 : 0;
    g->prof_prev[i] = prev;
    g->prof_stream[i] = s;
    g->prof_used++;
}
void rs::prof_begin(rs_graph *g, cudaStream_t s) {
    if (g->prof_on) prof_record(g, s, nullptr, false);
}
void rs::prof_mark(rs_graph *g, cudaStream_t s, const char *name, bool is_kernel) {
    if (is_kernel) g->launches++;
    if (g->prof_on) prof_record(g, s, name, is_kernel);
}

int rs::fork_aux(rs_graph *g, cudaStream_t s) {
    RS_CUDA_TRY(cudaEventRecord(g->ev_fork, s));
    for (int i = 0; i < rs_graph::kAux; ++i) {
        RS_CUDA_TRY(cudaStreamWaitEvent(g->aux[i], g->ev_fork, 0));
        prof_begin(g, g->aux[i]);
    }
    return 0;
}
int rs::join_aux(rs_graph *g, cudaStream_t s, int used) {
    for (int i = 0; i < used; ++i) {
        RS_CUDA_TRY(cudaEventRecord(g->ev_join[i], g->aux[i]));
        RS_CUDA_TRY(cudaStreamWaitEvent(s, g->ev_join[i], 0));
    }
    prof_begin(g, s);
    return 0;
}

extern "C" rs_status rs_profile_enable(rs_graph *g, int enable) {
    if (!g) return (rs_status)fail(RS_EINVAL, "rs_profile_enable: NULL graph");
    g->prof_on = enable != 0;
    g->prof_used = 0;
    return RS_OK;
}

extern "C" rs_status rs_profile_read(rs_graph *g, int32_t *n_out, const char **names, float *ms,
                                     int32_t *is_kernel, int32_t cap) {
    if (!g || !n_out) return (rs_status)fail(RS_EINVAL, "rs_profile_read: NULL argument");
    int32_t n = 0;
    if (g->prof_used) {
        if (cudaError_t e = cudaEventSynchronize(g->prof_ev[g->prof_used - 1]))
            return (rs_status)cuda_fail(e, "rs_profile_read");
    }
    for (size_t i = 1; i < g->prof_used; ++i) {
        if (!g->prof_name[i] || g->prof_prev[i] < 0) continue;   // a segment start: nothing ran before it
        if (n < cap) {
            float t = 0.0f;
            cudaEventElapsedTime(&t, g->prof_ev[g->prof_prev[i]], g->prof_ev[i]);
            if (names) names[n] = g->prof_name[i];
            if (ms) ms[n] = t;
            if (is_kernel) is_kernel[n] = g->prof_is_kernel[i];
        }
        n++;
    }
    *n_out = n;
    return RS_OK;
}

extern "C" rs_status rs_launch_count(const rs_graph *g, int64_t *launches) {
    if (!g || !launches) return (rs_status)fail(RS_EINVAL, "rs_launch_count: NULL argument");
    *launches = g->launches;
    return RS_OK;
}

// ---------------------------------------------------------------------------
// constant tables: LG[f] = round(log2 f * 2^58), RD[d] = 1/(d(d-1))
// log2 by the series ln m = 2 atanh((m-1)/(m+1)) in 64-bit fixed point
// (integer arithmetic only), divided by ln 2 = 2 atanh(1/3).
// ---------------------------------------------------------------------------
__device__ uint64_t frac_div(uint64_t a, uint64_t b) {  // floor(a 2^64 / b), a < b
    uint64_t q = 0, r = a;
    for (int i = 63; i >= 0; --i) {
        bool carry = (r >> 63) != 0;
        r <<= 1;
        if (carry || r >= b) { r -= b; q |= 1ull << i; }
    }
    return q;
}
__device__ uint64_t atanh_fixed(uint64_t z) {  // z < 1/2 in 2^-64 units
    uint64_t z2 = (uint64_t)(((u128)z * z) >> 64);
    uint64_t p = z, s = z;
    for (uint64_t k = 3; k < 200; k += 2) {
        p = (uint64_t)(((u128)p * z2) >> 64);
        uint64_t t = p / k;
        if (!t) break;
        s += t;
    }
    return s;
}
// LG[0] is never used as a logarithm (it only multiplies a zero count); it holds the
// weight convention instead: 1 = Alg. 2's |L| = L_all - 1 for every column
__global__ void init_tables_kernel(uint64_t *LG, double *RD, int32_t dmax, int alg2) {
    int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f > dmax) return;
    uint64_t lg = 0;
    if (f >= 1) {
        int e = 63 - __clzll((long long)f);
        uint64_t p2 = 1ull << e;
        if ((uint64_t)f == p2) {
            lg = (uint64_t)e << kLogFrac;
        } else {
            uint64_t ln2 = atanh_fixed(frac_div(1, 3)) << 1;
            uint64_t lnm = atanh_fixed(frac_div((uint64_t)f - p2, (uint64_t)f + p2)) << 1;
            uint64_t l2m = frac_div(lnm, ln2);                       // log2(f / 2^e) in [0, 1)
            const int drop = 64 - kLogFrac;
            lg = ((uint64_t)e << kLogFrac) + (l2m >> drop) + ((l2m >> (drop - 1)) & 1);
        }
    }
    LG[f] = f == 0 ? (uint64_t)(alg2 ? 1 : 0) : lg;
    RD[f] = f >= 2 ? 1.0 / ((double)f * (double)(f - 1)) : 0.0;
}

// ---------------------------------------------------------------------------
// validation
// ---------------------------------------------------------------------------
enum : int { V_OFF = 1, V_COLRANGE = 2, V_SELF = 4, V_ORDER = 8, V_LABEL = 16 };

__global__ void validate_offsets_kernel(const int64_t *off, int64_t n, int64_t nnz, int *flag) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v > n) return;
    bool bad = false;
    if (v == 0 && off[0] != 0) bad = true;
    if (v == n && off[n] != nnz) bad = true;
    if (v < n && off[v + 1] < off[v]) bad = true;
    if (bad) atomicOr(flag, V_OFF);
}

// Symmetry: with every row strictly ascending (checked in the same pass) the directed
// edges form a set E, and E is symmetric iff it equals its transpose.  A keyed 64-bit
// hash of each entry is summed as h(u, v) - h(v, u) modulo 2^64 over all entries; for a
// symmetric E every term cancels with its reverse's, so the sum is 0.  An asymmetric E
// passes only if the sum vanishes by chance (about 2^-64 for inputs not built against
// the key).  The mixer is the SplitMix64 finaliser (Steele, Lea and Flood, OOPSLA 2014).
__device__ __forceinline__ uint64_t mix64(uint64_t x) {
    x ^= x >> 30;
    x *= 0xbf58476d1ce4e5b9ull;
    x ^= x >> 27;
    x *= 0x94d049bb133111ebull;
    x ^= x >> 31;
    return x;
}
constexpr uint64_t kSymKey = 0x243f6a8885a308d3ull;

// tiles of 32 consecutive rows per warp: the tile's entries are streamed one per
// lane (coalesced), and an entry's row is the last lane whose row starts at or
// before it (binary lifting over the lanes' row starts by shuffles)
__global__ void validate_rows_kernel(const int64_t *off, const int32_t *col, const int32_t *lab,
                                     int64_t n, int32_t k, int *flag, unsigned long long *sym) {
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int bad = 0;
    uint64_t hs = 0;
    for (int64_t r0 = w * 32; r0 < n; r0 += nw * 32) {
        const int64_t v = r0 + lane;
        const bool have = v < n;
        const int64_t start = off[have ? v : n];
        const int64_t tile_end = off[min(r0 + 32, n)];
        if (have && (lab[v] < 0 || lab[v] >= k)) bad |= V_LABEL;
        const int64_t e0 = __shfl_sync(0xFFFFFFFFu, start, 0);
        for (int64_t base = e0; base < tile_end; base += 32) {
            const int64_t e = base + lane;
            int r = 0;
            for (int step = 16; step; step >>= 1) {
                int64_t sb = __shfl_sync(0xFFFFFFFFu, start, r + step);
                if (sb <= e) r += step;
            }
            const int64_t rs = __shfl_sync(0xFFFFFFFFu, start, r);
            if (e < tile_end) {
                int32_t x = col[e];
                const uint32_t u = (uint32_t)(r0 + r);
                if (x < 0 || x >= n) bad |= V_COLRANGE;
                if (x == (int32_t)u) bad |= V_SELF;
                if (e > rs && col[e - 1] >= x) bad |= V_ORDER;
                hs += mix64((((uint64_t)u << 32) | (uint32_t)x) ^ kSymKey) -
                      mix64((((uint64_t)(uint32_t)x << 32) | u) ^ kSymKey);
            }
        }
    }
    bad |= __shfl_xor_sync(0xFFFFFFFFu, bad, 16);
    bad |= __shfl_xor_sync(0xFFFFFFFFu, bad, 8);
    bad |= __shfl_xor_sync(0xFFFFFFFFu, bad, 4);
    bad |= __shfl_xor_sync(0xFFFFFFFFu, bad, 2);
    bad |= __shfl_xor_sync(0xFFFFFFFFu, bad, 1);
    if (lane == 0 && bad) atomicOr(flag, bad);
    for (int o = 16; o; o >>= 1) hs += __shfl_xor_sync(0xFFFFFFFFu, hs, o);
    if (lane == 0 && hs) atomicAdd(sym, (unsigned long long)hs);
}

__device__ __forceinline__ int64_t find_in_row(const int64_t *off, const int32_t *col, int32_t row,
                                                int32_t key) {
    int64_t lo = off[row], hi = off[row + 1];
    while (lo < hi) {
        int64_t mid = lo + ((hi - lo) >> 1);
        if (col[mid] < key) lo = mid + 1; else hi = mid;
    }
    return (lo < off[row + 1] && col[lo] == key) ? lo : -1;
}

static int read_flag(rs_graph *g, cudaStream_t s, int *out) {
    RS_CUDA_TRY(cudaMemcpyAsync(out, g->d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    RS_CUDA_TRY(cudaStreamSynchronize(s));
    return 0;
}

static int validate_graph(rs_graph *g, cudaStream_t s) {
    int flag = 0;
    RS_CUDA_TRY(cudaMemsetAsync(g->d_flag, 0, sizeof(int), s));
    validate_offsets_kernel<<<(unsigned)((g->n + 1 + 255) / 256), 256, 0, s>>>(g->off, g->n, g->nnz, g->d_flag);
    RS_CUDA_TRY(cudaGetLastError());
    if (int rc = read_flag(g, s, &flag)) return rc;
    if (flag) return fail(RS_EINVAL, "invalid graph: row_offsets must start at 0, end at nnz and not decrease");
    // with the offsets valid, one pass checks the rows and sums the symmetry hash
    unsigned long long *sym = (unsigned long long *)(g->d_flag + 8);      // ints 8..9 of the 16
    RS_CUDA_TRY(cudaMemsetAsync(sym, 0, sizeof(unsigned long long), s));
    validate_rows_kernel<<<grid_for(g->n, kThreads, 16), kThreads, 0, s>>>(g->off, g->col, g->lab, g->n, g->k,
                                                                         g->d_flag, sym);
    RS_CUDA_TRY(cudaGetLastError());
    unsigned long long h[2] = {0, 0};                                     // the flag word, then the sum
    RS_CUDA_TRY(cudaMemcpyAsync(h, g->d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    RS_CUDA_TRY(cudaMemcpyAsync(h + 1, sym, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    RS_CUDA_TRY(cudaStreamSynchronize(s));
    flag = (int)h[0];
    if (flag & V_COLRANGE) return fail(RS_EINVAL, "invalid graph: column id outside [0, n)");
    if (flag & V_SELF) return fail(RS_EINVAL, "invalid graph: self-loop");
    if (flag & V_ORDER) return fail(RS_EINVAL, "invalid graph: a row is not strictly ascending (unsorted or duplicate neighbour)");
    if (flag & V_LABEL) return fail(RS_EINVAL, "invalid graph: label outside [0, k)");
    if (h[1]) return fail(RS_EINVAL, "invalid graph: an edge is missing its reverse direction");
    return 0;
}

// ---------------------------------------------------------------------------
// row classification
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t row_cap(int64_t d, int32_t k) {
    int64_t m = d < k ? d : k;
    uint32_t cap = 1;
    while ((int64_t)cap < 2 * m) cap <<= 1;
    return cap;
}
// 0 small, 1 mid (warp), 2 large (CTA), 3 hub, by the split points of rs_tuning
struct ClassSplit { int32_t small_max, warp_cap, cta_cap; };
__device__ __forceinline__ int row_class(int64_t d, int32_t k, const ClassSplit &cs) {
    if (d <= cs.small_max) return 0;
    uint32_t cap = row_cap(d, k);
    if (cap <= (uint32_t)cs.warp_cap) return 1;
    return cap <= (uint32_t)cs.cta_cap ? 2 : 3;
}

// flags for one class into a[v], plus dmax / large cap / hub list on the first pass
// (a batch bounds each row's table by the communities of the row's own graph)
__global__ void classify_kernel(const int64_t *off, int64_t n, int32_t k, const int32_t *gid, const int32_t *gk,
                                ClassSplit cs, int cls, int64_t *a, int *dmax, int *largecap, int32_t *hub_list,
                                int *n_hub) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    int64_t d = off[v + 1] - off[v];
    if (gid) k = gk[gid[v]];
    int c = row_class(d, k, cs);
    a[v] = (c == cls) ? 1 : 0;
    if (cls == 0) {
        atomicMax(dmax, (int)d);
        if (c == 2) atomicMax(largecap, (int)row_cap(d, k));
        if (c == 3) hub_list[atomicAdd(n_hub, 1)] = (int32_t)v;
    }
}

// per hub: row bounds and the communities of its graph
// mid and large rows, largest first: the row kernels hand rows out dynamically,
// so taking the longest ones first leaves short rows for the end (bucket of a
// degree: 4 per octave, descending)
constexpr int kDegBuckets = 4 * 32;
__device__ __forceinline__ int desc_bucket(int64_t d) {
    int e = 63 - __clzll((long long)(d | 1));
    int q = e >= 2 ? (int)((d >> (e - 2)) & 3) : 0;
    return kDegBuckets - 1 - (4 * e + q);
}
// lanes with the same bucket count (and later take positions) with one atomic
__global__ void bucket_hist_kernel(const int64_t *off, const int32_t *rows, int64_t m, int *hist) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int b = i < m ? desc_bucket(off[rows[i] + 1] - off[rows[i]]) : kDegBuckets;
    unsigned same = __match_any_sync(0xFFFFFFFFu, b);
    if (i < m && (threadIdx.x & 31) == __ffs(same) - 1) atomicAdd(&hist[b], __popc(same));
}
__global__ void bucket_prefix_kernel(int *hist) {
    int acc = 0;
    for (int b = 0; b < kDegBuckets; ++b) { int c = hist[b]; hist[b] = acc; acc += c; }
}
__global__ void bucket_scatter_kernel(const int64_t *off, const int32_t *rows, int64_t m, int *cursor, int32_t *out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int b = i < m ? desc_bucket(off[rows[i] + 1] - off[rows[i]]) : kDegBuckets;
    unsigned same = __match_any_sync(0xFFFFFFFFu, b);
    int lane = threadIdx.x & 31, leader = __ffs(same) - 1;
    int base = 0;
    if (i < m && lane == leader) base = atomicAdd(&cursor[b], __popc(same));
    base = __shfl_sync(same, base, leader);
    if (i < m) out[base + __popc(same & ((1u << lane) - 1u))] = rows[i];
}

__global__ void hub_bounds_kernel(const int64_t *off, const int32_t *hubs, int64_t nh, int32_t k, const int32_t *gid,
                                  const int32_t *gk, int64_t *bounds) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nh) {
        int32_t h = hubs[i];
        bounds[3 * i] = off[h];
        bounds[3 * i + 1] = off[h + 1];
        bounds[3 * i + 2] = gid ? gk[gid[h]] : k;
    }
}

// distinct foreign communities of each hub row (neighbours outside the hub's own
// community), counted by inserting their labels into a scratch table per hub sized by
// the row's degree; the scoring tables are then sized by these counts
__global__ void hub_distinct_kernel(const int64_t *off, const int32_t *col, const int32_t *lab, const HubInfo *hubs,
                                    const int32_t *items, const int32_t *chunks, int64_t nitems, int32_t chunk_len,
                                    int32_t *tkey, int32_t *lf, int *err) {
    for (int64_t it = blockIdx.x; it < nitems; it += gridDim.x) {
        const HubInfo h = hubs[items[it]];
        const int64_t b = off[h.row], d = off[h.row + 1] - b;
        const int64_t lo = (int64_t)chunks[it] * chunk_len, hi = min(d, lo + chunk_len);
        const int32_t cv = lab[h.row];
        const uint32_t mask = (uint32_t)h.cap - 1;
        int32_t fresh = 0;
        for (int64_t e = lo + threadIdx.x; e < hi; e += blockDim.x) {
            const int32_t c = lab[col[b + e]];
            if (c == cv) continue;
            uint32_t s = hash_label(c);
            s = (s ^ (s >> 15)) & mask;
            uint32_t t = 0;
            for (; t <= mask; ++t) {
                const int32_t prev = atomicCAS(&tkey[h.tab + s], kEmpty, c);
                if (prev == kEmpty) { ++fresh; break; }
                if (prev == c) break;
                s = (s + 1) & mask;
            }
            if (t > mask) atomicOr(err, 1);
        }
        if (fresh) atomicAdd(&lf[items[it]], fresh);
    }
}

__global__ void scatter_class_kernel(const int64_t *a, int64_t n, int32_t *rows) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    int64_t prev = v ? a[v - 1] : 0;
    if (a[v] != prev) rows[prev] = (int32_t)v;
}

static void free_hub_tables(rs_graph *g) {
    void *ptrs[] = {g->hubs, g->hub_items, g->hub_item_chunk, g->hkey, g->hcnt, g->hq, g->hsig, g->hagg,
                    g->hitem_out, g->hitem_in, g->hub_sitem, g->hub_srange, g->hslot};
    pool_free_many(ptrs, sizeof(ptrs) / sizeof(ptrs[0]));
    g->hubs = nullptr; g->hub_items = g->hub_item_chunk = nullptr; g->hkey = nullptr;
    g->hub_sitem = g->hub_srange = g->hslot = nullptr;
    g->n_hub_sitems = 0;
    g->hcnt = nullptr; g->hq = nullptr; g->hsig = nullptr; g->hagg = nullptr;
    g->hitem_out = g->hitem_in = nullptr;
    g->n_hubs = g->n_hub_items = g->hub_slots = 0;
}

// ---------------------------------------------------------------------------
// device memory: one stream-ordered pool per device (created on first use)
// ---------------------------------------------------------------------------
namespace {
constexpr uint64_t kPoolKeep = 16ull << 30;      // freed bytes the pool keeps for reuse
constexpr int kMaxDevices = 64;
std::mutex pool_mutex;
cudaMemPool_t pools[kMaxDevices];
cudaStream_t pool_streams[kMaxDevices];

cudaError_t pool_of_device(cudaMemPool_t *pool, cudaStream_t *st) {
    int dev = 0;
    if (cudaError_t e = cudaGetDevice(&dev)) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(pool_mutex);
    if (!pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pl = nullptr;
        if (cudaError_t e = cudaMemPoolCreate(&pl, &props)) return e;
        uint64_t keep = kPoolKeep;
        if (cudaError_t e = cudaMemPoolSetAttribute(pl, cudaMemPoolAttrReleaseThreshold, &keep)) return e;
        cudaStream_t s = nullptr;
        if (cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) return e;
        pools[dev] = pl;
        pool_streams[dev] = s;
    }
    *pool = pools[dev];
    *st = pool_streams[dev];
    return cudaSuccess;
}
}  // namespace

cudaError_t rs::pool_malloc(void **p, size_t bytes) {
    cudaMemPool_t pl;
    cudaStream_t st;
    if (cudaError_t e = pool_of_device(&pl, &st)) return e;
    if (cudaError_t e = cudaMallocFromPoolAsync(p, std::max<size_t>(bytes, 1), pl, st)) return e;
    return cudaStreamSynchronize(st);            // usable on every stream from here on
}

cudaError_t rs::pool_free_many(void *const *p, size_t n) {
    bool any = false;
    for (size_t i = 0; i < n; ++i) any = any || p[i];
    if (!any) return cudaSuccess;
    cudaMemPool_t pl;
    cudaStream_t st;
    if (cudaError_t e = pool_of_device(&pl, &st)) return e;
    if (cudaError_t e = cudaDeviceSynchronize()) return e;   // no kernel still uses the blocks
    for (size_t i = 0; i < n; ++i)
        if (p[i])
            if (cudaError_t e = cudaFreeAsync(p[i], st)) return e;
    return cudaSuccess;
}

cudaError_t rs::pool_free(void *p) { return pool_free_many(&p, 1); }

template <class T>
static cudaError_t dmalloc(T **p, size_t count) {
    return pool_malloc((void **)p, std::max<size_t>(count, 1) * sizeof(T));
}

// builds rows_small / rows_mid / rows_large / hub tables from the current offsets; syncs
static int classify_rows(rs_graph *g, cudaStream_t s) {
    int64_t n = g->n;
    g->version++;                  // row lists and hub tables are rebuilt: captured steps are stale
    const ClassSplit cs{g->tune.small_max, g->tune.warp_cap, g->tune.cta_cap};
    int hdr[4] = {0, 0, 0, 0};   // dmax, large cap, n_hub, unused
    int *d_hdr = g->d_flag;      // d_flag has room for 4 ints
    RS_CUDA_TRY(cudaMemsetAsync(d_hdr, 0, 4 * sizeof(int), s));
    int32_t *hub_list = g->xout;  // n int32 scratch (workspace is allocated by now)
    unsigned blocks = (unsigned)((n + 255) / 256);
    int64_t *a = g->xoff;
    int32_t *lists[3] = {g->rows_small, g->rows_mid, g->rows_large};
    int64_t counts[3] = {0, 0, 0};
    for (int cls = 0; cls < 3; ++cls) {
        if (n > 0) {
            classify_kernel<<<blocks, 256, 0, s>>>(g->off, n, g->k, g->gid, g->gk, cs, cls, a, d_hdr, d_hdr + 1,
                                                   hub_list, d_hdr + 2);
            RS_CUDA_TRY(cudaGetLastError());
            if (int rc = inclusive_scan_i64(a, n, g->scan_tmp, s)) return rc;
            scatter_class_kernel<<<blocks, 256, 0, s>>>(a, n, lists[cls]);
            RS_CUDA_TRY(cudaGetLastError());
            RS_CUDA_TRY(cudaMemcpyAsync(&counts[cls], a + n - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        }
    }
    RS_CUDA_TRY(cudaMemcpyAsync(hdr, d_hdr, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
    RS_CUDA_TRY(cudaStreamSynchronize(s));
    g->n_small = counts[0]; g->n_mid = counts[1]; g->n_large = counts[2];
    g->dmax = hdr[0];
    g->large_cap = std::max(hdr[1], 64);
    // mid and large rows by degree, largest first (a counting sort by degree bucket through
    // the scratch list; the counters live in the scan scratch, free at this point)
    for (int cls = 1; cls < 3; ++cls) {
        int32_t *rows = cls == 1 ? g->rows_mid : g->rows_large;
        int64_t m = cls == 1 ? g->n_mid : g->n_large;
        if (m < 2) continue;
        int *hist = (int *)g->scan_tmp;
        unsigned mb = (unsigned)((m + 255) / 256);
        RS_CUDA_TRY(cudaMemsetAsync(hist, 0, kDegBuckets * sizeof(int), s));
        bucket_hist_kernel<<<mb, 256, 0, s>>>(g->off, rows, m, hist);
        RS_CUDA_TRY(cudaGetLastError());
        bucket_prefix_kernel<<<1, 1, 0, s>>>(hist);
        RS_CUDA_TRY(cudaGetLastError());
        bucket_scatter_kernel<<<mb, 256, 0, s>>>(g->off, rows, m, hist, g->rows_sort);
        RS_CUDA_TRY(cudaGetLastError());
        RS_CUDA_TRY(cudaMemcpyAsync(rows, g->rows_sort, m * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    }
    // hubs: host-side work list (hubs are few)
    int nh = hdr[2];
    std::vector<int32_t> hl(nh);
    std::vector<int64_t> offs(3 * (size_t)nh);
    if (nh) {
        // the hubs' row bounds and graph sizes in one gather and one copy
        int64_t *d_bounds = nullptr;
        RS_CUDA_TRY(dmalloc(&d_bounds, 3 * (size_t)nh));
        hub_bounds_kernel<<<(unsigned)((nh + 255) / 256), 256, 0, s>>>(g->off, hub_list, nh, g->k, g->gid, g->gk,
                                                                     d_bounds);
        cudaError_t e = cudaGetLastError();
        if (!e) e = cudaMemcpyAsync(hl.data(), hub_list, nh * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        if (!e) e = cudaMemcpyAsync(offs.data(), d_bounds, 3 * nh * sizeof(int64_t), cudaMemcpyDeviceToHost, s);
        if (!e) e = cudaStreamSynchronize(s);
        pool_free(d_bounds);
        if (e) return cuda_fail(e, "hub bounds");
        // sort the hubs by row id, keeping their bounds
        std::vector<int> order(nh);
        for (int i = 0; i < nh; ++i) order[i] = i;
        std::sort(order.begin(), order.end(), [&](int a, int b) { return hl[a] < hl[b]; });
        std::vector<int32_t> hl2(nh);
        std::vector<int64_t> offs2(3 * (size_t)nh);
        for (int i = 0; i < nh; ++i) {
            hl2[i] = hl[order[i]];
            for (int j = 0; j < 3; ++j) offs2[3 * i + j] = offs[3 * order[i] + j];
        }
        hl.swap(hl2);
        offs.swap(offs2);
    }
    std::vector<HubInfo> info(nh);
    std::vector<int32_t> items, chunks;
    int64_t slots = 0, hub_entries = 0;
    for (int i = 0; i < nh; ++i) {
        int64_t d = offs[3 * i + 1] - offs[3 * i];
        info[i].ent = hub_entries;
        hub_entries += d;
        int64_t m = std::min<int64_t>(d, offs[3 * i + 2]);
        info[i].row = hl[i];
        info[i].cap = (int32_t)pow2_at_least((uint64_t)(2 * m));   // by degree: the scratch count below
        info[i].tab = slots;
        info[i].first_item = (int32_t)items.size();
        int nc = (int)((d + g->tune.hub_chunk - 1) / g->tune.hub_chunk);
        info[i].n_items = nc;
        for (int c = 0; c < nc; ++c) { items.push_back(i); chunks.push_back(c); }
        slots += info[i].cap;
    }
    free_hub_tables(g);
    g->n_hubs = nh;
    g->n_hub_items = (int64_t)items.size();
    if (nh) {
        RS_CUDA_TRY(dmalloc(&g->hubs, nh));
        RS_CUDA_TRY(dmalloc(&g->hub_items, items.size()));
        RS_CUDA_TRY(dmalloc(&g->hub_item_chunk, items.size()));
        RS_CUDA_TRY(cudaMemcpy(g->hubs, info.data(), nh * sizeof(HubInfo), cudaMemcpyHostToDevice));
        RS_CUDA_TRY(cudaMemcpy(g->hub_items, items.data(), items.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
        RS_CUDA_TRY(cudaMemcpy(g->hub_item_chunk, chunks.data(), chunks.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
        // each hub's distinct foreign communities L_f, in scratch tables sized by degree;
        // the scoring tables then take 2 L_f slots (rounded up to a power of two), which
        // is far less on hub-skewed graphs (degree 54,097 with 4,671 communities)
        int32_t *tkey = nullptr, *lf = nullptr;
        cudaError_t e = dmalloc(&tkey, (size_t)slots);
        if (!e) e = dmalloc(&lf, (size_t)nh);
        if (!e) e = cudaMemsetAsync(tkey, 0xFF, (size_t)slots * sizeof(int32_t), s);
        if (!e) e = cudaMemsetAsync(lf, 0, (size_t)nh * sizeof(int32_t), s);
        if (!e) e = cudaMemsetAsync(d_hdr + 3, 0, sizeof(int), s);
        if (!e) {
            hub_distinct_kernel<<<grid_for((int64_t)items.size(), 1, 8), 256, 0, s>>>(
                g->off, g->col, g->lab, g->hubs, g->hub_items, g->hub_item_chunk, (int64_t)items.size(),
                g->tune.hub_chunk, tkey, lf, d_hdr + 3);
            e = cudaGetLastError();
        }
        std::vector<int32_t> L(nh);
        int overflow = 0;
        if (!e) e = cudaMemcpyAsync(L.data(), lf, nh * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        if (!e) e = cudaMemcpyAsync(&overflow, d_hdr + 3, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (!e) e = cudaStreamSynchronize(s);
        pool_free(tkey);
        pool_free(lf);
        if (e) return cuda_fail(e, "hub community counts");
        if (overflow) return fail(RS_ECUDA, "hub community count: scratch table full (library bug)");
        slots = 0;
        for (int i = 0; i < nh; ++i) {
            info[i].cap = (int32_t)std::max<uint64_t>(2, pow2_at_least((uint64_t)(2 * (int64_t)L[i])));
            info[i].tab = slots;
            slots += info[i].cap;
        }
        RS_CUDA_TRY(cudaMemcpy(g->hubs, info.data(), nh * sizeof(HubInfo), cudaMemcpyHostToDevice));
        std::vector<int32_t> sitem, srange;
        for (int i = 0; i < nh; ++i)
            for (int32_t r = 0; (int64_t)r * kHubSlotRange < info[i].cap; ++r) {
                sitem.push_back(i);
                srange.push_back(r);
            }
        g->n_hub_sitems = (int64_t)sitem.size();
        RS_CUDA_TRY(dmalloc(&g->hub_sitem, sitem.size()));
        RS_CUDA_TRY(dmalloc(&g->hub_srange, srange.size()));
        RS_CUDA_TRY(cudaMemcpy(g->hub_sitem, sitem.data(), sitem.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
        RS_CUDA_TRY(cudaMemcpy(g->hub_srange, srange.data(), srange.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
        RS_CUDA_TRY(dmalloc(&g->hslot, (size_t)hub_entries));
        RS_CUDA_TRY(dmalloc(&g->hkey, slots));
        RS_CUDA_TRY(dmalloc(&g->hcnt, slots));
        RS_CUDA_TRY(dmalloc(&g->hq, 2 * slots));
        RS_CUDA_TRY(dmalloc(&g->hsig, slots));
        RS_CUDA_TRY(dmalloc(&g->hagg, nh));
        RS_CUDA_TRY(dmalloc(&g->hitem_out, items.size()));
        RS_CUDA_TRY(dmalloc(&g->hitem_in, items.size()));
    }
    g->hub_slots = slots;
    return 0;
}

int rs::reclassify(rs_graph *g, cudaStream_t s) {
    if (int rc = classify_rows(g, s)) return rc;
    RS_CUDA_TRY(cudaStreamSynchronize(s));
    return 0;
}

static int build_tables(rs_graph *g, cudaStream_t s) {
    pool_free(g->LG); pool_free(g->RD);
    g->LG = nullptr; g->RD = nullptr;
    int64_t m = (int64_t)g->dmax + 1;
    RS_CUDA_TRY(dmalloc(&g->LG, m));
    RS_CUDA_TRY(dmalloc(&g->RD, m));
    init_tables_kernel<<<(unsigned)((m + 127) / 128), 128, 0, s>>>(g->LG, g->RD, g->dmax, g->alg2 ? 1 : 0);
    RS_CUDA_TRY(cudaGetLastError());
    return 0;
}

// xR (one reverse value per G_x slot) exists while the mirror pass is selected
int rs::set_mirror_buffer(rs_graph *g) {
    if (g->tune.p3_mirror && !g->xR) {
        RS_CUDA_TRY(dmalloc(&g->xR, std::max<int64_t>(g->nnz, 1)));
        RS_CUDA_TRY(dmalloc(&g->xtile, g->nnz / kMirTile + 2));
    } else if (!g->tune.p3_mirror && g->xR) {
        RS_CUDA_TRY(pool_free(g->xR));
        RS_CUDA_TRY(pool_free(g->xtile));
        g->xR = nullptr;
        g->xtile = nullptr;
    }
    return 0;
}

static int alloc_workspace(rs_graph *g) {
    int64_t n = g->n, nnz = g->nnz;
    // streams 0 and 1 carry the many-short-rows kernels at the lowest priority; the
    // others carry rows with long dependent chains, whose blocks go first
    int lowest = 0, highest = 0;
    RS_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&lowest, &highest));
    for (int i = 0; i < rs_graph::kAux; ++i) {
        RS_CUDA_TRY(cudaStreamCreateWithPriority(&g->aux[i], cudaStreamNonBlocking, i < 2 ? lowest : highest));
        RS_CUDA_TRY(cudaEventCreateWithFlags(&g->ev_join[i], cudaEventDisableTiming));
    }
    RS_CUDA_TRY(cudaEventCreateWithFlags(&g->ev_fork, cudaEventDisableTiming));
    RS_CUDA_TRY(dmalloc(&g->rec, n));
    RS_CUDA_TRY(dmalloc(&g->acc, 2 * n));
    RS_CUDA_TRY(dmalloc(&g->wmax_bits, g->n_graphs));
    RS_CUDA_TRY(dmalloc(&g->winv, g->n_graphs));
    RS_CUDA_TRY(dmalloc(&g->Lall, n));
    RS_CUDA_TRY(dmalloc(&g->rsum, n));
    RS_CUDA_TRY(dmalloc(&g->cl_col, nnz));
    RS_CUDA_TRY(dmalloc(&g->cl_lab, nnz));
    RS_CUDA_TRY(dmalloc(&g->xoff, n + 1));
    RS_CUDA_TRY(dmalloc(&g->xcol, nnz + 8));
    RS_CUDA_TRY(dmalloc(&g->xsk, nnz / 8 + 1));
    RS_CUDA_TRY(dmalloc(&g->xS, nnz));
    RS_CUDA_TRY(dmalloc(&g->xout, n));
    RS_CUDA_TRY(dmalloc(&g->xin, n));
    if (int rc = rs::set_mirror_buffer(g)) return rc;
    RS_CUDA_TRY(dmalloc(&g->p2rows, 4 * (size_t)n));
    RS_CUDA_TRY(dmalloc(&g->p2cnt, 16));
    RS_CUDA_TRY(dmalloc(&g->wq, wq_words(n, nnz)));
    if (g->strict) RS_CUDA_TRY(dmalloc(&g->sx, 2 * (size_t)nnz));
    RS_CUDA_TRY(dmalloc(&g->scan_tmp, scan_tmp_words(std::max<int64_t>(n + 1, 1)) + 64));
    RS_CUDA_TRY(dmalloc(&g->rows_small, n));
    RS_CUDA_TRY(dmalloc(&g->rows_mid, n));
    RS_CUDA_TRY(dmalloc(&g->rows_large, n));
    RS_CUDA_TRY(dmalloc(&g->rows_sort, n));
    RS_CUDA_TRY(dmalloc(&g->d_flag, 64));
    return 0;
}

static void free_graph(rs_graph *g) {
    if (!g) return;
    void *ptrs[] = {g->off, g->off_alt, g->col, g->col_alt, g->lab, g->removed, g->dead,
                    g->rows_small, g->rows_mid, g->rows_large, g->rows_sort, g->LG, g->RD, g->rec, g->acc, g->wmax_bits,
                    g->Lall, g->xoff, g->xcol, g->xsk, g->xS, g->xout, g->xin, g->scan_tmp, g->tk_hist,
                    g->tk_ctrl, g->tk_keys, g->tk_ids, g->d_flag, g->xR, g->xtile, g->rsum, g->cl_col, g->cl_lab,
                    g->winv, g->gid, g->gk, g->gnode, g->p2rows, g->p2cnt, g->sx, g->wq, g->perm};
    pool_free_many(ptrs, sizeof(ptrs) / sizeof(ptrs[0]));
    free_hub_tables(g);
    for (cudaEvent_t e : g->prof_ev) cudaEventDestroy(e);
    for (int i = 0; i < rs_graph::kAux; ++i) {
        if (g->aux[i]) cudaStreamDestroy(g->aux[i]);
        if (g->ev_join[i]) cudaEventDestroy(g->ev_join[i]);
    }
    if (g->ev_fork) cudaEventDestroy(g->ev_fork);
    delete g;
}

__global__ void widen_offsets_kernel(const int32_t *in, int64_t *out, int64_t m) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) out[i] = in[i];
}

// allocations and tables for a graph whose CSR/labels/removed are already on the device
static int reorder_graph(rs_graph *g, cudaStream_t s);

static int finish_graph(rs_graph *g, cudaStream_t s, bool reorder = false) {
    if (int rc = alloc_workspace(g)) return rc;
    if (reorder)
        if (int rc = reorder_graph(g, s)) return rc;
    if (int rc = classify_rows(g, s)) return rc;
    if (g->dmax >= (1 << 24)) return fail(RS_EINVAL, "max degree must be < 2^24");
    if (int rc = build_tables(g, s)) return rc;
    RS_CUDA_TRY(cudaStreamSynchronize(s));
    return 0;
}

static rs_status rs_build_graph_impl(int64_t n, int64_t nnz, const void *row_offsets, int offsets_are_i64,
                                     const int32_t *cols, const int32_t *labels, int32_t num_communities,
                                     int inputs_on_device, uint32_t flags, cudaStream_t s, rs_graph **out,
                                     bool finish) {
    if (!out) return (rs_status)fail(RS_EINVAL, "rs_build_graph: out is NULL");
    if (n < 0 || n >= (1LL << 31)) return (rs_status)fail(RS_EINVAL, "rs_build_graph: n must be in [0, 2^31)");
    if (nnz < 0 || nnz >= (1LL << 40)) return (rs_status)fail(RS_EINVAL, "rs_build_graph: nnz must be in [0, 2^40)");
    if (!offsets_are_i64 && nnz >= (1LL << 31))
        return (rs_status)fail(RS_EINVAL, "rs_build_graph: nnz >= 2^31 needs int64 offsets");
    if (num_communities < 1) return (rs_status)fail(RS_EINVAL, "rs_build_graph: num_communities must be >= 1");
    if (!row_offsets || (nnz > 0 && !cols) || (n > 0 && !labels))
        return (rs_status)fail(RS_EINVAL, "rs_build_graph: NULL input array");
    rs_graph *g = new rs_graph();
    g->n = n; g->nnz = nnz; g->k = num_communities;
    g->alg2 = (flags & RS_ALG2_COMPAT) != 0;
    g->strict = (flags & RS_TRIAD_STRICT) != 0;
    cudaGetDevice(&g->device);
    auto bail = [&](int rc) { free_graph(g); return (rs_status)rc; };
    cudaMemcpyKind kind = inputs_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (cudaError_t e = dmalloc(&g->off, n + 1)) return bail(cuda_fail(e, "alloc offsets"));
    if (cudaError_t e = dmalloc(&g->off_alt, n + 1)) return bail(cuda_fail(e, "alloc offsets"));
    if (cudaError_t e = dmalloc(&g->col, nnz)) return bail(cuda_fail(e, "alloc cols"));
    if (cudaError_t e = dmalloc(&g->col_alt, nnz)) return bail(cuda_fail(e, "alloc cols"));
    if (cudaError_t e = dmalloc(&g->lab, n)) return bail(cuda_fail(e, "alloc labels"));
    if (cudaError_t e = dmalloc(&g->removed, 4 * std::max<int64_t>(n, 1))) return bail(cuda_fail(e, "alloc flags"));
    if (cudaError_t e = dmalloc(&g->dead, 4 * ((nnz + 31) / 32))) return bail(cuda_fail(e, "alloc marks"));
    if (offsets_are_i64) {
        if (cudaError_t e = cudaMemcpyAsync(g->off, row_offsets, (n + 1) * sizeof(int64_t), kind, s))
            return bail(cuda_fail(e, "copy offsets"));
    } else {
        // stage int32 offsets in col_alt's storage when it is large enough, else a temporary
        int32_t *tmp = nullptr;
        if (cudaError_t e = dmalloc(&tmp, n + 1)) return bail(cuda_fail(e, "alloc offsets"));
        cudaError_t e = cudaMemcpyAsync(tmp, row_offsets, (n + 1) * sizeof(int32_t), kind, s);
        if (!e) {
            widen_offsets_kernel<<<(unsigned)((n + 1 + 255) / 256), 256, 0, s>>>(tmp, g->off, n + 1);
            e = cudaGetLastError();
        }
        if (!e) e = cudaStreamSynchronize(s);
        pool_free(tmp);
        if (e) return bail(cuda_fail(e, "copy offsets"));
    }
    if (nnz > 0)
        if (cudaError_t e = cudaMemcpyAsync(g->col, cols, nnz * sizeof(int32_t), kind, s))
            return bail(cuda_fail(e, "copy cols"));
    if (n > 0)
        if (cudaError_t e = cudaMemcpyAsync(g->lab, labels, n * sizeof(int32_t), kind, s))
            return bail(cuda_fail(e, "copy labels"));
    if (cudaError_t e = cudaMemsetAsync(g->removed, 0, 4 * std::max<int64_t>(n, 1), s))
        return bail(cuda_fail(e, "clear flags"));
    if (cudaError_t e = dmalloc(&g->d_flag, 16)) return bail(cuda_fail(e, "alloc flag"));   // flags + 2 hash sums
    if (flags & RS_VALIDATE) {
        if (int rc = validate_graph(g, s)) return bail(rc);
    }
    if ((flags & RS_REORDER) && !finish) return bail(fail(RS_EINVAL, "rs_build_batch: RS_REORDER is for single graphs"));
    if (!finish) {                 // the caller completes the graph (batches)
        *out = g;
        return RS_OK;
    }
    pool_free(g->d_flag);
    g->d_flag = nullptr;
    if (int rc = finish_graph(g, s, (flags & RS_REORDER) != 0)) return bail(rc);
    *out = g;
    return RS_OK;
}

extern "C" rs_status rs_build_graph(int64_t n, int64_t nnz, const void *row_offsets, int offsets_are_i64,
                                    const int32_t *cols, const int32_t *labels, int32_t num_communities,
                                    int inputs_on_device, uint32_t flags, void *stream, rs_graph **out) {
    return rs_build_graph_impl(n, nnz, row_offsets, offsets_are_i64, cols, labels, num_communities,
                               inputs_on_device, flags, as_stream(stream), out, true);
}

// ---------------------------------------------------------------------------
// batches of independent graphs packed into one CSR
// ---------------------------------------------------------------------------
__global__ void batch_gid_kernel(const int64_t *gnode, int32_t ng, int64_t n, int32_t *gid) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    int32_t lo = 0, hi = ng;                    // last graph with gnode[g] <= v
    while (hi - lo > 1) {
        int32_t mid = (lo + hi) >> 1;
        if (gnode[mid] <= v) lo = mid; else hi = mid;
    }
    gid[v] = lo;
}

// every neighbour inside the row's graph, every label inside [0, k of the graph)
__global__ void batch_validate_kernel(const int64_t *off, const int32_t *col, const int32_t *lab,
                                      const int32_t *gid, const int64_t *gnode, const int32_t *gk, int64_t n,
                                      int *flag) {
    int lane = threadIdx.x & 31;
    int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = w; v < n; v += nw) {
        int32_t gi = gid[v];
        int64_t lo = gnode[gi], hi = gnode[gi + 1];
        int bad = 0;
        if (lane == 0 && (lab[v] < 0 || lab[v] >= gk[gi])) bad |= 1;
        for (int64_t e = off[v] + lane; e < off[v + 1]; e += 32)
            if (col[e] < lo || col[e] >= hi) bad |= 2;
        if (bad) atomicOr(flag, bad);
    }
}

__global__ void batch_labels_kernel(int32_t *lab, const int32_t *gid, const int64_t *koff, int64_t n) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) lab[v] = (int32_t)(lab[v] + koff[gid[v]]);
}

extern "C" rs_status rs_build_batch(int32_t n_graphs, const int64_t *graph_node_offsets, const int32_t *graph_k,
                                    int64_t nnz, const void *row_offsets, int offsets_are_i64, const int32_t *cols,
                                    const int32_t *labels, int inputs_on_device, uint32_t flags, void *stream,
                                    rs_graph **out) {
    cudaStream_t s = as_stream(stream);
    if (!out || !graph_node_offsets || !graph_k || n_graphs < 1)
        return (rs_status)fail(RS_EINVAL, "rs_build_batch: bad arguments");
    if (graph_node_offsets[0] != 0) return (rs_status)fail(RS_EINVAL, "rs_build_batch: graph offsets must start at 0");
    int64_t ksum = 0;
    std::vector<int64_t> koff(n_graphs);
    for (int32_t i = 0; i < n_graphs; ++i) {
        if (graph_node_offsets[i + 1] < graph_node_offsets[i])
            return (rs_status)fail(RS_EINVAL, "rs_build_batch: graph offsets decrease");
        if (graph_k[i] < 1) return (rs_status)fail(RS_EINVAL, "rs_build_batch: every graph needs k >= 1");
        koff[i] = ksum;
        ksum += graph_k[i];
    }
    if (ksum >= (1LL << 31)) return (rs_status)fail(RS_EINVAL, "rs_build_batch: too many communities in total");
    int64_t n = graph_node_offsets[n_graphs];
    // load the packed CSR as one graph; labels are still local to their graph here
    rs_graph *g = nullptr;
    int32_t kmax = 1;
    for (int32_t i = 0; i < n_graphs; ++i) kmax = std::max(kmax, graph_k[i]);
    rs_status st = rs_build_graph_impl(n, nnz, row_offsets, offsets_are_i64, cols, labels, kmax, inputs_on_device,
                                       flags & ~RS_VALIDATE, s, &g, /*finish=*/false);
    if (st != RS_OK) return st;
    auto bail = [&](int rc) { free_graph(g); return (rs_status)rc; };
    g->n_graphs = n_graphs;
    if (cudaError_t e = dmalloc(&g->gid, n)) return bail(cuda_fail(e, "alloc batch"));
    if (cudaError_t e = dmalloc(&g->gk, n_graphs)) return bail(cuda_fail(e, "alloc batch"));
    if (cudaError_t e = dmalloc(&g->gnode, n_graphs + 1)) return bail(cuda_fail(e, "alloc batch"));
    int64_t *d_koff = nullptr;
    if (cudaError_t e = dmalloc(&d_koff, n_graphs)) return bail(cuda_fail(e, "alloc batch"));
    cudaError_t e = cudaMemcpyAsync(g->gnode, graph_node_offsets, (n_graphs + 1) * sizeof(int64_t),
                                    cudaMemcpyHostToDevice, s);
    if (!e) e = cudaMemcpyAsync(g->gk, graph_k, n_graphs * sizeof(int32_t), cudaMemcpyHostToDevice, s);
    if (!e) e = cudaMemcpyAsync(d_koff, koff.data(), n_graphs * sizeof(int64_t), cudaMemcpyHostToDevice, s);
    if (!e && n > 0) {
        batch_gid_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(g->gnode, n_graphs, n, g->gid);
        e = cudaGetLastError();
    }
    if (!e) e = cudaStreamSynchronize(s);
    if (e) { pool_free(d_koff); return bail(cuda_fail(e, "batch set-up")); }
    if (flags & RS_VALIDATE) {
        g->k = (int32_t)std::min<int64_t>(kmax, INT32_MAX);
        int rc = validate_graph(g, s);
        int flag = 0;
        if (!rc) {
            e = cudaMemsetAsync(g->d_flag, 0, sizeof(int), s);
            if (!e && n > 0) {
                batch_validate_kernel<<<grid_for(n * 32, kThreads, 16), kThreads, 0, s>>>(
                    g->off, g->col, g->lab, g->gid, g->gnode, g->gk, n, g->d_flag);
                e = cudaGetLastError();
            }
            if (!e) rc = read_flag(g, s, &flag); else rc = cuda_fail(e, "batch validation");
        }
        if (!rc && (flag & 2)) rc = fail(RS_EINVAL, "invalid batch: an edge leaves its graph");
        if (!rc && (flag & 1)) rc = fail(RS_EINVAL, "invalid batch: a label outside [0, k of its graph)");
        if (rc) { pool_free(d_koff); return bail(rc); }
    }
    if (n > 0) {
        batch_labels_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(g->lab, g->gid, d_koff, n);
        e = cudaGetLastError();
        if (!e) e = cudaStreamSynchronize(s);
    }
    pool_free(d_koff);
    if (e) return bail(cuda_fail(e, "batch labels"));
    g->k = (int32_t)ksum;
    pool_free(g->d_flag);
    g->d_flag = nullptr;
    if (int rc = finish_graph(g, s)) return bail(rc);
    *out = g;
    return RS_OK;
}

extern "C" rs_status rs_batch_omega_max(rs_graph *g, double *wmax_out, void *stream) {
    if (!g || !wmax_out) return (rs_status)fail(RS_EINVAL, "rs_batch_omega_max: NULL argument");
    std::vector<unsigned long long> bits(g->n_graphs);
    cudaStream_t s = as_stream(stream);
    if (cudaError_t e = cudaMemcpyAsync(bits.data(), g->wmax_bits, g->n_graphs * sizeof(unsigned long long),
                                        cudaMemcpyDeviceToHost, s))
        return (rs_status)cuda_fail(e, "read w_max");
    if (cudaError_t e = cudaStreamSynchronize(s)) return (rs_status)cuda_fail(e, "read w_max");
    for (int32_t i = 0; i < g->n_graphs; ++i) memcpy(&wmax_out[i], &bits[i], sizeof(double));
    return RS_OK;
}

extern "C" void rs_free_graph(rs_graph *g) { free_graph(g); }

extern "C" rs_status rs_graph_info(const rs_graph *g, int64_t *n, int64_t *nnz, int32_t *k, int32_t *max_degree) {
    if (!g) return (rs_status)fail(RS_EINVAL, "rs_graph_info: NULL graph");
    if (n) *n = g->n;
    if (nnz) *nnz = g->nnz;
    if (k) *k = g->k;
    if (max_degree) *max_degree = g->dmax;
    return RS_OK;
}

extern "C" rs_status rs_clone_graph(const rs_graph *src, rs_graph **out, void *stream) {
    cudaStream_t s = as_stream(stream);
    if (!src || !out) return (rs_status)fail(RS_EINVAL, "rs_clone_graph: NULL argument");
    rs_graph *g = new rs_graph();
    g->n = src->n; g->nnz = src->nnz; g->k = src->k; g->device = src->device;
    g->tune = src->tune;
    g->alg2 = src->alg2;
    g->strict = src->strict;
    auto bail = [&](int rc) { free_graph(g); return (rs_status)rc; };
    int64_t n = g->n, nnz = g->nnz;
    if (cudaError_t e = dmalloc(&g->off, n + 1)) return bail(cuda_fail(e, "alloc"));
    if (cudaError_t e = dmalloc(&g->off_alt, n + 1)) return bail(cuda_fail(e, "alloc"));
    if (cudaError_t e = dmalloc(&g->col, nnz)) return bail(cuda_fail(e, "alloc"));
    if (cudaError_t e = dmalloc(&g->col_alt, nnz)) return bail(cuda_fail(e, "alloc"));
    if (cudaError_t e = dmalloc(&g->lab, n)) return bail(cuda_fail(e, "alloc"));
    if (cudaError_t e = dmalloc(&g->removed, 4 * std::max<int64_t>(n, 1))) return bail(cuda_fail(e, "alloc"));
    if (cudaError_t e = dmalloc(&g->dead, 4 * ((nnz + 31) / 32))) return bail(cuda_fail(e, "alloc"));
    int64_t cur_nnz = 0;
    if (cudaError_t e = cudaMemcpy(&cur_nnz, src->off + n, sizeof(int64_t), cudaMemcpyDeviceToHost))
        return bail(cuda_fail(e, "read offsets"));
    cudaError_t e = cudaMemcpyAsync(g->off, src->off, (n + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s);
    if (!e && cur_nnz) e = cudaMemcpyAsync(g->col, src->col, cur_nnz * sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
    if (!e && n) e = cudaMemcpyAsync(g->lab, src->lab, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
    if (!e && n) e = cudaMemcpyAsync(g->removed, src->removed, 4 * n, cudaMemcpyDeviceToDevice, s);
    if (!e && src->perm) {
        g->iperm = src->iperm;
        e = dmalloc(&g->perm, n);
        if (!e) e = cudaMemcpyAsync(g->perm, src->perm, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
    }
    if (e) return bail(cuda_fail(e, "copy graph"));
    g->n_graphs = src->n_graphs;
    if (src->gid) {
        if ((e = dmalloc(&g->gid, n))) return bail(cuda_fail(e, "alloc batch"));
        if ((e = dmalloc(&g->gk, g->n_graphs))) return bail(cuda_fail(e, "alloc batch"));
        if ((e = dmalloc(&g->gnode, g->n_graphs + 1))) return bail(cuda_fail(e, "alloc batch"));
        e = cudaMemcpyAsync(g->gid, src->gid, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
        if (!e) e = cudaMemcpyAsync(g->gk, src->gk, g->n_graphs * sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
        if (!e) e = cudaMemcpyAsync(g->gnode, src->gnode, (g->n_graphs + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s);
        if (e) return bail(cuda_fail(e, "copy batch"));
    }
    if (int rc = finish_graph(g, s)) return bail(rc);
    *out = g;
    return RS_OK;
}

// ---------------------------------------------------------------------------
// removals: mark dead CSR entries (bit set), then compact into the alt buffers
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool mark_dead(uint32_t *dead, int64_t e) {
    uint32_t bit = 1u << (e & 31);
    return (atomicOr(&dead[e >> 5], bit) & bit) == 0;
}

__global__ void remove_nodes_kernel(const int64_t *off, const int32_t *col, int32_t *removed,
                                    uint32_t *dead, const int32_t *nodes, int64_t m,
                                    unsigned long long *applied) {
    int lane = threadIdx.x & 31;
    int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = w; i < m; i += nw) {
        int32_t v = nodes[i];
        int first = 0;
        if (lane == 0) first = atomicExch(&removed[v], 1) == 0;
        first = __shfl_sync(0xFFFFFFFFu, first, 0);
        if (!first) continue;
        if (lane == 0) atomicAdd(applied, 1ull);
        for (int64_t e = off[v] + lane; e < off[v + 1]; e += 32) {
            mark_dead(dead, e);
            int64_t r = find_in_row(off, col, col[e], v);
            if (r >= 0) mark_dead(dead, r);
        }
    }
}

__global__ void remove_edges_kernel(const int64_t *off, const int32_t *col, uint32_t *dead,
                                    const int32_t *src, const int32_t *dst, int64_t m,
                                    unsigned long long *applied) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    int32_t a = src[i], b = dst[i];
    if (a == b) return;
    int32_t lo = a < b ? a : b, hi = a < b ? b : a;
    int64_t e = find_in_row(off, col, lo, hi);
    if (e < 0) return;
    // the entry in the smaller endpoint's row decides, so (a,b) and (b,a) count once
    if (!mark_dead(dead, e)) return;
    int64_t r = find_in_row(off, col, hi, lo);
    if (r >= 0) mark_dead(dead, r);
    atomicAdd(applied, 1ull);
}

__global__ void alive_degree_kernel(const int64_t *off, const uint32_t *dead, int64_t n, int64_t *deg) {
    int lane = threadIdx.x & 31;
    int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = w; v < n; v += nw) {
        int64_t c = 0;
        for (int64_t e = off[v] + lane; e < off[v + 1]; e += 32) c += !((dead[e >> 5] >> (e & 31)) & 1u);
        for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
        if (lane == 0) deg[v + 1] = c;
        if (v == 0 && lane == 0) deg[0] = 0;
    }
}

__global__ void compact_rows_kernel(const int64_t *off, const int32_t *col, const uint32_t *dead,
                                    int64_t n, const int64_t *noff, int32_t *ncol) {
    int lane = threadIdx.x & 31;
    int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = w; v < n; v += nw) {
        int64_t out = noff[v];
        for (int64_t base = off[v]; base < off[v + 1]; base += 32) {
            int64_t e = base + lane;
            bool keep = e < off[v + 1] && !((dead[e >> 5] >> (e & 31)) & 1u);
            unsigned m = __ballot_sync(0xFFFFFFFFu, keep);
            if (keep) ncol[out + __popc(m & ((1u << lane) - 1))] = col[e];
            out += __popc(m);
        }
    }
}

extern "C" rs_status rs_apply_removals(rs_graph *g, const int32_t *nodes, int64_t n_nodes,
                                       const int32_t *edge_src, const int32_t *edge_dst, int64_t n_edges,
                                       int64_t *applied_out, void *stream) {
    cudaStream_t s = as_stream(stream);
    if (!g) return (rs_status)fail(RS_EINVAL, "rs_apply_removals: NULL graph");
    if (n_nodes < 0 || n_edges < 0 || (n_nodes && !nodes) || (n_edges && (!edge_src || !edge_dst)))
        return (rs_status)fail(RS_EINVAL, "rs_apply_removals: bad arrays");
    for (int64_t i = 0; i < n_nodes; ++i)
        if (nodes[i] < 0 || nodes[i] >= g->n)
            return (rs_status)fail(RS_EINVAL, "rs_apply_removals: node id out of range");
    for (int64_t i = 0; i < n_edges; ++i)
        if (edge_src[i] < 0 || edge_src[i] >= g->n || edge_dst[i] < 0 || edge_dst[i] >= g->n)
            return (rs_status)fail(RS_EINVAL, "rs_apply_removals: edge endpoint out of range");
    // a reordered graph takes the caller's ids: map them to internal ones
    std::vector<int32_t> mapped;
    if (g->perm) {
        mapped.resize(n_nodes + 2 * n_edges);
        for (int64_t i = 0; i < n_nodes; ++i) mapped[i] = g->iperm[nodes[i]];
        for (int64_t i = 0; i < n_edges; ++i) {
            mapped[n_nodes + i] = g->iperm[edge_src[i]];
            mapped[n_nodes + n_edges + i] = g->iperm[edge_dst[i]];
        }
        nodes = mapped.data();
        edge_src = mapped.data() + n_nodes;
        edge_dst = mapped.data() + n_nodes + n_edges;
    }
    int32_t *buf = nullptr;
    unsigned long long *d_applied = nullptr;
    int64_t words = n_nodes + 2 * n_edges;
    auto done = [&](int rc) { pool_free(buf); pool_free(d_applied); return (rs_status)rc; };
    if (cudaError_t e = dmalloc(&buf, words)) return done(cuda_fail(e, "alloc removal lists"));
    if (cudaError_t e = dmalloc(&d_applied, 1)) return done(cuda_fail(e, "alloc counter"));
    cudaError_t e = cudaMemsetAsync(d_applied, 0, sizeof(unsigned long long), s);
    if (!e && n_nodes) e = cudaMemcpyAsync(buf, nodes, n_nodes * 4, cudaMemcpyHostToDevice, s);
    if (!e && n_edges) e = cudaMemcpyAsync(buf + n_nodes, edge_src, n_edges * 4, cudaMemcpyHostToDevice, s);
    if (!e && n_edges) e = cudaMemcpyAsync(buf + n_nodes + n_edges, edge_dst, n_edges * 4, cudaMemcpyHostToDevice, s);
    int64_t nnz_cur = 0;
    if (!e) e = cudaMemcpyAsync(&nnz_cur, g->off + g->n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (!e && nnz_cur) e = cudaMemsetAsync(g->dead, 0, 4 * ((nnz_cur + 31) / 32), s);
    if (e) return done(cuda_fail(e, "stage removals"));
    if (n_nodes) {
        remove_nodes_kernel<<<grid_for(n_nodes * 32, kThreads, 8), kThreads, 0, s>>>(
            g->off, g->col, (int32_t *)g->removed, (uint32_t *)g->dead, buf, n_nodes, d_applied);
        if ((e = cudaGetLastError())) return done(cuda_fail(e, "remove nodes"));
    }
    if (n_edges) {
        remove_edges_kernel<<<(unsigned)((n_edges + 255) / 256), 256, 0, s>>>(
            g->off, g->col, (uint32_t *)g->dead, buf + n_nodes, buf + n_nodes + n_edges, n_edges, d_applied);
        if ((e = cudaGetLastError())) return done(cuda_fail(e, "remove edges"));
    }
    if (g->n > 0) {
        int grid = grid_for(g->n * 32, kThreads, 16);
        alive_degree_kernel<<<grid, kThreads, 0, s>>>(g->off, (uint32_t *)g->dead, g->n, g->off_alt);
        if ((e = cudaGetLastError())) return done(cuda_fail(e, "count alive"));
        if (int rc = inclusive_scan_i64(g->off_alt + 1, g->n, g->scan_tmp, s)) return done(rc);
        compact_rows_kernel<<<grid, kThreads, 0, s>>>(g->off, g->col, (uint32_t *)g->dead, g->n, g->off_alt, g->col_alt);
        if ((e = cudaGetLastError())) return done(cuda_fail(e, "compact rows"));
        std::swap(g->off, g->off_alt);
        std::swap(g->col, g->col_alt);
    }
    unsigned long long applied = 0;
    if ((e = cudaMemcpyAsync(&applied, d_applied, sizeof(applied), cudaMemcpyDeviceToHost, s)))
        return done(cuda_fail(e, "read applied"));
    if (int rc = classify_rows(g, s)) return done(rc);
    if (int rc = build_tables(g, s)) return done(rc);
    if ((e = cudaStreamSynchronize(s))) return done(cuda_fail(e, "removals"));
    if (applied_out) *applied_out = (int64_t)applied;
    return done(RS_OK);
}

// ---------------------------------------------------------------------------
// target-community subset: drop every edge with an endpoint outside the targets
// ---------------------------------------------------------------------------
__global__ void mark_nontarget_kernel(const int64_t *off, const int32_t *col, const int32_t *lab, const int32_t *map,
                                      int64_t n, uint32_t *dead) {
    int lane = threadIdx.x & 31;
    int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = w; v < n; v += nw) {
        bool out_v = map[lab[v]] < 0;
        for (int64_t e = off[v] + lane; e < off[v + 1]; e += 32)
            if (out_v || map[lab[col[e]]] < 0) mark_dead(dead, e);
    }
}
__global__ void relabel_kernel(int32_t *lab, const int32_t *map, int64_t n) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) { int32_t m = map[lab[v]]; lab[v] = m >= 0 ? m : 0; }
}

extern "C" rs_status rs_target_subset(const rs_graph *g, const int32_t *targets, int32_t n_targets, void *stream,
                                      rs_graph **out) {
    cudaStream_t s = as_stream(stream);
    if (!g || !targets || !out || n_targets < 1) return (rs_status)fail(RS_EINVAL, "rs_target_subset: bad arguments");
    if (g->n_graphs != 1) return (rs_status)fail(RS_EINVAL, "rs_target_subset: not for batches");
    std::vector<int32_t> map(std::max(g->k, 1), -1);
    for (int32_t i = 0; i < n_targets; ++i) {
        if (targets[i] < 0 || targets[i] >= g->k) return (rs_status)fail(RS_EINVAL, "rs_target_subset: target outside [0, k)");
        if (map[targets[i]] >= 0) return (rs_status)fail(RS_EINVAL, "rs_target_subset: repeated target");
        map[targets[i]] = i;
    }
    rs_graph *c = nullptr;
    if (rs_status st = rs_clone_graph(g, &c, stream)) return st;
    auto bail = [&](int rc) { free_graph(c); return (rs_status)rc; };
    int32_t *d_map = nullptr;
    int64_t n = c->n;
    cudaError_t e = dmalloc(&d_map, map.size());
    if (!e) e = cudaMemcpyAsync(d_map, map.data(), map.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s);
    if (!e && c->nnz) e = cudaMemsetAsync(c->dead, 0, 4 * ((c->nnz + 31) / 32), s);
    if (!e && n > 0) {
        int grid = grid_for(n * 32, kThreads, 16);
        mark_nontarget_kernel<<<grid, kThreads, 0, s>>>(c->off, c->col, c->lab, d_map, n, (uint32_t *)c->dead);
        e = cudaGetLastError();
        if (!e) {
            alive_degree_kernel<<<grid, kThreads, 0, s>>>(c->off, (uint32_t *)c->dead, n, c->off_alt);
            e = cudaGetLastError();
        }
        if (!e) {
            if (int rc = inclusive_scan_i64(c->off_alt + 1, n, c->scan_tmp, s)) { pool_free(d_map); return bail(rc); }
            compact_rows_kernel<<<grid, kThreads, 0, s>>>(c->off, c->col, (uint32_t *)c->dead, n, c->off_alt, c->col_alt);
            e = cudaGetLastError();
        }
        if (!e) {
            std::swap(c->off, c->off_alt);
            std::swap(c->col, c->col_alt);
            relabel_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(c->lab, d_map, n);
            e = cudaGetLastError();
        }
    }
    if (!e) e = cudaStreamSynchronize(s);
    pool_free(d_map);
    if (e) return bail(cuda_fail(e, "rs_target_subset"));
    c->k = n_targets;
    if (int rc = classify_rows(c, s)) return bail(rc);
    if (int rc = build_tables(c, s)) return bail(rc);
    if ((e = cudaStreamSynchronize(s))) return bail(cuda_fail(e, "rs_target_subset"));
    *out = c;
    return RS_OK;
}

// ---------------------------------------------------------------------------
// interaction table (sorted per row): labels of each row are sorted in place
// in a scratch copy, then run-length encoded
// ---------------------------------------------------------------------------
__global__ void gather_labels_kernel(const int32_t *col, const int32_t *lab, int64_t nnz, int32_t *out) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < nnz) out[e] = lab[col[e]];
}

// sort each row segment of `a` ascending: warps for rows <= 32, CTAs otherwise
__global__ void sort_small_rows_kernel(const int64_t *off, int64_t n, int32_t *a) {
    int lane = threadIdx.x & 31;
    int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = w; v < n; v += nw) {
        int64_t b = off[v];
        int d = (int)(off[v + 1] - b);
        if (d > 32 || d < 2) continue;
        int32_t x = lane < d ? a[b + lane] : 0x7FFFFFFF;
        for (int size = 2; size <= 32; size <<= 1)
            for (int st = size >> 1; st; st >>= 1) {
                int32_t y = __shfl_xor_sync(0xFFFFFFFFu, x, st);
                bool up = ((lane & size) == 0);
                bool lower = (lane & st) == 0;
                x = (lower == up) ? min(x, y) : max(x, y);
            }
        if (lane < d) a[b + lane] = x;
    }
}

__global__ void sort_large_rows_kernel(const int64_t *off, int64_t n, int32_t *a) {
    for (int64_t v = blockIdx.x; v < n; v += gridDim.x) {
        int64_t b = off[v];
        int64_t d = off[v + 1] - b;
        if (d <= 32) continue;
        int64_t P = 1;
        while (P < d) P <<= 1;
        int32_t *s = a + b;
        for (int64_t size = 2; size <= P; size <<= 1) {
            // mirror step, then half-cleaners; the smaller key moves to the lower index
            for (int64_t st = size >> 1; st; st >>= 1) {
                for (int64_t i = threadIdx.x; i < P / 2; i += blockDim.x) {
                    int64_t lo, hi;
                    if (st == (size >> 1)) {
                        int64_t blk = i / st, off_in = i % st;
                        lo = blk * size + off_in;
                        hi = blk * size + size - 1 - off_in;
                    } else {
                        lo = (i / st) * 2 * st + (i % st);
                        hi = lo + st;
                    }
                    if (hi < d && s[lo] > s[hi]) { int32_t t = s[lo]; s[lo] = s[hi]; s[hi] = t; }
                }
                __syncthreads();
            }
        }
    }
}

__global__ void count_runs_kernel(const int64_t *off, const int32_t *a, int64_t n, int64_t *cnt) {
    int lane = threadIdx.x & 31;
    int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = w; v < n; v += nw) {
        int64_t c = 0;
        for (int64_t e = off[v] + lane; e < off[v + 1]; e += 32) c += (e == off[v] || a[e] != a[e - 1]);
        for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
        if (lane == 0) cnt[v + 1] = c;
        if (v == 0 && lane == 0) cnt[0] = 0;
    }
}

// rows in the caller's order: internal row v lands at rp[perm[v]] (perm null: no reorder)
__global__ void emit_runs_kernel(const int64_t *off, const int32_t *a, int64_t n, const int64_t *rp,
                                 const int32_t *perm, int32_t *comm, int32_t *count) {
    int lane = threadIdx.x & 31;
    int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = w; v < n; v += nw) {
        int64_t out = rp[perm ? perm[v] : v];
        int64_t end = off[v + 1];
        for (int64_t base = off[v]; base < end; base += 32) {
            int64_t e = base + lane;
            bool head = e < end && (e == off[v] || a[e] != a[e - 1]);
            unsigned m = __ballot_sync(0xFFFFFFFFu, head);
            if (head) {
                int64_t j = e + 1;
                while (j < end && a[j] == a[e]) ++j;
                int64_t slot = out + __popc(m & ((1u << lane) - 1));
                comm[slot] = a[e];
                count[slot] = (int32_t)(j - e);
            }
            out += __popc(m);
        }
    }
}

__global__ void permute_counts_kernel(const int64_t *cnt_internal, const int32_t *perm, int64_t n, int64_t *cnt) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v == 0) cnt[0] = 0;
    if (v < n) cnt[(int64_t)perm[v] + 1] = cnt_internal[v + 1];
}

// ---------------------------------------------------------------------------
// RS_REORDER: internal ids by (community, degree descending, the caller's id).  The
// permutation is a host counting sort (two stable passes); the CSR is rebuilt on the
// device: degrees and rows gathered through the permutation, columns renamed, rows
// sorted again, labels gathered.
// ---------------------------------------------------------------------------
__global__ void reorder_degrees_kernel(const int64_t *off, const int32_t *perm, int64_t n, int64_t *deg1) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) deg1[-1] = 0;
    if (i < n) deg1[i] = off[(int64_t)perm[i] + 1] - off[perm[i]];
}
__global__ void reorder_rows_kernel(const int64_t *off, const int32_t *col, const int32_t *perm, const int32_t *iperm,
                                    int64_t n, const int64_t *noff, int32_t *ncol) {
    int lane = threadIdx.x & 31;
    int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = w; i < n; i += nw) {
        int64_t src = off[perm[i]], d = off[(int64_t)perm[i] + 1] - src, dst = noff[i];
        for (int64_t j = lane; j < d; j += 32) ncol[dst + j] = iperm[col[src + j]];
    }
}
__global__ void reorder_labels_kernel(const int32_t *lab, const int32_t *perm, int64_t n, int32_t *nlab) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) nlab[i] = lab[perm[i]];
}

static int reorder_graph(rs_graph *g, cudaStream_t s) {
    const int64_t n = g->n;
    if (n == 0) return 0;
    std::vector<int64_t> off(n + 1);
    std::vector<int32_t> lab(n);
    RS_CUDA_TRY(cudaMemcpyAsync(off.data(), g->off, (n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    RS_CUDA_TRY(cudaMemcpyAsync(lab.data(), g->lab, n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    RS_CUDA_TRY(cudaStreamSynchronize(s));
    int64_t dmax = 0;
    for (int64_t v = 0; v < n; ++v) dmax = std::max(dmax, off[v + 1] - off[v]);
    // pass 1: stable by degree, largest first; pass 2: stable by community
    std::vector<int64_t> cnt(std::max<int64_t>(dmax, g->k) + 2, 0);
    std::vector<int32_t> by_deg(n), order(n);
    for (int64_t v = 0; v < n; ++v) cnt[dmax - (off[v + 1] - off[v]) + 1]++;
    for (int64_t b = 1; b <= dmax + 1; ++b) cnt[b] += cnt[b - 1];
    for (int64_t v = 0; v < n; ++v) by_deg[cnt[dmax - (off[v + 1] - off[v])]++] = (int32_t)v;
    std::fill(cnt.begin(), cnt.end(), 0);
    for (int64_t v = 0; v < n; ++v) cnt[(int64_t)lab[v] + 1]++;
    for (int64_t c = 1; c <= g->k; ++c) cnt[c] += cnt[c - 1];
    for (int64_t i = 0; i < n; ++i) order[cnt[lab[by_deg[i]]]++] = by_deg[i];
    g->iperm.assign(n, 0);
    for (int64_t i = 0; i < n; ++i) g->iperm[order[i]] = (int32_t)i;
    int32_t *d_iperm = nullptr;
    RS_CUDA_TRY(dmalloc(&g->perm, n));
    RS_CUDA_TRY(dmalloc(&d_iperm, n));
    cudaError_t e = cudaMemcpyAsync(g->perm, order.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, s);
    if (!e) e = cudaMemcpyAsync(d_iperm, g->iperm.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, s);
    // new offsets in off_alt, new rows in col_alt, new labels through the removed flags' storage
    if (!e) {
        reorder_degrees_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(g->off, g->perm, n, g->off_alt + 1);
        e = cudaGetLastError();
    }
    if (!e) {
        if (int rc = inclusive_scan_i64(g->off_alt + 1, n, g->scan_tmp, s)) { pool_free(d_iperm); return rc; }
        int grid = grid_for(n * 32, kThreads, 16);
        reorder_rows_kernel<<<grid, kThreads, 0, s>>>(g->off, g->col, g->perm, d_iperm, n, g->off_alt, g->col_alt);
        e = cudaGetLastError();
        if (!e) {
            sort_small_rows_kernel<<<grid, kThreads, 0, s>>>(g->off_alt, n, g->col_alt);
            e = cudaGetLastError();
        }
        if (!e) {
            sort_large_rows_kernel<<<grid_for(n, 1, 8), 512, 0, s>>>(g->off_alt, n, g->col_alt);
            e = cudaGetLastError();
        }
        if (!e) {
            reorder_labels_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(g->lab, g->perm, n, (int32_t *)g->removed);
            e = cudaGetLastError();
        }
        if (!e) e = cudaMemcpyAsync(g->lab, g->removed, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
        if (!e) e = cudaMemsetAsync(g->removed, 0, 4 * n, s);
        if (!e) e = cudaStreamSynchronize(s);
    }
    pool_free(d_iperm);
    if (e) return cuda_fail(e, "RS_REORDER");
    std::swap(g->off, g->off_alt);
    std::swap(g->col, g->col_alt);
    return 0;
}

int rs::interaction_table(rs_graph *g, int64_t *t_out, int64_t *row_ptr, int32_t *comm, int32_t *count,
                          cudaStream_t s) {
    int64_t n = g->n, nnz_cur = 0;
    RS_CUDA_TRY(cudaMemcpyAsync(&nnz_cur, g->off + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    RS_CUDA_TRY(cudaStreamSynchronize(s));
    int32_t *a = g->col_alt;           // scratch: labels of every CSR entry
    int64_t *rp = g->off_alt;          // scratch: row pointer
    if (nnz_cur) {
        gather_labels_kernel<<<(unsigned)((nnz_cur + 255) / 256), 256, 0, s>>>(g->col, g->lab, nnz_cur, a);
        RS_CUDA_TRY(cudaGetLastError());
    }
    if (n > 0) {
        int grid = grid_for(n * 32, kThreads, 16);
        sort_small_rows_kernel<<<grid, kThreads, 0, s>>>(g->off, n, a);
        RS_CUDA_TRY(cudaGetLastError());
        sort_large_rows_kernel<<<grid_for(n, 1, 8), 512, 0, s>>>(g->off, n, a);
        RS_CUDA_TRY(cudaGetLastError());
        if (g->perm) {
            // counts per internal row, then moved to the caller's row order before the scan
            count_runs_kernel<<<grid, kThreads, 0, s>>>(g->off, a, n, g->xoff);
            RS_CUDA_TRY(cudaGetLastError());
            permute_counts_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(g->xoff, g->perm, n, rp);
        } else {
            count_runs_kernel<<<grid, kThreads, 0, s>>>(g->off, a, n, rp);
        }
        RS_CUDA_TRY(cudaGetLastError());
        if (int rc = inclusive_scan_i64(rp + 1, n, g->scan_tmp, s)) return rc;
    } else {
        RS_CUDA_TRY(cudaMemsetAsync(rp, 0, sizeof(int64_t), s));
    }
    int64_t t = 0;
    RS_CUDA_TRY(cudaMemcpyAsync(&t, rp + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    RS_CUDA_TRY(cudaStreamSynchronize(s));
    if (row_ptr) RS_CUDA_TRY(cudaMemcpyAsync(row_ptr, rp, (n + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    if (comm && count && n > 0) {
        emit_runs_kernel<<<grid_for(n * 32, kThreads, 16), kThreads, 0, s>>>(g->off, a, n, rp, g->perm, comm,
                                                                              count);
        RS_CUDA_TRY(cudaGetLastError());
    }
    RS_CUDA_TRY(cudaStreamSynchronize(s));
    *t_out = t;
    return 0;
}

extern "C" rs_status rs_get_interaction(rs_graph *g, int64_t *t_out, int64_t *row_ptr, int32_t *comm,
                                        int32_t *count, void *stream) {
    if (!g || !t_out) return (rs_status)fail(RS_EINVAL, "rs_get_interaction: NULL argument");
    if ((comm == nullptr) != (count == nullptr))
        return (rs_status)fail(RS_EINVAL, "rs_get_interaction: comm and count go together");
    int64_t t = 0;
    int rc = interaction_table(g, &t, row_ptr, comm, count, as_stream(stream));
    if (rc) return (rs_status)rc;
    *t_out = t;
    return RS_OK;
}

extern "C" rs_status rs_score(rs_graph *g, double *scores, double *omega_max_out, void *stream) {
    cudaStream_t s = as_stream(stream);
    if (!g || (!scores && g->n > 0)) return (rs_status)fail(RS_EINVAL, "rs_score: NULL argument");
    int rc = score_graph(g, scores, s);
    if (rc) return (rs_status)rc;
    if (omega_max_out) {
        unsigned long long bits = 0;
        int32_t flags = 0;
        if (cudaError_t e = cudaMemcpyAsync(&bits, g->wmax_bits, sizeof(bits), cudaMemcpyDeviceToHost, s))
            return (rs_status)cuda_fail(e, "read w_max");
        if (g->n > 0)
            if (cudaError_t e = cudaMemcpyAsync(&flags, g->d_flag + 4, sizeof(flags), cudaMemcpyDeviceToHost, s))
                return (rs_status)cuda_fail(e, "read device flags");
        if (cudaError_t e = cudaStreamSynchronize(s)) return (rs_status)cuda_fail(e, "rs_score");
        if (flags & 32)
            return (rs_status)fail(RS_ETIMEOUT, "rs_score: a bounded wait of the G_x offset scan ran out "
                                                "(the offsets were summed directly instead)");
        double w;
        memcpy(&w, &bits, sizeof(w));
        *omega_max_out = w;
    }
    return RS_OK;
}

extern "C" rs_status rs_test_gx_stall(rs_graph *g, int64_t tile, int64_t spin_limit) {
    if (!g || spin_limit < 1) return (rs_status)fail(RS_EINVAL, "rs_test_gx_stall: bad arguments");
    g->gx_withhold = tile < 0 ? -1 : tile;
    g->gx_spin = tile < 0 ? (1l << 24) : (long)spin_limit;
    g->version++;                                  // captured steps hold the old launch arguments
    return RS_OK;
}

__global__ void gather_awcc_kernel(const int32_t *nodes, int64_t m, const int32_t *Lall, const int64_t *off,
                                   int32_t *out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) {
        int32_t v = nodes[i];
        out[2 * i] = Lall[v];
        out[2 * i + 1] = (int32_t)(off[v + 1] - off[v]);
    }
}

extern "C" rs_status rs_awcc(rs_graph *g, const int32_t *nodes, int64_t m, const int64_t *deg_ref, double *awcc_out,
                             int32_t *zeta_out, void *stream) {
    cudaStream_t s = as_stream(stream);
    if (!g || (m > 0 && !nodes) || m < 0 || !awcc_out) return (rs_status)fail(RS_EINVAL, "rs_awcc: bad arguments");
    if (g->scored_version != g->version)
        return (rs_status)fail(RS_EINVAL, "rs_awcc: call rs_score after the last change of the graph");
    for (int64_t i = 0; i < m; ++i)
        if (nodes[i] < 0 || nodes[i] >= g->n) return (rs_status)fail(RS_EINVAL, "rs_awcc: node id out of range");
    if (m == 0) { *awcc_out = 0.0; return RS_OK; }
    std::vector<int32_t> mapped;
    if (g->perm) {                               // the caller's ids -> internal ones
        mapped.resize(m);
        for (int64_t i = 0; i < m; ++i) mapped[i] = g->iperm[nodes[i]];
        nodes = mapped.data();
    }
    int32_t *d_buf = nullptr;
    std::vector<int32_t> h(2 * (size_t)m);
    cudaError_t e = dmalloc(&d_buf, 3 * (size_t)m);
    if (!e) e = cudaMemcpyAsync(d_buf, nodes, m * sizeof(int32_t), cudaMemcpyHostToDevice, s);
    if (!e) {
        gather_awcc_kernel<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(d_buf, m, g->Lall, g->off, d_buf + m);
        e = cudaGetLastError();
    }
    if (!e) e = cudaMemcpyAsync(h.data(), d_buf + m, 2 * m * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);
    pool_free(d_buf);
    if (e) return (rs_status)cuda_fail(e, "rs_awcc");
    double sum = 0.0;
    for (int64_t i = 0; i < m; ++i) {
        int64_t d = deg_ref ? deg_ref[i] : h[2 * i + 1];
        int32_t z = h[2 * i + 1] > 0 ? h[2 * i] : 0;       // an isolated node reaches no community
        if (zeta_out) zeta_out[i] = z;
        if (d > 0) sum += (double)z / (double)d;
    }
    *awcc_out = sum / (double)m;
    return RS_OK;
}

extern "C" rs_status rs_device_errors(rs_graph *g, int32_t *flags_out, void *stream) {
    if (!g || !flags_out) return (rs_status)fail(RS_EINVAL, "rs_device_errors: NULL argument");
    cudaStream_t s = as_stream(stream);
    int32_t f = 0;
    if (g->n > 0) {
        if (cudaError_t e = cudaMemcpyAsync(&f, g->d_flag + 4, sizeof(int32_t), cudaMemcpyDeviceToHost, s))
            return (rs_status)cuda_fail(e, "rs_device_errors");
        if (cudaError_t e = cudaStreamSynchronize(s)) return (rs_status)cuda_fail(e, "rs_device_errors");
    }
    *flags_out = f;
    return RS_OK;
}

extern "C" rs_status rs_topk(rs_graph *g, const double *scores, int32_t k, int32_t *ids_out,
                             double *scores_out, void *stream) {
    if (!g || !scores || !ids_out) return (rs_status)fail(RS_EINVAL, "rs_topk: NULL argument");
    if (k < 1 || (int64_t)k > g->n || k > 16384)
        return (rs_status)fail(RS_EINVAL, "rs_topk: k must be in [1, min(n, 16384)]");
    return (rs_status)topk_scores(g, scores, g->n, k, ids_out, scores_out, as_stream(stream));
}
