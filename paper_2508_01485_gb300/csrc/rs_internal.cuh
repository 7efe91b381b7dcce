// rs_internal.cuh -- device graph layout and kernels shared by the library's
// translation units.  Not part of the public ABI (include/rs.h).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "rs.h"
#include "rs_numeric.cuh"

namespace rs {

// Row classes by degree d and by the hash-table size cap = pow2 >= 2 min(d, k)
// (k bounds the number of distinct neighbour communities).  The split points
// are launch parameters (rs_tuning in rs.h); these are their upper limits,
// which size the shared-memory tables:
//   small: d <= small_max (<= kSmallMax), tiles of 32 rows per warp;
//   mid:   cap <= warp_cap (<= kWarpCap), one warp per row, a per-warp
//          shared-memory table;
//   large: cap <= cta_cap (<= kMidCap), one CTA per row, a per-CTA
//          shared-memory table;
//   hub:   larger rows; a hash table in global memory, rows split into chunks
//          of hub_chunk neighbours processed by separate CTAs and merged by
//          atomics into the row's table.
constexpr int kSmallMax = 32;
constexpr int kWarpCap = 512;
constexpr int kMidCap = 2048;
constexpr int32_t kEmpty = -1;

// per-node record written by the first pass and gathered by the second
struct __align__(16) NodeRec {
    uint64_t s_fix;   // s_v = w_v(C(v))^(1/3) in 2^-52 fixed point
    int32_t label;    // C(v)
    int32_t dx;       // cross-community degree (neighbours with another label)
};

// per-hub state (global hash table and row aggregates)
// the per-slot passes over the hubs' tables (their sums, column maxima and sigma) take a
// hub's table in ranges of this many slots, so that a large hub's table is spread over
// CTAs instead of walked by one
constexpr int32_t kHubSlotRange = 4096;
struct HubInfo {
    int32_t row;
    int32_t cap;          // table slots (power of two)
    int64_t tab;          // first slot in the hub table arrays
    int32_t first_item;   // first chunk item of this hub
    int32_t n_items;
    int64_t ent;          // first of its entries in hslot (the hubs' entries, hub by hub)
};
struct __align__(16) HubAgg {
    u128 X;               // sum over foreign groups of f LG[f] (own group added later)
    uint32_t L;           // foreign groups
    uint32_t own;         // neighbours in C(row)
    uint32_t pad[2];
};

// Graphs of a batch (many independent graphs packed into one CSR): each node's
// graph, each graph's number of communities and its own w_max slot.  For a
// single graph gid is null and k / wmax[0] apply to every node.
struct Batch {
    const int32_t *gid;
    const int32_t *gk;
    int32_t k;
    unsigned long long *wmax;
};
__device__ __forceinline__ int32_t graph_of(const Batch &B, int32_t v) { return B.gid ? B.gid[v] : 0; }
__device__ __forceinline__ int32_t k_of(const Batch &B, int32_t gi) { return B.gid ? B.gk[gi] : B.k; }

// row aggregates kept from P1 for P2: X = sum_c f_c LG[f_c] (exact) and the
// number of distinct neighbour communities L
struct __align__(8) RowSum {
    uint64_t xlo, xhi;
    uint32_t L, pad;
};

inline uint32_t pow2_at_least(uint64_t x) {
    uint32_t c = 1;
    while (c < x) c <<= 1;
    return c;
}

__device__ __forceinline__ uint32_t hash_label(int32_t c) { return (uint32_t)c * 0x9E3779B1u; }

// whether u is ordered after w for triangle orientation: (dx, id) ascending
__device__ __forceinline__ bool rank_after(int32_t dxu, int32_t u, int32_t dxw, int32_t w) {
    return dxu > dxw || (dxu == dxw && u > w);
}

}  // namespace rs

namespace rs {
// the launch parameters a new graph starts with (see rs_tuning in rs.h)
inline rs_tuning default_tuning_value() {
    rs_tuning t;
    t.small_max = kSmallMax;
    t.warp_cap = kWarpCap;
    t.cta_cap = kMidCap;
    t.hub_chunk = 4096;
    t.p2_cta_dx = kWarpCap / 2;
    t.p1_cta_threads = 256;
    t.p2_cta_threads = 1024;
    t.ctas_per_sm = 8;
    t.p3_mirror = 1;
    t.p1_stage = 0;
    t.rows_streams = -1;
    return t;
}
}  // namespace rs

struct rs_graph {
    int64_t n = 0, nnz = 0;
    int32_t k = 0, dmax = 0;               // k: communities (batch: the sum over its graphs)
    int32_t n_graphs = 1;                  // > 1 for a batch of packed graphs
    int32_t *gid = nullptr;                // batch: graph of each node
    int32_t *gk = nullptr;                 // batch: communities of each graph
    int64_t *gnode = nullptr;              // batch: first node of each graph (n_graphs + 1)
    double *winv = nullptr;                // 1 / w_max per graph (0 when w_max = 0)
    int device = 0;
    // CSR (int64 offsets) and labels; *_alt are the compaction targets of removals
    int64_t *off = nullptr, *off_alt = nullptr;
    int32_t *col = nullptr, *col_alt = nullptr;
    int32_t *lab = nullptr;
    uint8_t *removed = nullptr;       // n removed-node flags
    uint8_t *dead = nullptr;          // nnz edge marks used by removals
    // row classes
    int32_t *rows_small = nullptr, *rows_mid = nullptr, *rows_large = nullptr;
    int32_t *rows_sort = nullptr;        // scratch of the degree ordering of the mid and large rows
    int64_t n_small = 0, n_mid = 0, n_large = 0;
    int32_t large_cap = 0;            // largest table among large rows
    rs::HubInfo *hubs = nullptr;      // device copy
    int32_t *hub_items = nullptr;     // per chunk item: hub index
    int32_t *hub_item_chunk = nullptr;// per chunk item: chunk number within the hub
    int64_t n_hubs = 0, n_hub_items = 0, hub_slots = 0;
    int32_t *hub_sitem = nullptr;     // per slot-range item: hub index (a hub's table in ranges of
    int32_t *hub_srange = nullptr;    //   kHubSlotRange slots) and the range's number in the hub
    int64_t n_hub_sitems = 0;
    int32_t *hslot = nullptr;         // per hub entry: its community's table slot (-1: own community)
    int32_t *hkey = nullptr;          // hub hash tables
    uint32_t *hcnt = nullptr;
    unsigned long long *hq = nullptr; // 2 words per slot
    rs::df *hsig = nullptr;           // per slot sigma of the column
    rs::HubAgg *hagg = nullptr;
    int32_t *hitem_out = nullptr, *hitem_in = nullptr;  // per item G_x out / in counts
    // constant tables, sized dmax + 1
    uint64_t *LG = nullptr;           // round(log2(f) 2^58)
    double *RD = nullptr;             // 1 / (d (d - 1))
    // scoring workspace
    rs::NodeRec *rec = nullptr;
    unsigned long long *acc = nullptr;        // 2 words per node
    unsigned long long *wmax_bits = nullptr;  // double bits of w_max, one per graph
    int32_t *Lall = nullptr;                  // distinct neighbour communities per node
    rs::RowSum *rsum = nullptr;               // per-node aggregates from P1
    int32_t *cl_col = nullptr;                // cross lists: row v's cross neighbours at
    int32_t *cl_lab = nullptr;                //   [off[v], off[v] + dx(v)) (ids, labels)
    int64_t *xoff = nullptr;                  // G_x row offsets (n + 1)
    int32_t *xcol = nullptr;                  // G_x neighbours (capacity nnz + 8: whole 8-slot sectors)
    int32_t *xsk = nullptr;                   // first id of every 8-slot sector of xcol (nnz / 8 + 1)
    rs::df *xS = nullptr;                     // S(w -> u) = w_w(C(u))^(1/3)
    int32_t *xout = nullptr, *xin = nullptr;  // out / in counts per node
    int32_t *p2rows = nullptr;                // P2 row lists by cross degree (4 n), counted in p2cnt
    int32_t *p2cnt = nullptr;
    unsigned long long *wq = nullptr;         // per-pass row counters of the dynamically scheduled kernels
    int64_t *scan_tmp = nullptr;              // block sums for scans
    // top-k workspace
    uint32_t *tk_hist = nullptr;
    int32_t *tk_ctrl = nullptr;
    unsigned long long *tk_keys = nullptr;    // candidate (key, id) pairs
    int32_t *tk_ids = nullptr;
    int64_t tk_cap = 0;
    // misc
    int32_t *d_flag = nullptr;                // device error / scalar slot
    // launch accounting and optional per-kernel event timing
    int64_t launches = 0;
    bool prof_on = false;
    std::vector<cudaEvent_t> prof_ev;         // event pool (created on demand)
    std::vector<const char *> prof_name;      // per recorded event: kernel name, or nullptr (segment start)
    std::vector<char> prof_is_kernel;
    std::vector<int> prof_prev;               // index of the previous event on the same stream
    std::vector<cudaStream_t> prof_stream;
    size_t prof_used = 0;
    // auxiliary streams for independent row classes (fork / join by events)
    static constexpr int kAux = 6;
    cudaStream_t aux[kAux] = {};
    cudaEvent_t ev_fork = nullptr;
    cudaEvent_t ev_join[kAux] = {};
    // launch parameters and a counter bumped whenever buffers or row classes change
    rs::df *xR = nullptr;                     // p3_mirror: at out-slot (w -> u) the reverse value S(u -> w)
    int32_t *xtile = nullptr;                 // p3_mirror: node holding the first slot of each mirror tile
    int32_t *perm = nullptr;                  // RS_REORDER: internal id -> the caller's id (device)
    std::vector<int32_t> iperm;               // RS_REORDER: the caller's id -> internal id (host)
    rs_tuning tune = rs::default_tuning_value();
    uint64_t version = 0;
    bool alg2 = false;                        // RS_ALG2_COMPAT: |L| = L_all - 1 for every column
    bool strict = false;                      // RS_TRIAD_STRICT: no closed triad with C(v) = C(u)
    unsigned long long *sx = nullptr;         // strict: X(w, u) per CSR entry (2 words), else null
    uint64_t scored_version = ~0ull;          // version of the last rs_score (Lall and the scores are current)
    // bounded waits of the G_x offset scan: reads of a tile's word before giving up, and
    // a tile kept from publishing (-1: none; set only by rs_test_gx_stall)
    long gx_spin = 1l << 24;
    int64_t gx_withhold = -1;
};

namespace rs {

constexpr int kThreads = 256;
constexpr int kMirTile = 2048;               // G_x slots per tile of the mirror pass
constexpr int kGxTile = 4096;                // nodes per tile of the G_x offset scan
// P3: a node with more than kWinCap G_x out-neighbours is heavy, and its walk is cut into
// tasks of kHvBlock out-neighbours.  Every G_x edge has one tail, and a heavy node has
// d+ >= 129 out-neighbours, so its (d+ + 127) / 128 tasks are at most d+ 256 / (128 129),
// and all tasks together at most 2 m_x / 129 <= nnz / 129 (m_x <= nnz / 2).
constexpr int kWinCap = 128, kHvBlock = 128;
static_assert(kWinCap == 128 && kHvBlock == 128, "hv_cap's bound is worked out for these values");
inline int64_t hv_cap(int64_t nnz) { return nnz / 129 + 1; }
// words of rs_graph::wq: 0..7 the row and group counters of the row kernels, 8 the
// ticket of the G_x offset scan, 9 and 10 the append and claim counters of P3's
// heavy-node task list, 16.. the scan's tile words (all these zeroed before every
// scoring pass: wq_hv_word words); then the task list, hv_cap words (node << 32 | block),
// each written before it is read
constexpr int kWqGxTicket = 8, kWqHvCount = 9, kWqHvNext = 10, kWqGxStatus = 16;
inline int64_t wq_hv_word(int64_t n) { return kWqGxStatus + (n + kGxTile - 1) / kGxTile + 1; }
inline int64_t wq_words(int64_t n, int64_t nnz) { return wq_hv_word(n) + hv_cap(nnz); }

// error reporting (rs_api.cu): returns the status after recording the message
int fail(int status, const std::string &msg);
int cuda_fail(cudaError_t e, const char *where);
#define RS_CUDA_TRY(expr)                                            \
    do {                                                             \
        cudaError_t _e = (expr);                                     \
        if (_e != cudaSuccess) return ::rs::cuda_fail(_e, #expr);    \
    } while (0)

// in-place inclusive scan of a[0..m) (int64), tmp >= scan_tmp_words(m) words;
// adds the number of kernels launched to *launches when given
int64_t scan_tmp_words(int64_t m);
int inclusive_scan_i64(int64_t *a, int64_t m, int64_t *tmp, cudaStream_t s, int64_t *launches = nullptr);

// launch accounting: count a kernel launch (or record a non-kernel operation)
// and, when profiling is on, record an event after it on the stream
int set_mirror_buffer(rs_graph *g);
// Device memory of the library's graphs and workspaces comes from a stream-ordered
// pool per device that keeps up to kPoolKeep bytes of freed blocks for the next
// graph: cudaMalloc / cudaFree of a 1M-node graph's ~30 buffers take about 1.0 /
// 1.4 ms, the warm pool 0.03 / 0.015 ms.  pool_malloc returns memory usable on any
// stream; pool_free synchronises the device first, as cudaFree does.
cudaError_t pool_malloc(void **p, size_t bytes);
cudaError_t pool_free(void *p);
cudaError_t pool_free_many(void *const *p, size_t n);   // one device synchronisation for all
void prof_begin(rs_graph *g, cudaStream_t s);
void prof_mark(rs_graph *g, cudaStream_t s, const char *name, bool is_kernel);
// make the auxiliary streams wait for s / make s wait for the first `used` auxiliary streams
int fork_aux(rs_graph *g, cudaStream_t s);
int join_aux(rs_graph *g, cudaStream_t s, int used);
#define RS_LAUNCHED(g, s, name)                        \
    do {                                               \
        RS_CUDA_TRY(cudaGetLastError());               \
        ::rs::prof_mark((g), (s), (name), true);       \
    } while (0)

// grid size for grid-stride kernels: at most `cap_per_sm` CTAs per SM
int grid_for(int64_t items, int per_block, int cap_per_sm);

// scoring (rs_score.cu) and ranking (rs_topk.cu); return an rs_status value
int score_graph(rs_graph *g, double *scores, cudaStream_t s);
int topk_scores(rs_graph *g, const double *scores, int64_t n, int32_t k, int32_t *ids,
                double *out_scores, cudaStream_t s);
int interaction_table(rs_graph *g, int64_t *t_out, int64_t *row_ptr, int32_t *comm,
                      int32_t *count, cudaStream_t s);
// one-time kernel attributes / launch shapes and workspaces, so that a step can
// be captured into a CUDA graph without allocating or configuring inside it
int prepare_score_kernels();
int topk_prepare(rs_graph *g, int64_t n);
// re-split g's rows by g->tune (rs_api.cu); synchronises s
int reclassify(rs_graph *g, cudaStream_t s);

}  // namespace rs
