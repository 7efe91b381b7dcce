/*
 * rs.h -- C ABI of the GB300 Robust Spanning Index library (librs.so).
 *
 * Robust spanners (arXiv 2508.01485): every node u of an undirected graph
 * G = (V, E) whose nodes carry non-overlapping community labels C(u) gets the
 * Robust Spanning Index
 *
 *   R(u) = 1/(d(u)(d(u)-1)) * sum_{w in N(u), v in N(w) : 1(u,w,v)}
 *          (w_v(u) w_w(v) w_w(u))^(1/3)                   (Sec. III-B, Eq. RSI)
 *
 * with weights w_v(u) = H(L(u,v)) |L(u,v)| from the entropy of v's neighbour
 * communities other than C(u) (Eq. cont, entropy, weight), normalised by the
 * largest weight w_max (Alg. 1 Step 2), and the triad indicator 1(u,w,v)
 * (Sec. III-A: Type-I closed triads across three communities, Type-II open
 * triads closed by an "augmented edge" inside C(u)).  The library computes
 * the per-node community counts (the paper's interaction_matrix, Sec. V-A),
 * the weights, all scores and a top-K ranking (Alg. 1 Step 4) on one GPU.
 *
 * Conventions shared by every call:
 *  - All device work is enqueued on `stream` (a cudaStream_t passed as void*;
 *    NULL is the legacy default stream).  Calls return once the work is
 *    enqueued, except where a host out-parameter must be filled, which
 *    synchronises `stream`.
 *  - Inputs are copied; the caller may free or reuse them once the call's
 *    stream work has completed.  Outputs are caller-allocated.
 *  - Out-parameters are written only when the call returns RS_OK.
 *  - On failure the call returns a non-zero rs_status and rs_last_error()
 *    gives a message (thread-local, valid until the next call on the thread).
 *  - The library owns the device memory behind an rs_graph.  Calls on one
 *    rs_graph must not run concurrently (they share its workspace).
 *  - Node ids are 0..n-1 (int32); community labels are 0..k-1 (int32).
 */
#ifndef RS_H_
#define RS_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rs_graph rs_graph;

typedef enum {
    RS_OK = 0,
    RS_EINVAL = 1,    /* invalid argument or invalid graph */
    RS_ENOMEM = 2,    /* device or host allocation failed */
    RS_ECUDA = 3,     /* a CUDA call failed (message holds the CUDA error) */
    RS_ETIMEOUT = 4,  /* a bounded device wait gave up */
    RS_EBUDGET = 5    /* a request does not fit the memory budget */
} rs_status;

/* rs_build_graph flags */
#define RS_VALIDATE 1u      /* check the CSR on the device (see rs_build_graph) */
#define RS_ALG2_COMPAT 2u   /* weights with |L| = L_all - 1 for every column, as Alg. 2
                               (compute_weights) takes it, instead of the definition's number of
                               communities left (Eq. weight); differs only for communities
                               absent from N(v): w_max and s of nodes without own-community
                               neighbours */
#define RS_REORDER 8u      /* renumber the nodes internally by community, then degree (largest
                               first), for locality; every id the caller sees or passes -- scores,
                               top-K ids, interaction rows, removals, AWCC nodes -- stays the
                               caller's own.  Not for rs_build_batch; graphs built with it are not
                               served by rs_server */
#define RS_TRIAD_STRICT 4u  /* the strict reading of the triad types (Sec. III-A): a closed
                               triangle (u, w, v) with C(v) = C(u) != C(w) is not a triad for
                               u (by default it counts once, as an augmented-edge triad).
                               Needs 16 bytes per CSR entry more; resident graphs served by
                               rs_server take the full path with it */

/*
 * rs_build_graph -- load a community-labelled graph (Sec. II; CSR of Sec. V-A).
 *
 *   n, nnz          number of nodes and of CSR entries (2 x undirected edges);
 *                   0 <= n < 2^31, 0 <= nnz < 2^40, max degree < 2^24.
 *   row_offsets     n+1 offsets, int64 if offsets_are_i64 else int32;
 *                   row_offsets[0] = 0, row_offsets[n] = nnz.
 *   cols            nnz int32 neighbour ids; row v is cols[off[v] .. off[v+1]).
 *   labels          n int32 community ids in [0, num_communities).
 *   num_communities k >= 1.
 *   inputs_on_device  non-zero: the three arrays are device pointers, else
 *                   host pointers (copied with cudaMemcpyAsync on `stream`).
 *   flags           RS_VALIDATE: verify on the device that the graph is simple
 *                   and undirected -- offsets non-decreasing, ids in range,
 *                   every row strictly ascending (sorted, no duplicates), no
 *                   self-loops, every edge present in both directions -- and
 *                   that labels lie in [0, k).  Returns RS_EINVAL otherwise.
 *                   Symmetry is checked by a keyed 64-bit hash sum of the
 *                   directed edges against their reverses, which cancels
 *                   exactly for a symmetric graph; an asymmetric one passes
 *                   only by a 2^-64-scale coincidence.
 *                   Without the flag the input must already satisfy this.
 *   out             receives the new graph (free with rs_free_graph).
 * Synchronises `stream` (the degree profile is read back to size workspaces).
 */
rs_status rs_build_graph(int64_t n, int64_t nnz, const void *row_offsets, int offsets_are_i64,
                         const int32_t *cols, const int32_t *labels, int32_t num_communities,
                         int inputs_on_device, uint32_t flags, void *stream, rs_graph **out);

/*
 * rs_build_batch -- many independent community-labelled graphs packed into one
 * CSR and scored together: every graph keeps its own labels, its own w_max
 * and therefore its own scores, exactly as if built alone.
 *
 *   n_graphs              >= 1.
 *   graph_node_offsets    host int64[n_graphs+1]: graph i owns nodes
 *                         [graph_node_offsets[i], graph_node_offsets[i+1]); starts at 0.
 *   graph_k               host int32[n_graphs]: communities of each graph (>= 1);
 *                         their sum must stay below 2^31.
 *   nnz, row_offsets, offsets_are_i64, cols, inputs_on_device, flags, stream
 *                         as rs_build_graph, over the packed node ids; every
 *                         neighbour lies in its row's graph.
 *   labels                int32[n]: each node's label local to its graph, in [0, k_i).
 * RS_VALIDATE adds the per-graph checks (neighbours inside the graph, labels
 * below its k).  rs_score then normalises each node by its own graph's w_max;
 * rs_get_interaction reports community ids offset by the sum of the k of the
 * graphs before (graph i's community c is reported as k_0 + .. + k_{i-1} + c).
 */
rs_status rs_build_batch(int32_t n_graphs, const int64_t *graph_node_offsets, const int32_t *graph_k, int64_t nnz,
                         const void *row_offsets, int offsets_are_i64, const int32_t *cols, const int32_t *labels,
                         int inputs_on_device, uint32_t flags, void *stream, rs_graph **out);

/* rs_batch_omega_max -- w_max of each graph of the last rs_score call, to host
 * double[n_graphs] (one entry for a single graph).  Synchronises `stream`. */
rs_status rs_batch_omega_max(rs_graph *g, double *wmax_out, void *stream);

/*
 * rs_score -- Robust Spanning Index of every node (Alg. 1 Steps 1-3, Eq. RSI).
 *
 *   scores          device buffer of n doubles, written with R(u) in node-id
 *                   order.  R(u) = 0 when d(u) < 2 or w_max = 0.
 *   omega_max_out   optional host pointer: receives w_max, the largest
 *                   un-normalised weight w_v(c) over all nodes v and all
 *                   communities c in [0, k) (including communities absent from
 *                   N(v)).  Passing it synchronises `stream`.
 * Scores agree with the fp64 definition to ~1e-13 relative; they are
 * bit-identical from run to run (all sums are exact fixed-point).
 */
rs_status rs_score(rs_graph *g, double *scores, double *omega_max_out, void *stream);
/*
 * Every wait inside rs_score's kernels is bounded.  When rs_score synchronises
 * (omega_max_out given) and a wait of this call ran out, it returns RS_ETIMEOUT
 * (the scores are still written: the wait's data is then recomputed directly);
 * without omega_max_out, rs_device_errors reports it (bit 32).
 */

/*
 * rs_get_interaction -- the per-node community counts f_v(c) (Sec. V-A,
 * interaction_matrix, stored sparsely).
 *
 *   t_out     host: number of (node, community) entries with f_v(c) > 0.
 *   row_ptr   device int64[n+1] or NULL; comm / count device int32[t] or NULL.
 * Rows are in node order; within a row, communities ascend.  Call with NULL
 * arrays to learn t.  Synchronises `stream`.
 */
rs_status rs_get_interaction(rs_graph *g, int64_t *t_out, int64_t *row_ptr, int32_t *comm,
                             int32_t *count, void *stream);

/*
 * rs_topk -- the K best nodes by (score descending, node id ascending)
 * (Alg. 1 Step 4).
 *
 *   scores      device double[n] (normally rs_score's output); every value
 *               must be >= 0 (not NaN).
 *   k           1 <= k <= min(n, 16384).
 *   ids_out     device int32[k]; scores_out device double[k] (may be NULL).
 */
rs_status rs_topk(rs_graph *g, const double *scores, int32_t k, int32_t *ids_out,
                  double *scores_out, void *stream);

/*
 * rs_apply_removals -- delete nodes (every incident edge) and undirected edges
 * (both directions) from the resident graph (the perturbations of Sec. VI-B).
 *
 *   nodes           host int32[n_nodes] node ids.
 *   edge_src/dst    host int32[n_edges] endpoint pairs.
 *   applied_out     optional host pointer: number of effective removals.
 * Node removals are applied first, then edge removals.  Removing a node that
 * is already removed, or an edge that is absent (or already removed), is a
 * no-op and is not counted.  Any id outside [0, n) makes the call fail with
 * RS_EINVAL before anything is changed.  Node ids keep their meaning; a
 * removed node has degree 0 and scores 0.  Synchronises `stream` when
 * applied_out is given.
 */
rs_status rs_apply_removals(rs_graph *g, const int32_t *nodes, int64_t n_nodes,
                            const int32_t *edge_src, const int32_t *edge_dst, int64_t n_edges,
                            int64_t *applied_out, void *stream);

/* rs_clone_graph -- deep copy of a graph (its current edges and removals). */
rs_status rs_clone_graph(const rs_graph *g, rs_graph **out, void *stream);

/* rs_graph_info -- sizes of a graph (any pointer may be NULL). */
rs_status rs_graph_info(const rs_graph *g, int64_t *n, int64_t *nnz, int32_t *k, int32_t *max_degree);

/*
 * rs_topk_noalloc -- the same ranking as rs_topk over a device array of n
 * scores, for callers that cannot allocate device memory: code whose device
 * memory is owned by another allocator (a framework's caching allocator, a
 * fixed memory budget), and latency-critical loops that cannot afford
 * cudaMalloc's implicit device synchronisation or its failure mid-request.
 * The paper has no counterpart; it ranks like rs_topk.
 *
 *   scores      device double[n], every value >= 0 (not NaN); 1 <= n < 2^31.
 *   k           1 <= k <= min(n, 16384); larger k returns RS_EINVAL.
 *   ids_out     device int32[k]; scores_out device double[k] (may be NULL).
 * Allocates nothing: its scratch is one static device array of about 213 KB
 * (histogram, control words, 16384 keys) that every GPU loading the library
 * holds until the process exits.  The first call on a device looks up that
 * array's address and sets the kernel up (per device, once); make that first
 * call before any stream capture.  Every call shares the array and the kernel
 * re-initialises it, so calls whose work overlaps on the GPU (other streams,
 * other host threads) race and must not overlap.  Stream-ordered; no host
 * synchronisation.
 */
rs_status rs_topk_noalloc(const double *scores, int64_t n, int32_t k, int32_t *ids_out, double *scores_out,
                          void *stream);

/*
 * Instrumentation (no counterpart in the paper; used by benchmarks and tuning).
 *
 * rs_profile_enable -- when enable != 0, every later rs_score / rs_topk call on
 *   g records a CUDA event on its stream after each device operation; the
 *   record is cleared by every rs_profile_enable call.
 * rs_profile_read -- waits for the last recorded event, then returns up to
 *   `cap` entries in order: names[i] (static strings owned by the library),
 *   ms[i] the device time since the previous event of the same call, and
 *   is_kernel[i] (1 for a kernel of this library, 0 for a memset).  *n_out is
 *   the number of entries recorded (may exceed cap).  Any array may be NULL.
 * rs_launch_count -- number of kernels this library has launched for g.
 */
rs_status rs_profile_enable(rs_graph *g, int enable);
rs_status rs_profile_read(rs_graph *g, int32_t *n_out, const char **names, float *ms, int32_t *is_kernel,
                          int32_t cap);
rs_status rs_launch_count(const rs_graph *g, int64_t *launches);

/*
 * Launch parameters of the scoring kernels.  None of them changes a result:
 * every sum is accumulated in exact fixed point, so scores are bit-identical
 * under any valid setting (the paper has no counterpart; its kernels use
 * fixed launch shapes, Sec. V).  Rows are split by degree d and by the hash
 * capacity cap = smallest power of two >= 2 min(d, k):
 *   small_max    rows with d <= small_max take the 32-row tile kernels    [1, 32]
 *   warp_cap     other rows with cap <= warp_cap take one warp each       {64,...,512}
 *   cta_cap      then rows with cap <= cta_cap take one CTA each;         {warp_cap,...,2048}
 *                larger rows are hubs (global table, split into chunks)
 *   hub_chunk    neighbours per hub work item                             {512,...,65536}
 *   p2_cta_dx    CTA rows with more cross neighbours than this take a     [32, 256]
 *                CTA in the second pass (else one warp)
 *   p1_cta_threads  threads per CTA row in the first pass                 {128, 256, 512}
 *   p2_cta_threads  threads per CTA row in the second pass                {256, 512, 1024}
 *   ctas_per_sm  grid size of the grid-stride kernels, in CTAs per SM     [1, 32]
 *   p3_mirror    1: a pass pairs every G_x edge's two directed values     {0, 1}
 *                before the triangle listing (an extra array of nnz
 *                float pairs); 0: the listing looks the reverse values of
 *                each triangle up in in-lists (fewer searches when G_x has
 *                few triangles per edge)
 *   p1_stage     1: the small-row tiles of the first pass copy their          {0, 1}
 *                columns, then the neighbours' labels, into shared memory
 *                with asynchronous copies (cp.async) before matching; 0:
 *                the loads are pipelined in registers two chunks ahead
 *   rows_streams how the row kernels of the two passes share the GPU:     {-1, 0, 1, 2}
 *                0: each row class on a stream of its own, the classes
 *                with long per-row chains at high priority; 1: the hub
 *                rows' kernels on one stream and the other classes, in
 *                turn, on a second; 2: every row kernel in turn on the
 *                step's stream; -1 (the default): 1 when the graph has
 *                hub rows and at least 32,000,000 CSR entries, else 0
 * Powers of two are required where a set is given.
 */
typedef struct {
    int32_t small_max;
    int32_t warp_cap;
    int32_t cta_cap;
    int32_t hub_chunk;
    int32_t p2_cta_dx;
    int32_t p1_cta_threads;
    int32_t p2_cta_threads;
    int32_t ctas_per_sm;
    int32_t p3_mirror;
    int32_t p1_stage;
    int32_t rows_streams;
} rs_tuning;

/* rs_default_tuning -- the parameters a new graph starts with. */
void rs_default_tuning(rs_tuning *out);
/* rs_get_tuning -- the parameters g uses now. */
rs_status rs_get_tuning(const rs_graph *g, rs_tuning *out);
/*
 * rs_set_tuning -- validate t (RS_EINVAL, g unchanged, if a field is outside
 *   its range) and re-split g's rows by it.  Synchronises `stream`.
 */
rs_status rs_set_tuning(rs_graph *g, const rs_tuning *t, void *stream);
/*
 * rs_autotune -- time one scoring step (rs_score, plus rs_topk(topk_k) when
 *   topk_k > 0) under a coordinate sweep of the parameters above, starting
 *   from the current ones, and leave g on the fastest.  Each candidate's step
 *   is captured as rs_step_capture does and timed as the median of `reps`
 *   replays (>= 1) with CUDA events on `stream`, after one untimed replay.
 *   When the sweep ends away from the starting parameters, both are timed
 *   again with 3 reps replays and the faster is kept.  `scores` (device, n doubles), `ids_out` and
 *   `vals_out` (device, topk_k each; may be NULL when topk_k == 0) are
 *   scratch.  best_out / best_ms_out (host, nullable) receive the choice and
 *   its median step time; n_tried_out (nullable) the candidates timed.
 */
rs_status rs_autotune(rs_graph *g, double *scores, int32_t topk_k, int32_t *ids_out, double *vals_out,
                      int32_t reps, void *stream, rs_tuning *best_out, float *best_ms_out,
                      int32_t *n_tried_out);

/*
 * A captured scoring step: rs_score(g, scores) followed, when topk_k > 0, by
 * rs_topk(g, scores, topk_k, ids_out, vals_out), recorded once as a CUDA graph
 * and replayed by rs_step_launch on any stream with one launch call.  The
 * graph holds g's current buffers and launch parameters: a later
 * rs_apply_removals or rs_set_tuning on g invalidates it (rs_step_launch then
 * returns RS_EINVAL).  Profiling must be off while capturing.
 */
typedef struct rs_step rs_step;
rs_status rs_step_capture(rs_graph *g, double *scores, int32_t topk_k, int32_t *ids_out, double *vals_out,
                          rs_step **out);
rs_status rs_step_launch(rs_step *st, void *stream);
void rs_step_free(rs_step *st);

/*
 * rs_target_subset -- the graph restricted to target communities.  The paper
 * searches spanners in user-provided (large) communities only and counts only
 * neighbours in them (T = sum of f_l over the k targets, Sec. V-A); its
 * experiments take the k largest communities (Sec. VI).  targets: host
 * int32[n_targets], distinct labels of g in [0, k).  The new graph (free with
 * rs_free_graph) keeps every node id; every edge with an endpoint outside the
 * targets is dropped, so such nodes are isolated and score 0; target i becomes
 * community i and k = n_targets (so w_max ranges over the target columns).
 * Not for batches.  Synchronises `stream`.
 */
rs_status rs_target_subset(const rs_graph *g, const int32_t *targets, int32_t n_targets, void *stream,
                           rs_graph **out);

/*
 * rs_awcc -- the community-spanning diversity of a node set S (Sec. VI-C):
 *   AWCC(S) = 1/|S| sum_{v in S} |zeta(v)| / d(v), zeta(v) = the communities of
 *   v's neighbours.  nodes: host int32[m] (S).  deg_ref: host int64[m] or NULL;
 *   when given, d(v) = deg_ref[i] (the paper's "absolute" AWCC after a
 *   disruption: only |zeta(v)| follows the changed graph), else the current
 *   degree; nodes with d(v) = 0 add 0.  zeta_out: host int32[m] or NULL.
 *   |zeta(v)| is counted by rs_score: the graph must have been scored since its
 *   last change (RS_EINVAL otherwise).  Synchronises `stream`.
 */
rs_status rs_awcc(rs_graph *g, const int32_t *nodes, int64_t m, const int64_t *deg_ref, double *awcc_out,
                  int32_t *zeta_out, void *stream);

/*
 * Serving: what-if rescoring of resident graphs.  The paper has no counterpart
 * (its dynamic networks are future work, Sec. VII; its removal experiments,
 * Sec. VI-C, remove nodes cumulatively and rescore from scratch).
 *
 * A request removes nodes (with every incident edge) and undirected edges from
 * one resident graph and asks for the top_k nodes of the changed graph's
 * scores.  Every request applies to the resident (base) graph, never to
 * another request's result, so a result does not depend on what else runs.
 *
 * rs_server_create -- take ownership of n_graphs graphs (single graphs, not
 *   batches; rs_server_free frees them), score each once (its base state,
 *   kept on the device) and create up to max_slots request slots: the requests
 *   that run concurrently, each on its own stream.  Slots are created while
 *   their device memory stays within budget_bytes (RS_EBUDGET if not even one
 *   fits); full copies of graphs made by the full path count against the
 *   budget too.  max_top_k bounds top_k (<= 16384).  mode:
 *     RS_SERVE_INCREMENTAL  a request recounts only the rows it touches and
 *                           updates the exact fixed-point sums by the terms that
 *                           change (bit-identical to a full rescoring); requests
 *                           whose touched rows exceed a slot's buffers, or whose
 *                           touched rows' degrees (bounded from the removed
 *                           nodes' 2-hop degree sums) exceed 1/4 of the CSR
 *                           entries, are rescored in full instead;
 *     RS_SERVE_FULL         every request restores a full copy of its graph,
 *                           applies the removals and rescores it completely.
 * rs_server_submit -- queue a request (lists are copied, ids are checked);
 *   returns its ticket.  No device work starts before rs_server_poll.
 * rs_server_poll -- start queued requests, in order, on free slots when the
 *   memory budget allows, and collect finished ones without waiting (block = 0)
 *   or until at least one finished or nothing is left (block != 0).  For each
 *   of at most `max` finished requests: tickets[i], status[i] (RS_OK, or
 *   RS_EBUDGET when it could not fit), path[i] (1 incremental, 0 full; may be
 *   NULL), and its min(kmax, top_k) best (id, score) pairs at ids[i*kmax] and
 *   scores[i*kmax] (host arrays, may be NULL); *n_done = how many.
 * rs_server_info -- slots, device bytes held by slots and full copies, queued
 *   and running requests (any out-pointer may be NULL).
 * rs_server_whatif -- run one request at once (no request may be in flight) and
 *   write the changed graph's scores for all n nodes to scores_out (device);
 *   full = 0 chooses as the server does, 1 forces the full path, 2 takes the
 *   incremental path whenever the slot's buffers hold the request (whatever
 *   its cost); *path_out (nullable) tells which ran.
 *   Synchronises `stream`.
 * rs_server_base_scores -- the base scores of a resident graph (device double[n]).
 */
typedef struct rs_server rs_server;
#define RS_SERVE_INCREMENTAL 0
#define RS_SERVE_FULL 1
rs_status rs_server_create(rs_graph *const *graphs, int32_t n_graphs, int32_t max_slots, int64_t budget_bytes,
                           int32_t max_top_k, int32_t mode, rs_server **out);
rs_status rs_server_submit(rs_server *srv, int32_t graph, const int32_t *nodes, int64_t n_nodes,
                           const int32_t *edge_src, const int32_t *edge_dst, int64_t n_edges, int32_t top_k,
                           int64_t *ticket_out);
rs_status rs_server_poll(rs_server *srv, int32_t max, int32_t kmax, int64_t *tickets, int32_t *status,
                         int32_t *path, int32_t *ids, double *scores, int32_t *n_done, int32_t block);
rs_status rs_server_info(const rs_server *srv, int32_t *slots, int64_t *bytes_used, int64_t *queued,
                         int32_t *in_flight);
rs_status rs_server_whatif(rs_server *srv, int32_t graph, const int32_t *nodes, int64_t n_nodes,
                           const int32_t *edge_src, const int32_t *edge_dst, int64_t n_edges, int32_t full,
                           double *scores_out, int32_t *path_out, void *stream);
rs_status rs_server_base_scores(rs_server *srv, int32_t graph, double *scores_out, void *stream);
void rs_server_free(rs_server *srv);

/*
 * rs_device_errors -- synchronise `stream` and return in *flags_out the
 *   internal consistency checks that failed in g's kernels during the last
 *   rs_score (bit flags; 0 when none).  A non-zero value means a library bug,
 *   not bad input: inputs are checked before any kernel runs.  The bits:
 *   1 a community hash table found full; 2, 4, 8 a community missing from a
 *   row's table in P2; 16 the reverse value of a G_x edge not found (P3);
 *   32 the G_x offset scan gave up waiting for a tile; 64 P3's heavy-node task
 *   list over its capacity or holding an invalid entry.
 */
rs_status rs_device_errors(rs_graph *g, int32_t *flags_out, void *stream);

/*
 * rs_test_gx_stall -- test hook (no counterpart in the paper): from the next
 * rs_score on, tile `tile` of the G_x offset scan does not publish its words and
 * every wait of the scan gives up after spin_limit reads, so that the tiles after
 * it run out of their bounded waits and take the fallback.  tile < 0 restores the
 * normal scan.  Invalidates captured steps.
 */
rs_status rs_test_gx_stall(rs_graph *g, int64_t tile, int64_t spin_limit);

/* rs_free_graph -- release a graph and its device memory (NULL is a no-op). */
void rs_free_graph(rs_graph *g);

/* rs_last_error -- message of the last failed call on this thread ("" if none). */
const char *rs_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* RS_H_ */
