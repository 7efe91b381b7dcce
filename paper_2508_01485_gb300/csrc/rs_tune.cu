// rs_tune.cu -- launch parameters, the autotuner and captured scoring steps.
//
// The scoring kernels' row split points, CTA sizes and grid sizes are runtime
// parameters (rs_tuning).  None changes a result: every sum of the score is
// accumulated in exact fixed point, so any valid setting gives bit-identical
// scores.  rs_autotune times a scoring step under a coordinate sweep of the
// parameters and keeps the fastest.  rs_step_capture records a whole step
// (the kernels of every auxiliary stream, joined back by events) as one CUDA
// graph that rs_step_launch replays with a single launch call.
#include <algorithm>
#include <cstring>
#include <vector>

#include "rs.h"
#include "rs_internal.cuh"

using namespace rs;

static cudaStream_t as_stream(void *s) { return (cudaStream_t)s; }

static bool is_pow2(int32_t x) { return x > 0 && (x & (x - 1)) == 0; }

static int check_tuning(const rs_tuning &t) {
    if (t.small_max < 1 || t.small_max > kSmallMax)
        return fail(RS_EINVAL, "rs_tuning: small_max must be in [1, 32]");
    if (!is_pow2(t.warp_cap) || t.warp_cap < 64 || t.warp_cap > kWarpCap)
        return fail(RS_EINVAL, "rs_tuning: warp_cap must be a power of two in [64, 512]");
    if (!is_pow2(t.cta_cap) || t.cta_cap < t.warp_cap || t.cta_cap > kMidCap)
        return fail(RS_EINVAL, "rs_tuning: cta_cap must be a power of two in [warp_cap, 2048]");
    if (!is_pow2(t.hub_chunk) || t.hub_chunk < 512 || t.hub_chunk > 65536)
        return fail(RS_EINVAL, "rs_tuning: hub_chunk must be a power of two in [512, 65536]");
    if (t.p2_cta_dx < 32 || t.p2_cta_dx > kWarpCap / 2)
        return fail(RS_EINVAL, "rs_tuning: p2_cta_dx must be in [32, 256]");
    if (t.p1_cta_threads != 128 && t.p1_cta_threads != 256 && t.p1_cta_threads != 512)
        return fail(RS_EINVAL, "rs_tuning: p1_cta_threads must be 128, 256 or 512");
    if (t.p2_cta_threads != 256 && t.p2_cta_threads != 512 && t.p2_cta_threads != 1024)
        return fail(RS_EINVAL, "rs_tuning: p2_cta_threads must be 256, 512 or 1024");
    if (t.ctas_per_sm < 1 || t.ctas_per_sm > 32)
        return fail(RS_EINVAL, "rs_tuning: ctas_per_sm must be in [1, 32]");
    if (t.p3_mirror != 0 && t.p3_mirror != 1)
        return fail(RS_EINVAL, "rs_tuning: p3_mirror must be 0 or 1");
    if (t.p1_stage != 0 && t.p1_stage != 1)
        return fail(RS_EINVAL, "rs_tuning: p1_stage must be 0 or 1");
    if (t.rows_streams < -1 || t.rows_streams > 2)
        return fail(RS_EINVAL, "rs_tuning: rows_streams must be -1, 0, 1 or 2");
    return 0;
}

static bool same_split(const rs_tuning &a, const rs_tuning &b) {
    return a.small_max == b.small_max && a.warp_cap == b.warp_cap && a.cta_cap == b.cta_cap &&
           a.hub_chunk == b.hub_chunk;
}

// apply t; rows are re-split only when a split point changed
static int apply_tuning(rs_graph *g, const rs_tuning &t, cudaStream_t s) {
    bool resplit = !same_split(g->tune, t);
    g->tune = t;
    if (int rc = set_mirror_buffer(g)) return rc;
    if (resplit) return reclassify(g, s);
    g->version++;                    // launch shapes changed: captured steps are stale
    return 0;
}

extern "C" void rs_default_tuning(rs_tuning *out) {
    if (out) *out = default_tuning_value();
}

extern "C" rs_status rs_get_tuning(const rs_graph *g, rs_tuning *out) {
    if (!g || !out) return (rs_status)fail(RS_EINVAL, "rs_get_tuning: NULL argument");
    *out = g->tune;
    return RS_OK;
}

extern "C" rs_status rs_set_tuning(rs_graph *g, const rs_tuning *t, void *stream) {
    if (!g || !t) return (rs_status)fail(RS_EINVAL, "rs_set_tuning: NULL argument");
    if (int rc = check_tuning(*t)) return (rs_status)rc;
    cudaStream_t s = as_stream(stream);
    rs_tuning old = g->tune;
    if (int rc = apply_tuning(g, *t, s)) {
        g->tune = old;               // best effort: restore the previous split
        reclassify(g, s);
        return (rs_status)rc;
    }
    return RS_OK;
}

// ---------------------------------------------------------------------------
// autotuner
// ---------------------------------------------------------------------------

// median device time of `reps` replays of the step captured for the current
// parameters (as rs_step_capture records it), after one untimed replay
static int time_step(rs_graph *g, double *scores, int32_t topk_k, int32_t *ids, double *vals, int32_t reps,
                     cudaStream_t s, std::vector<cudaEvent_t> &ev, float *ms_out) {
    rs_step *st = nullptr;
    if (rs_status rc = rs_step_capture(g, scores, topk_k, ids, vals, &st)) return rc;
    int rc = rs_step_launch(st, s);
    for (int32_t r = 0; !rc && r < reps; ++r) {
        if (cudaError_t e = cudaEventRecord(ev[2 * r], s)) rc = cuda_fail(e, "rs_autotune: event");
        if (!rc) rc = rs_step_launch(st, s);
        if (!rc)
            if (cudaError_t e = cudaEventRecord(ev[2 * r + 1], s)) rc = cuda_fail(e, "rs_autotune: event");
    }
    if (!rc)
        if (cudaError_t e = cudaStreamSynchronize(s)) rc = cuda_fail(e, "rs_autotune: synchronize");
    rs_step_free(st);
    if (rc) return rc;
    std::vector<float> t(reps);
    for (int32_t r = 0; r < reps; ++r) RS_CUDA_TRY(cudaEventElapsedTime(&t[r], ev[2 * r], ev[2 * r + 1]));
    std::sort(t.begin(), t.end());
    *ms_out = t[reps / 2];
    return 0;
}

extern "C" rs_status rs_autotune(rs_graph *g, double *scores, int32_t topk_k, int32_t *ids_out, double *vals_out,
                                 int32_t reps, void *stream, rs_tuning *best_out, float *best_ms_out,
                                 int32_t *n_tried_out) {
    if (!g || (!scores && g->n > 0)) return (rs_status)fail(RS_EINVAL, "rs_autotune: NULL argument");
    if (reps < 1 || reps > 1000) return (rs_status)fail(RS_EINVAL, "rs_autotune: reps must be in [1, 1000]");
    if (topk_k < 0 || topk_k > 16384 || (topk_k > 0 && ((int64_t)topk_k > g->n || !ids_out)))
        return (rs_status)fail(RS_EINVAL, "rs_autotune: topk_k must be 0 or in [1, min(n, 16384)] with ids_out");
    if (g->prof_on) return (rs_status)fail(RS_EINVAL, "rs_autotune: profiling is on");
    cudaStream_t s = as_stream(stream);
    if (g->n == 0) {
        if (best_out) *best_out = g->tune;
        if (best_ms_out) *best_ms_out = 0.0f;
        if (n_tried_out) *n_tried_out = 0;
        return RS_OK;
    }
    const int32_t confirm_reps = 3 * reps;          // the final comparison takes three times the replays
    std::vector<cudaEvent_t> ev(2 * (size_t)confirm_reps, nullptr);
    auto cleanup = [&]() {
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
    };
    for (auto &e : ev)
        if (cudaError_t ce = cudaEventCreate(&e)) {
            cleanup();
            return (rs_status)cuda_fail(ce, "rs_autotune: events");
        }
    const rs_tuning start = g->tune;
    rs_tuning best = g->tune;
    float best_ms = 0.0f;
    int32_t tried = 1;
    int rc = time_step(g, scores, topk_k, ids_out, vals_out, reps, s, ev, &best_ms);
    // one parameter at a time, the others at the best found so far
    struct Axis { int32_t rs_tuning::*field; std::vector<int32_t> values; };
    const std::vector<Axis> axes = {
        {&rs_tuning::ctas_per_sm, {4, 8, 16}},
        {&rs_tuning::small_max, {16, 24, 32}},
        {&rs_tuning::warp_cap, {128, 256, 512}},
        {&rs_tuning::cta_cap, {512, 1024, 2048}},
        {&rs_tuning::p2_cta_dx, {64, 128, 256}},
        {&rs_tuning::p1_cta_threads, {128, 256, 512}},
        {&rs_tuning::p2_cta_threads, {256, 512, 1024}},
        {&rs_tuning::hub_chunk, {1024, 4096, 16384}},
        {&rs_tuning::p3_mirror, {0, 1}},
        {&rs_tuning::p1_stage, {0, 1}},
        {&rs_tuning::rows_streams, {0, 1, 2}},
    };
    for (size_t a = 0; !rc && a < axes.size(); ++a) {
        for (int32_t v : axes[a].values) {
            rs_tuning t = best;
            if (t.*(axes[a].field) == v) continue;
            t.*(axes[a].field) = v;
            if (check_tuning(t)) continue;          // e.g. cta_cap below warp_cap
            if ((rc = apply_tuning(g, t, s))) break;
            float ms = 0.0f;
            if ((rc = time_step(g, scores, topk_k, ids_out, vals_out, reps, s, ev, &ms))) break;
            ++tried;
            if (ms < 0.99f * best_ms) { best = t; best_ms = ms; }
        }
    }
    // a sweep that moved away from the starting parameters: both are timed again with
    // more replays, so that a difference at the level of the timing noise cannot win
    if (!rc && std::memcmp(&best, &start, sizeof(rs_tuning)) != 0) {
        float ms_best = 0.0f, ms_start = 0.0f;
        if (!(rc = apply_tuning(g, best, s))) rc = time_step(g, scores, topk_k, ids_out, vals_out, confirm_reps, s, ev, &ms_best);
        if (!rc && !(rc = apply_tuning(g, start, s)))
            rc = time_step(g, scores, topk_k, ids_out, vals_out, confirm_reps, s, ev, &ms_start);
        tried += 2;
        if (!rc) {
            if (ms_start <= ms_best) { best = start; best_ms = ms_start; }
            else best_ms = ms_best;
        }
    }
    cleanup();
    if (!rc) rc = apply_tuning(g, best, s);
    if (rc) return (rs_status)rc;
    if (best_out) *best_out = best;
    if (best_ms_out) *best_ms_out = best_ms;
    if (n_tried_out) *n_tried_out = tried;
    return RS_OK;
}

// ---------------------------------------------------------------------------
// captured steps
// ---------------------------------------------------------------------------
struct rs_step {
    rs_graph *g = nullptr;
    uint64_t version = 0;
    int64_t launches = 0;            // kernels per replay
    cudaGraphExec_t exec = nullptr;
};

extern "C" rs_status rs_step_capture(rs_graph *g, double *scores, int32_t topk_k, int32_t *ids_out, double *vals_out,
                                     rs_step **out) {
    if (!g || !out || (!scores && g->n > 0)) return (rs_status)fail(RS_EINVAL, "rs_step_capture: NULL argument");
    if (topk_k < 0 || topk_k > 16384 || (topk_k > 0 && ((int64_t)topk_k > g->n || !ids_out)))
        return (rs_status)fail(RS_EINVAL, "rs_step_capture: topk_k must be 0 or in [1, min(n, 16384)] with ids_out");
    if (g->prof_on) return (rs_status)fail(RS_EINVAL, "rs_step_capture: profiling is on");
    if (int rc = prepare_score_kernels()) return (rs_status)rc;
    if (topk_k > 0)
        if (int rc = topk_prepare(g, g->n)) return (rs_status)rc;
    cudaStream_t cap = nullptr;
    if (cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking))
        return (rs_status)cuda_fail(e, "rs_step_capture: stream");
    int64_t l0 = g->launches;
    cudaGraph_t graph = nullptr;
    int rc = 0;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e) {
        rc = cuda_fail(e, "rs_step_capture: begin capture");
    } else {
        rc = score_graph(g, scores, cap);
        if (!rc && topk_k > 0) rc = topk_scores(g, scores, g->n, topk_k, ids_out, vals_out, cap);
        cudaError_t e2 = cudaStreamEndCapture(cap, &graph);   // always ends the capture
        if (!rc && e2) rc = cuda_fail(e2, "rs_step_capture: end capture");
    }
    int64_t captured = g->launches - l0;
    g->launches = l0;                // recorded, not launched
    cudaGraphExec_t exec = nullptr;
    if (!rc) {
        if (cudaError_t e3 = cudaGraphInstantiate(&exec, graph, 0)) rc = cuda_fail(e3, "rs_step_capture: instantiate");
    }
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cap);
    if (rc) return (rs_status)rc;
    rs_step *st = new rs_step();
    st->g = g;
    st->version = g->version;
    st->launches = captured;
    st->exec = exec;
    *out = st;
    return RS_OK;
}

extern "C" rs_status rs_step_launch(rs_step *st, void *stream) {
    if (!st) return (rs_status)fail(RS_EINVAL, "rs_step_launch: NULL step");
    if (st->version != st->g->version)
        return (rs_status)fail(RS_EINVAL, "rs_step_launch: the graph changed since the step was captured");
    if (cudaError_t e = cudaGraphLaunch(st->exec, as_stream(stream)))
        return (rs_status)cuda_fail(e, "rs_step_launch");
    st->g->launches += st->launches;
    return RS_OK;
}

extern "C" void rs_step_free(rs_step *st) {
    if (!st) return;
    if (st->exec) cudaGraphExecDestroy(st->exec);
    delete st;
}
