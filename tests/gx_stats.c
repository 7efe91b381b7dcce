/*
 * gx_stats.c -- counts of the triangle listing on the cross-community subgraph G_x, for
 * the figures the design notes give as "counted on the host".  Test infrastructure: no
 * part of the library uses it, and it uses no part of the library.
 *
 * Input: G_x oriented by rank (cross degree, id), as out-lists: xoff[n + 1], xcol[m] (each
 * node's higher-ranked G_x neighbours, sorted by id), and dx[n] (the cross degree that
 * ranks the nodes).  A node with 2..128 out-neighbours is light (its pairs of
 * out-neighbours are tested), one with more is heavy (its wedges are walked, one walk per
 * out-neighbour b, in tasks of 128 out-neighbours).
 *
 * out[ 0] light pairs                 sum over light a of d+(a) (d+(a) - 1) / 2
 * out[ 1] light triangles             triangles whose lowest-ranked node is light
 * out[ 2] heavy nodes
 * out[ 3] heavy tasks                 sum over heavy a of ceil(d+(a) / 128)
 * out[ 4] heavy walks                 sum over heavy a of d+(a)
 * out[ 5] heavy wedges                sum over heavy a, b in N+(a) of d+(b)
 * out[ 6] heavy triangles             triangles whose lowest-ranked node is heavy
 * out[ 7] finishes                    sum over walks of ceil(t / 32), t = the walk's triangles
 * out[ 8] part-empty finishes         walks whose t is not a multiple of 32
 * out[ 9] edges whose tail's out-list has more than 64 ids (the mirror pass searches the
 *         tail's out-list for the head)
 * out[10] light pairs whose lower-ranked node's out-list has more than 64 ids
 * hist[L] (L <= hist_max; longer lists counted at hist_max): light pairs by the out-list
 *         length of their lower-ranked node, the list a pair's closing edge is looked up in
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static int rank_less(const int32_t *dx, int32_t a, int32_t b) {
    return dx[a] < dx[b] || (dx[a] == dx[b] && a < b);
}

int gx_stats(int64_t n, const int64_t *xoff, const int32_t *xcol, const int32_t *dx, int64_t *out,
             int64_t *hist, int32_t hist_max) {
    uint8_t *mark = (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
    if (!mark) return 1;
    memset(out, 0, 11 * sizeof(int64_t));
    memset(hist, 0, ((size_t)hist_max + 1) * sizeof(int64_t));
    for (int64_t a = 0; a < n; ++a) {
        const int64_t lo = xoff[a], hi = xoff[a + 1], d = hi - lo;
        if (d > 64) out[9] += d;
        if (d < 2) continue;
        for (int64_t i = lo; i < hi; ++i) mark[xcol[i]] = 1;
        if (d <= 128) {
            out[0] += d * (d - 1) / 2;
            for (int64_t i = lo; i < hi; ++i) {
                const int32_t b = xcol[i];
                for (int64_t j = i + 1; j < hi; ++j) {
                    const int32_t c = xcol[j];
                    const int32_t low = rank_less(dx, b, c) ? b : c;
                    int64_t len = xoff[low + 1] - xoff[low];
                    if (len > 64) out[10]++;
                    hist[len < hist_max ? len : hist_max]++;
                }
                for (int64_t j = xoff[b]; j < xoff[b + 1]; ++j) out[1] += mark[xcol[j]];
            }
        } else {
            out[2]++;
            out[3] += (d + 127) / 128;
            out[4] += d;
            for (int64_t i = lo; i < hi; ++i) {
                const int32_t b = xcol[i];
                int64_t t = 0;
                out[5] += xoff[b + 1] - xoff[b];
                for (int64_t j = xoff[b]; j < xoff[b + 1]; ++j) t += mark[xcol[j]];
                out[6] += t;
                out[7] += (t + 31) / 32;
                out[8] += (t % 32) != 0;
            }
        }
        for (int64_t i = lo; i < hi; ++i) mark[xcol[i]] = 0;
    }
    free(mark);
    return 0;
}
