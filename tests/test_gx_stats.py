"""The host counting tool behind the design notes' "counted on the host" figures
(tests/gx_stats.py): its counts against a plain recount on small graphs, no GPU."""
import itertools

import numpy as np
import pytest

import graphgen
import gx_stats


def _recount(g):
    """G_x from its definition (sets of cross edges, ranks by (dx, id)) and the counts from
    the enumerated triangles and pairs."""
    n = g.labels.shape[0]
    adj = [set(g.cols[g.offsets[v]:g.offsets[v + 1]].tolist()) for v in range(n)]
    lab = g.labels
    dx = [sum(1 for u in adj[v] if lab[u] != lab[v]) for v in range(n)]
    rank = lambda v: (dx[v], v)
    outs = [sorted(u for u in adj[v] if lab[u] != lab[v] and dx[u] >= 2 and dx[v] >= 2 and rank(u) > rank(v))
            for v in range(n)]
    out_sets = [set(o) for o in outs]
    r = dict.fromkeys(gx_stats.KEYS, 0)
    tri_total = 0
    for a in range(n):
        A = outs[a]
        d = len(A)
        if d > 64:
            r["edges_tail_list_over_64"] += d
        if d < 2:
            continue
        if d <= 128:
            r["light_pairs"] += d * (d - 1) // 2
            for b, c in itertools.combinations(A, 2):
                lo, hi = (b, c) if rank(b) < rank(c) else (c, b)
                if len(outs[lo]) > 64:
                    r["light_pairs_list_over_64"] += 1
                if hi in out_sets[lo]:
                    r["light_triangles"] += 1
        else:
            r["heavy_nodes"] += 1
            r["heavy_tasks"] += (d + 127) // 128
            r["heavy_walks"] += d
            for b in A:
                r["heavy_wedges"] += len(outs[b])
                t = len(out_sets[b] & out_sets[a])
                r["heavy_triangles"] += t
                r["finishes"] += (t + 31) // 32
                r["part_empty_finishes"] += t % 32 != 0
    # every triangle of the undirected G_x, counted once
    und = [set(o) for o in outs]
    for a in range(n):
        for b in outs[a]:
            und[b].add(a)
    for a in range(n):
        for b in und[a]:
            if b > a:
                tri_total += sum(1 for c in und[a] & und[b] if c > b)
    return r, tri_total, sum(len(o) for o in outs)


@pytest.mark.parametrize("which", ["dcsbm", "dense_core", "sbm"])
def test_counts_match_a_plain_recount(which):
    if which == "dcsbm":
        g = graphgen.dcsbm_small(6000, seed=3, dmax=600, mu=0.4)
    elif which == "dense_core":
        g = graphgen.dense_core(n_core=300, n_fan=700, fan_min=40, fan_max=260, n_full=4)
    else:
        g = graphgen.sbm_2000()
    got = gx_stats.stats(g)
    want, tri_total, m_x = _recount(g)
    for key in gx_stats.KEYS:
        assert got[key] == want[key], (key, got[key], want[key])
    # each triangle is listed once, at its lowest-ranked node
    assert got["light_triangles"] + got["heavy_triangles"] == tri_total
    assert got["gx_edges"] == m_x
    if which == "dense_core":
        assert got["heavy_nodes"] > 0 and got["heavy_triangles"] > 0 and got["part_empty_finishes"] > 0


def test_hub_rows_rule():
    # degrees 3000 and 10: with k = 5000 the first row's table has 8,192 slots (a hub), with
    # k = 1000 it has 2,048 (not a hub)
    off = np.array([0, 3000, 3010], np.int64)
    assert gx_stats.hub_rows(off, np.array([5000, 5000]))[0] == 1
    assert gx_stats.hub_rows(off, np.array([1000, 1000]))[0] == 0
    h, share = gx_stats.hub_rows(off, np.array([5000, 5000]))
    assert abs(share - 3000 / 3010) < 1e-12
