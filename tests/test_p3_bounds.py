"""The capacity of P3's heavy-node task list (host logic, no GPU).

A node with more than 128 G_x out-neighbours is walked in tasks of 128
out-neighbours, listed in a buffer sized from nnz alone before any kernel runs.
Every G_x edge has one tail, and a heavy node's ceil(d+/128) tasks are at most
d+ 256/(128 129), so the tasks number at most 2 m_x / 129 <= nnz / 129.  These graphs check that bound on the
orientation the library uses (cross degree, then id), including cliques and a
complete bipartite graph whose heavy nodes all sit at the 129-neighbour worst
case."""
import os
import re

import numpy as np

import graphgen

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(HERE, "..", "paper_2508_01485_gb300", "csrc", "rs_internal.cuh")


def _cap_divisor():
    src = open(HEADER).read()
    m = re.search(r"hv_cap\(int64_t nnz\) \{ return nnz / (\d+) \+ 1; \}", src)
    assert m, "hv_cap's formula not found"
    assert re.search(r"constexpr int kWinCap = 128, kHvBlock = 128;", src)
    return int(m.group(1))


def _tasks(offsets, cols, labels):
    """Tasks of the heavy nodes of G_x oriented by (cross degree, id)."""
    n = labels.shape[0]
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(offsets))
    cols = cols.astype(np.int64)
    cross = labels[rows] != labels[cols]
    dx = np.bincount(rows[cross], minlength=n)
    keep = cross & (dx[rows] >= 2) & (dx[cols] >= 2)
    a, b = rows[keep], cols[keep]
    out = (dx[b] > dx[a]) | ((dx[b] == dx[a]) & (b > a))
    xo = np.bincount(a[out], minlength=n)
    heavy = xo[xo > 128]
    return int(((heavy + 127) // 128).sum()), int(heavy.size)


def _csr(n, u, v):
    key = np.unique(np.minimum(u, v).astype(np.int64) * n + np.maximum(u, v))
    u, v = key // n, key % n
    src, dst = np.concatenate([u, v]), np.concatenate([v, u])
    o = np.lexsort((dst, src))
    off = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(src[o], minlength=n), out=off[1:])
    return off, dst[o].astype(np.int32)


def _clique(k):
    u, v = np.triu_indices(k, 1)
    off, cols = _csr(k, u, v)
    return off, cols, np.arange(k, dtype=np.int32)          # every node its own community


def _worst_case(leaves):
    """Complete bipartite: `leaves` nodes each joined to the same 129 hubs (other
    communities).  The hubs' cross degree is the larger, so every G_x edge's tail is a
    leaf with exactly 129 out-neighbours: 2 tasks per 129 edges, the bound's worst case."""
    n = leaves + 129
    u = np.repeat(np.arange(leaves), 129)
    v = leaves + np.tile(np.arange(129), leaves)
    off, cols = _csr(n, u, v)
    labels = np.concatenate([np.zeros(leaves), 1 + np.arange(129)]).astype(np.int32)
    return off, cols, labels


def test_task_list_capacity_holds():
    div = _cap_divisor()
    cases = [_clique(400), _clique(1500), _worst_case(300)]
    for g in (graphgen.dense_core(), graphgen.dcsbm_small(20000, seed=3, dmax=800)):
        cases.append((g.offsets, g.cols, g.labels))
    seen_heavy = 0
    for off, cols, labels in cases:
        tasks, heavy = _tasks(off, cols, labels)
        nnz = int(off[-1])
        assert tasks <= nnz // div + 1, (tasks, nnz)
        seen_heavy += heavy
    assert seen_heavy > 0


def test_worst_case_comes_close_to_the_capacity():
    div = _cap_divisor()
    off, cols, labels = _worst_case(300)
    tasks, heavy = _tasks(off, cols, labels)
    assert heavy == 300 and tasks == 600
    assert 0.95 * (int(off[-1]) // div + 1) < tasks <= int(off[-1]) // div + 1
