"""Counts of the triangle listing on the cross-community subgraph G_x, behind the figures the
design notes give as "counted on the host" -- test infrastructure, no part of the library.

G_x holds the edges {u, w} with C(u) != C(w) whose ends both have cross degree dx >= 2; it is
oriented by rank (dx, id), and each node's out-list holds its higher-ranked G_x neighbours by
id.  ``stats(g)`` returns the counts of ``gx_stats.c`` (pairs and triangles of the light nodes,
wedges, walks, triangles and finishes of the heavy ones, searches in long out-lists) and
``hub_rows`` the rows the library treats as hubs (a hash table of more than 2,048 slots: the
power of two >= 2 min(d, k)).

    python tests/gx_stats.py dcsbm_8m            # also dcsbm_1m, sbm_2000, dense_core,
    python tests/gx_stats.py dcsbm_hub 2000000   # dcsbm_hub N, serve N K SEED
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gx_stats.c")
_LIB = os.path.join(_HERE, "_build", "libgxstats.so")
KEYS = ("light_pairs", "light_triangles", "heavy_nodes", "heavy_tasks", "heavy_walks", "heavy_wedges",
        "heavy_triangles", "finishes", "part_empty_finishes", "edges_tail_list_over_64",
        "light_pairs_list_over_64")
HIST_MAX = 4096


def _lib():
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    lib = ctypes.CDLL(_LIB)
    P = ctypes.c_void_p
    lib.gx_stats.restype = ctypes.c_int
    lib.gx_stats.argtypes = [ctypes.c_int64, P, P, P, P, P, ctypes.c_int32]
    return lib


def orient(offsets, cols, labels):
    """(dx, xoff, xcol): cross degrees and the out-lists of G_x (sorted by id)."""
    n = labels.shape[0]
    rows = np.repeat(np.arange(n, dtype=np.int32), np.diff(offsets))
    cols = np.asarray(cols, dtype=np.int32)
    cross = labels[rows] != labels[cols]
    dx = np.bincount(rows[cross], minlength=n).astype(np.int32)
    keep = cross & (dx[rows] >= 2) & (dx[cols] >= 2)
    a, b = rows[keep], cols[keep]
    del rows, cross, keep
    out = (dx[b] > dx[a]) | ((dx[b] == dx[a]) & (b > a))
    a, b = a[out], b[out]
    order = np.lexsort((b, a))
    xoff = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(a, minlength=n), out=xoff[1:])
    return dx, xoff, np.ascontiguousarray(b[order], dtype=np.int32)


def stats(g):
    dx, xoff, xcol = orient(g.offsets, g.cols, g.labels)
    out = np.zeros(len(KEYS), np.int64)
    hist = np.zeros(HIST_MAX + 1, np.int64)
    rc = _lib().gx_stats(g.labels.shape[0], xoff.ctypes.data, xcol.ctypes.data, dx.ctypes.data, out.ctypes.data,
                         hist.ctypes.data, HIST_MAX)
    if rc:
        raise MemoryError("gx_stats")
    res = dict(zip(KEYS, (int(x) for x in out)))
    res["gx_edges"] = int(xcol.shape[0])
    res["max_out_degree"] = int(np.diff(xoff).max()) if xcol.shape[0] else 0
    c = np.cumsum(hist)
    res["median_searched_list"] = int(np.searchsorted(c, (c[-1] + 1) // 2)) if c[-1] else 0
    return res


def hub_rows(offsets, k_of_row):
    """Rows whose table (the power of two >= 2 min(d, k)) has more than 2,048 slots: their
    number and their share of the CSR entries."""
    d = np.diff(offsets)
    m = np.minimum(d, k_of_row).astype(np.float64)
    cap = np.where(m > 0, np.exp2(np.ceil(np.log2(np.maximum(2 * m, 1)))), 0)
    hub = cap > 2048
    return int(hub.sum()), float(d[hub].sum()) / max(1, int(d.sum()))


def _graph(argv):
    sys.path.insert(0, os.path.dirname(_HERE))
    import graphgen
    name = argv[0]
    if name == "dcsbm_hub":
        return graphgen.dcsbm_hub(int(argv[1]))
    if name == "serve":          # a serving graph: the 1M shape at n nodes with k communities
        n, k, seed = int(argv[1]), int(argv[2]), int(argv[3])
        return graphgen.dcsbm(n, k, 50.0, 2.5, 8, min(5000, n - 1), 0.2, seed)
    return getattr(graphgen, name)()


if __name__ == "__main__":
    g = _graph(sys.argv[1:])
    s = stats(g)
    h, share = hub_rows(g.offsets, g.k)
    for key, v in s.items():
        print("%-28s %d" % (key, v))
    print("%-28s %d (%.2f%% of the CSR entries)" % ("hub_rows", h, 100 * share))
