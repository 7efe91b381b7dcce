"""Seeded synthetic community-labelled graphs.

The one input module shared by the CPU oracle and the GPU path.  It draws
graphs shaped like the paper's social-network workloads (Sec. VI, the small and
large dataset tables): a planted-partition SBM and a degree-corrected SBM with
power-law community sizes and degrees.  It contains none of the scoring
arithmetic.  The C source is ``rsgen.c``; it is compiled on first use with gcc.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rsgen.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "librsgen.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile rsgen.c into graphgen/_build/librsgen.so (idempotent)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P, I64, I32, U64, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_double
        lib.rsgen_new.restype = P
        lib.rsgen_free.argtypes = [P]
        lib.rsgen_n.restype = I64; lib.rsgen_n.argtypes = [P]
        lib.rsgen_nnz.restype = I64; lib.rsgen_nnz.argtypes = [P]
        lib.rsgen_k.restype = I32; lib.rsgen_k.argtypes = [P]
        lib.rsgen_err.restype = ctypes.c_char_p; lib.rsgen_err.argtypes = [P]
        lib.rsgen_copy.argtypes = [P, P, P, P]
        lib.rsgen_sbm.restype = ctypes.c_int
        lib.rsgen_sbm.argtypes = [P, I32, I32, D, D, U64]
        lib.rsgen_dcsbm.restype = ctypes.c_int
        lib.rsgen_dcsbm.argtypes = [P, I64, I32, D, D, I32, I32, D, U64]
        _lib = lib
    return _lib


@dataclass
class Graph:
    """Undirected graph as symmetric CSR with community labels."""
    n: int
    k: int
    offsets: np.ndarray  # int64[n+1]
    cols: np.ndarray     # int32[nnz], each row sorted ascending
    labels: np.ndarray   # int32[n], values in [0, k)
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.cols.shape[0])

    @property
    def m(self) -> int:
        """Undirected edge count."""
        return self.nnz // 2

    def degrees(self) -> np.ndarray:
        return np.diff(self.offsets)


def _run(fn, *args, name=""):
    lib = _load()
    h = lib.rsgen_new()
    try:
        if fn(h, *args) != 0:
            raise ValueError(lib.rsgen_err(h).decode())
        n, nnz, k = lib.rsgen_n(h), lib.rsgen_nnz(h), lib.rsgen_k(h)
        off = np.empty(n + 1, np.int64)
        cols = np.empty(max(nnz, 1), np.int32)
        lab = np.empty(n, np.int32)
        lib.rsgen_copy(h, off.ctypes.data, cols.ctypes.data, lab.ctypes.data)
        return Graph(n=n, k=k, offsets=off, cols=cols[:nnz].copy(), labels=lab, name=name)
    finally:
        lib.rsgen_free(h)


def sbm(nblocks: int, block_size: int, p_in: float, p_out: float, seed: int, name: str = "") -> Graph:
    """Planted-partition SBM: equal blocks, independent Bernoulli edges over all pairs."""
    return _run(_load().rsgen_sbm, nblocks, block_size, p_in, p_out, seed, name=name or "sbm")


def dcsbm(n: int, k: int, size_min: float, gamma: float, dmin: int, dmax: int, mu: float,
          seed: int, name: str = "") -> Graph:
    """Degree-corrected SBM (configuration model) with rank-size community sizes."""
    return _run(_load().rsgen_dcsbm, n, k, size_min, gamma, dmin, dmax, mu, seed,
                name=name or "dcsbm")


# ---- named workloads -------------------------------------------------------

def sbm_2000(seed: int = 1) -> Graph:
    """2,000 nodes in 20 planted blocks of 100; mean intra degree 8, mean inter degree 1."""
    return sbm(20, 100, 8.0 / 99.0, 1.0 / 1900.0, seed, name="sbm-2k-20x100")


def dcsbm_1m(seed: int = 2) -> Graph:
    """1M nodes, 1,000 power-law communities (exponent 2, min 50), degrees power law 2.5 on
    [8, 5000], mu 0.2: about 10.3M undirected edges (min degree 8 rather than 2 gives ~10M)."""
    return dcsbm(1_000_000, 1000, 50.0, 2.5, 8, 5000, 0.2, seed, name="dcsbm-1m-k1000")


def dcsbm_1m_dmin2(seed: int = 2) -> Graph:
    """As dcsbm_1m with the literal minimum degree 2 (about 2.3M edges)."""
    return dcsbm(1_000_000, 1000, 50.0, 2.5, 2, 5000, 0.2, seed, name="dcsbm-1m-k1000-dmin2")


def dcsbm_8m(seed: int = 3) -> Graph:
    """8M nodes, 50,000 communities (sizes ~1/r), degrees power law 2.1 on [5, 100000], mu 0.1.

    Minimum degree 5 rather than 4: small communities push intra stubs out, so
    d_min = 4 realises only ~80M edges instead of the ~100M asked for."""
    return dcsbm(8_000_000, 50_000, 1.0, 2.1, 5, 100_000, 0.1, seed, name="dcsbm-8m-k50000")


def dcsbm_hub(n: int, seed: int = 13) -> Graph:
    """The 8M workload's shape scaled to n nodes: k = n / 160 communities (sizes ~1/r),
    degrees power law 2.1 on [5, 100000], mu 0.1.  At n = 2M it has ~23.6M edges and
    ~8,700 nodes with more than 128 G_x out-neighbours: the heavy-node triangle walk at
    about a tenth of the 8M graph's."""
    return dcsbm(n, max(2, n // 160), 1.0, 2.1, 5, 100_000, 0.1, seed, name="dcsbm-hub-%d" % n)


def dcsbm_small(n: int, seed: int, dmax: int = 1000, mu: float = 0.2, gamma: float = 2.5,
                dmin: int = 7) -> Graph:
    """Scaled DC-SBM with the 1M workload's shape: k = n / 100 communities (min size 50)."""
    k = max(2, n // 100)
    return dcsbm(n, k, 50.0 if n >= 100 * 50 else 1.0, gamma, dmin, dmax, mu, seed,
                 name="dcsbm-%d" % n)


# ---- batches of independent graphs -----------------------------------------

def dense_core(n_core: int = 600, n_fan: int = 2500, fan_min: int = 40, fan_max: int = 420, n_full: int = 6,
               core_edges: int = 400, fan_edges: int = 400, k: int = 40, seed: int = 11) -> Graph:
    """A dense bipartite core, so that many nodes have long G_x out-lists (G_x oriented by
    cross degree, then id).  Each of n_fan fan nodes is joined to a uniform random subset of
    the n_core core nodes (subset size uniform on [fan_min, fan_max]); n_full nodes are joined
    to every core node; core_edges random pairs of core nodes and fan_edges random pairs of
    fan nodes are joined as well (duplicates and loops dropped); labels uniform on [0, k).
    Core nodes end up with the largest cross degrees, so the fan nodes' out-lists (up to
    ~fan_max) and the full nodes' (~n_core) hold core nodes."""
    rng = np.random.default_rng(seed)
    n = n_core + n_fan + n_full
    parts = []
    for f in range(n_fan):
        s = int(rng.integers(fan_min, fan_max + 1))
        parts.append(np.stack([np.full(s, n_core + f), rng.choice(n_core, s, replace=False)], 1))
    for x in range(n_full):
        parts.append(np.stack([np.full(n_core, n_core + n_fan + x), np.arange(n_core)], 1))
    parts.append(rng.integers(0, n_core, (core_edges, 2)))
    parts.append(n_core + rng.integers(0, n_fan, (fan_edges, 2)))
    e = np.concatenate(parts).astype(np.int64)
    e = e[e[:, 0] != e[:, 1]]
    key = np.unique(np.minimum(e[:, 0], e[:, 1]) * n + np.maximum(e[:, 0], e[:, 1]))
    u, v = key // n, key % n
    src, dst = np.concatenate([u, v]), np.concatenate([v, u])
    order = np.lexsort((dst, src))
    src, dst = src[order], dst[order]
    offsets = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(src, minlength=n), out=offsets[1:])
    labels = rng.integers(0, k, n).astype(np.int32)
    return Graph(n=n, k=k, offsets=offsets, cols=dst.astype(np.int32), labels=labels,
                 name="dense-core-%d-%d" % (n_core, n_fan))


@dataclass
class Batch:
    """Independent graphs packed into one CSR (node ids global, labels local)."""
    graph_node_offsets: np.ndarray  # int64[G+1]
    graph_k: np.ndarray             # int32[G]
    offsets: np.ndarray             # int64[N+1]
    cols: np.ndarray                # int32[nnz]
    labels: np.ndarray              # int32[N], local to each graph
    name: str = ""

    @property
    def n_graphs(self) -> int:
        return int(self.graph_k.shape[0])

    @property
    def n(self) -> int:
        return int(self.offsets.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.cols.shape[0])

    def graph(self, i: int) -> Graph:
        """Graph i alone (node ids renumbered from 0)."""
        a, b = int(self.graph_node_offsets[i]), int(self.graph_node_offsets[i + 1])
        off = self.offsets[a:b + 1] - self.offsets[a]
        cols = self.cols[self.offsets[a]:self.offsets[b]] - a
        return Graph(n=b - a, k=int(self.graph_k[i]), offsets=off.astype(np.int64), cols=cols.astype(np.int32),
                     labels=self.labels[a:b].copy(), name="%s[%d]" % (self.name, i))


def pack(graphs, name="batch") -> Batch:
    """Pack independent graphs into one CSR (arrays filled in place, no int64 copies of the columns)."""
    G = len(graphs)
    gno = np.zeros(G + 1, np.int64)
    for i, g in enumerate(graphs):
        gno[i + 1] = gno[i] + g.n
    nnz = int(sum(g.nnz for g in graphs))
    N = int(gno[-1])
    offsets = np.zeros(N + 1, np.int64)
    cols = np.empty(nnz, np.int32)
    labels = np.empty(N, np.int32)
    base_e = 0
    for i, g in enumerate(graphs):
        a, b = int(gno[i]), int(gno[i + 1])
        offsets[a + 1:b + 1] = g.offsets[1:] + base_e
        np.add(g.cols, np.int32(a), out=cols[base_e:base_e + g.nnz], dtype=np.int32)
        labels[a:b] = g.labels
        base_e += g.nnz
    return Batch(graph_node_offsets=gno, graph_k=np.array([g.k for g in graphs], np.int32),
                 offsets=offsets, cols=cols, labels=labels, name=name)


def _batch_sizes(n_graphs: int, n_min: int, n_max: int, seed: int, first: int = 0):
    """Node counts of graphs first .. first + n_graphs - 1: graph i's is log-uniform on
    [n_min, n_max] from a hash of (seed, i), so any range of members can be drawn alone."""
    import math
    out = []
    for i in range(first, first + n_graphs):
        u = ((i * 0x9E3779B97F4A7C15 + seed * 0xBF58476D1CE4E5B9) % (1 << 64)) / float(1 << 64)
        out.append(int(round(math.exp(math.log(n_min) + u * (math.log(n_max) - math.log(n_min))))))
    return out


def _batch_member(args):
    n, seed, i, dmax = args
    k = max(2, n // 100)
    return dcsbm(n, k, 50.0 if n >= 100 * 50 else 1.0, 2.5, 8, min(dmax, n - 1), 0.2,
                 seed * 1_000_003 + i, name="g%d" % i)


def dcsbm_batch(n_graphs: int, n_min: int, n_max: int, seed: int, dmax: int = 5000, workers: int = 0) -> Batch:
    """Batched workload: graph sizes log-uniform on [n_min, n_max], each a DC-SBM shaped like
    the 1M workload (k = n/100 communities, min size 50 where possible; degrees power law 2.5
    on [8, dmax]; mixing 0.2).  Graph i uses seed (seed, i), so the batch does not depend on
    `workers` (> 1: generated by that many spawned processes)."""
    _load()
    jobs = [(n, seed, i, dmax) for i, n in enumerate(_batch_sizes(n_graphs, n_min, n_max, seed))]
    if workers and workers > 1 and n_graphs > 1:
        # spawned (not forked) workers; a worker that dies raises instead of being replaced
        import concurrent.futures as cf
        import multiprocessing as mp
        with cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
            graphs = list(ex.map(_batch_member, jobs, chunksize=max(1, n_graphs // (8 * workers))))
    else:
        graphs = [_batch_member(j) for j in jobs]
    return pack(graphs, name="dcsbm-batch-%d" % n_graphs)
