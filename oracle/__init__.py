"""CPU oracle for Robust Spanning Index scoring -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
``cpu_baseline`` / ``--impl reference`` leg may import this package.  It
shares no code with the CUDA library under ``paper_2508_01485_gb300/`` and
neither imports the other; the seeded graph generator (``graphgen``) is the
only module both sides use.

Two independent evaluations of the paper's definitions (Sec. III-B, Eq. cont,
entropy, weight, RSI and the indicator):

* ``rs_oracle.c`` (loaded here through ctypes): fp64 with compensated sums,
  used for every size the tests need;
* ``brute.py``: a pure-Python literal triple loop over node triples, for tiny
  graphs only, used to check the C oracle.

Parity pins (what fixes the oracle independently of itself) live in
``tests/test_oracle_pins.py``; functions without a pin are named there.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rs_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "librs_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile rs_oracle.c into oracle/_build/librs_oracle.so (idempotent)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P, I64, I32, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
        lib.rso_new.restype = P
        lib.rso_new.argtypes = [I64, I32, P, P, P, ctypes.c_int, ctypes.c_int, ctypes.c_char_p, ctypes.c_int]
        lib.rso_free.argtypes = [P]
        lib.rso_wmax.restype = D; lib.rso_wmax.argtypes = [P]
        lib.rso_table_size.restype = I64; lib.rso_table_size.argtypes = [P]
        lib.rso_table.argtypes = [P, P, P, P]
        lib.rso_omega.restype = D; lib.rso_omega.argtypes = [P, I32, I32]
        lib.rso_scores.argtypes = [P, P, I64, ctypes.c_int, P]
        lib.rso_scores_all.argtypes = [P, ctypes.c_int, P]
        lib.rso_topk.argtypes = [P, I64, I64, P]
        lib.rso_triad_term.restype = D; lib.rso_triad_term.argtypes = [D, D, D]
        lib.rso_finish.restype = D; lib.rso_finish.argtypes = [D, I64, D]
        lib.rso_set_threads.restype = ctypes.c_int; lib.rso_set_threads.argtypes = [ctypes.c_int]
        lib.rso_remove.restype = I64
        lib.rso_remove.argtypes = [I64, P, P, P, P, I64, P, P, I64, P, P]
        _lib = lib
    return _lib


def set_threads(n: int = 0) -> int:
    """Host threads for the loops over nodes (0: all cores).  Results are bit-identical
    for any count: every node is computed by one thread in a fixed order."""
    return int(_load().rso_set_threads(int(n)))


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


class Oracle:
    """Oracle state for one graph: community tables, weights and w_max."""

    def __init__(self, offsets, cols, labels, k, validate=True, alg2=False):
        lib = _load()
        self._off = _c(offsets, np.int64)
        self._col = _c(cols, np.int32) if len(cols) else np.zeros(1, np.int32)
        self._lab = _c(labels, np.int32) if len(labels) else np.zeros(1, np.int32)
        self.n = int(self._off.shape[0] - 1)
        self.k = int(k)
        err = ctypes.create_string_buffer(256)
        self._h = lib.rso_new(self.n, self.k, self._off.ctypes.data, self._col.ctypes.data,
                              self._lab.ctypes.data, 1 if validate else 0, 1 if alg2 else 0, err, 256)
        if not self._h:
            raise ValueError("oracle: " + err.value.decode())

    @classmethod
    def from_graph(cls, g, validate=True, alg2=False):
        return cls(g.offsets, g.cols, g.labels, g.k, validate, alg2)

    def close(self):
        if getattr(self, "_h", None):
            _load().rso_free(self._h)
            self._h = None

    def __del__(self):
        self.close()

    @property
    def wmax(self) -> float:
        """Largest weight w_v(c) over all nodes v and communities c."""
        return float(_load().rso_wmax(self._h))

    def table(self):
        """Per-node community counts f_v(c): (row_ptr int64[n+1], comm int32[t], count int32[t])."""
        lib = _load()
        t = int(lib.rso_table_size(self._h))
        ptr = np.empty(self.n + 1, np.int64)
        comm = np.empty(max(t, 1), np.int32)
        cnt = np.empty(max(t, 1), np.int32)
        lib.rso_table(self._h, ptr.ctypes.data, comm.ctypes.data, cnt.ctypes.data)
        return ptr, comm[:t], cnt[:t]

    def omega(self, v: int, c: int) -> float:
        """Un-normalised weight w_v(c) (Eq. weight with C(u) = c)."""
        return float(_load().rso_omega(self._h, int(v), int(c)))

    def scores(self, ids=None, strict=False) -> np.ndarray:
        """R(u) for the given node ids (all nodes if None)."""
        lib = _load()
        if ids is None:
            out = np.empty(self.n, np.float64)
            lib.rso_scores_all(self._h, 1 if strict else 0, out.ctypes.data)
            return out
        ids = _c(ids, np.int32)
        out = np.empty(ids.shape[0], np.float64)
        if ids.shape[0]:
            lib.rso_scores(self._h, ids.ctypes.data, ids.shape[0], 1 if strict else 0, out.ctypes.data)
        return out


def topk(scores, K: int) -> np.ndarray:
    """Ids of the K best nodes, ordered by (score descending, id ascending)."""
    s = _c(scores, np.float64)
    K = min(int(K), s.shape[0])
    out = np.empty(max(K, 1), np.int32)
    if s.shape[0]:
        _load().rso_topk(s.ctypes.data, s.shape[0], K, out.ctypes.data)
    return out[:K]


def triad_term(w_vu: float, w_wv: float, w_wu: float) -> float:
    return float(_load().rso_triad_term(w_vu, w_wv, w_wu))


def finish(total: float, d: int, wmax: float) -> float:
    return float(_load().rso_finish(total, d, wmax))


def remove(offsets, cols, removed, nodes=(), edges=()):
    """Apply node and edge removals to a host CSR copy.

    Returns (new_offsets, new_cols, applied).  ``removed`` is a uint8[n]
    array of removed-node flags, updated in place.
    """
    lib = _load()
    off = _c(offsets, np.int64)
    col = _c(cols, np.int32) if len(cols) else np.zeros(1, np.int32)
    n = off.shape[0] - 1
    assert removed.dtype == np.uint8 and removed.shape[0] == n and removed.flags.c_contiguous
    nn = len(nodes)
    nodes = _c(nodes, np.int32) if nn else np.zeros(1, np.int32)   # a valid pointer; nn = 0 removes none
    e = np.asarray(edges, dtype=np.int32).reshape(-1, 2) if len(edges) else np.zeros((0, 2), np.int32)
    es = _c(e[:, 0], np.int32) if e.shape[0] else np.zeros(1, np.int32)
    ed = _c(e[:, 1], np.int32) if e.shape[0] else np.zeros(1, np.int32)
    out_off = np.empty(n + 1, np.int64)
    out_col = np.empty(max(int(off[-1]), 1), np.int32)
    applied = lib.rso_remove(n, off.ctypes.data, col.ctypes.data, removed.ctypes.data,
                             nodes.ctypes.data, nn, es.ctypes.data, ed.ctypes.data, e.shape[0],
                             out_off.ctypes.data, out_col.ctypes.data)
    return out_off, out_col[: int(out_off[-1])].copy(), int(applied)
