"""ctypes binding of librs (include/rs.h).  Argument marshalling only: every
step of the scoring path runs in the library's CUDA kernels.  PyTorch supplies
device memory and the current CUDA stream.

The library must be built (``__graft_entry__.build()``); importing this module
without it raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

RS_OK, RS_EINVAL, RS_ENOMEM, RS_ECUDA, RS_ETIMEOUT, RS_EBUDGET = range(6)
RS_VALIDATE = 1
RS_ALG2_COMPAT = 2
RS_TRIAD_STRICT = 4
RS_REORDER = 8

_lib = None

TUNING_FIELDS = ("small_max", "warp_cap", "cta_cap", "hub_chunk", "p2_cta_dx", "p1_cta_threads",
                 "p2_cta_threads", "ctas_per_sm", "p3_mirror", "p1_stage", "rows_streams")


class Tuning(ctypes.Structure):
    """rs_tuning: the scoring kernels' launch parameters (no effect on results)."""
    _fields_ = [(f, ctypes.c_int32) for f in TUNING_FIELDS]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f in TUNING_FIELDS}


def default_tuning():
    t = Tuning()
    lib().rs_default_tuning(ctypes.byref(t))
    return t.as_dict()


class RSError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("rs status %d: %s" % (status, msg))
        self.status = status


def lib():
    """Load librs.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError("librs.so is not built (%s); run __graft_entry__.build()" % path)
        L = ctypes.CDLL(path)
        P, I64, I32, U32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32
        I = ctypes.c_int
        L.rs_build_graph.restype = I
        L.rs_build_graph.argtypes = [I64, I64, P, I, P, P, I32, I, U32, P, ctypes.POINTER(P)]
        L.rs_score.restype = I
        L.rs_score.argtypes = [P, P, P, P]
        L.rs_get_interaction.restype = I
        L.rs_get_interaction.argtypes = [P, ctypes.POINTER(I64), P, P, P, P]
        L.rs_topk.restype = I
        L.rs_topk.argtypes = [P, P, I32, P, P, P]
        L.rs_apply_removals.restype = I
        L.rs_apply_removals.argtypes = [P, P, I64, P, P, I64, ctypes.POINTER(I64), P]
        L.rs_clone_graph.restype = I
        L.rs_clone_graph.argtypes = [P, ctypes.POINTER(P), P]
        L.rs_graph_info.restype = I
        L.rs_graph_info.argtypes = [P, ctypes.POINTER(I64), ctypes.POINTER(I64), ctypes.POINTER(I32),
                                    ctypes.POINTER(I32)]
        L.rs_profile_enable.restype = I
        L.rs_profile_enable.argtypes = [P, I]
        L.rs_profile_read.restype = I
        L.rs_profile_read.argtypes = [P, ctypes.POINTER(I32), P, P, P, I32]
        L.rs_launch_count.restype = I
        L.rs_launch_count.argtypes = [P, ctypes.POINTER(I64)]
        L.rs_build_batch.restype = I
        L.rs_build_batch.argtypes = [I32, P, P, I64, P, I, P, P, I, U32, P, ctypes.POINTER(P)]
        L.rs_batch_omega_max.restype = I
        L.rs_batch_omega_max.argtypes = [P, P, P]
        L.rs_default_tuning.restype = None
        L.rs_default_tuning.argtypes = [ctypes.POINTER(Tuning)]
        L.rs_get_tuning.restype = I
        L.rs_get_tuning.argtypes = [P, ctypes.POINTER(Tuning)]
        L.rs_set_tuning.restype = I
        L.rs_set_tuning.argtypes = [P, ctypes.POINTER(Tuning), P]
        L.rs_autotune.restype = I
        L.rs_autotune.argtypes = [P, P, I32, P, P, I32, P, ctypes.POINTER(Tuning), ctypes.POINTER(ctypes.c_float),
                                  ctypes.POINTER(I32)]
        L.rs_step_capture.restype = I
        L.rs_step_capture.argtypes = [P, P, I32, P, P, ctypes.POINTER(P)]
        L.rs_step_launch.restype = I
        L.rs_step_launch.argtypes = [P, P]
        L.rs_step_free.restype = None
        L.rs_step_free.argtypes = [P]
        L.rs_awcc.restype = I
        L.rs_awcc.argtypes = [P, P, I64, P, ctypes.POINTER(ctypes.c_double), P, P]
        L.rs_target_subset.restype = I
        L.rs_target_subset.argtypes = [P, P, I32, P, ctypes.POINTER(P)]
        L.rs_server_create.restype = I
        L.rs_server_create.argtypes = [P, I32, I32, I64, I32, I32, ctypes.POINTER(P)]
        L.rs_server_submit.restype = I
        L.rs_server_submit.argtypes = [P, I32, P, I64, P, P, I64, I32, ctypes.POINTER(I64)]
        L.rs_server_poll.restype = I
        L.rs_server_poll.argtypes = [P, I32, I32, P, P, P, P, P, ctypes.POINTER(I32), I32]
        L.rs_server_info.restype = I
        L.rs_server_info.argtypes = [P, ctypes.POINTER(I32), ctypes.POINTER(I64), ctypes.POINTER(I64),
                                     ctypes.POINTER(I32)]
        L.rs_server_whatif.restype = I
        L.rs_server_whatif.argtypes = [P, I32, P, I64, P, P, I64, I32, P, ctypes.POINTER(I32), P]
        L.rs_server_base_scores.restype = I
        L.rs_server_base_scores.argtypes = [P, I32, P, P]
        L.rs_server_free.restype = None
        L.rs_server_free.argtypes = [P]
        L.rs_device_errors.restype = I
        L.rs_device_errors.argtypes = [P, ctypes.POINTER(I32), P]
        L.rs_test_gx_stall.restype = I
        L.rs_test_gx_stall.argtypes = [P, I64, I64]
        L.rs_free_graph.restype = None
        L.rs_free_graph.argtypes = [P]
        L.rs_last_error.restype = ctypes.c_char_p
        L.rs_last_error.argtypes = []
        _lib = L
    return _lib


def _check(status):
    if status != RS_OK:
        raise RSError(status, lib().rs_last_error().decode())


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


class Graph:
    """A community-labelled graph resident on the GPU (owns an rs_graph)."""

    def __init__(self, handle, n, k):
        self._h = handle
        self.n = int(n)
        self.k = int(k)

    @classmethod
    def build(cls, offsets, cols, labels, k, validate=True, stream=None, alg2=False, strict=False, reorder=False):
        """rs_build_graph from numpy arrays (host) or torch CUDA tensors (device).

        offsets: int64 or int32 [n+1]; cols: int32 [nnz]; labels: int32 [n].
        alg2: RS_ALG2_COMPAT (weights with |L| = L_all - 1 for every column).
        strict: RS_TRIAD_STRICT (no closed triad with C(v) = C(u) != C(w)).
        reorder: RS_REORDER (internal ids by community, then degree; ids stay the caller's).
        """
        import torch
        on_dev = isinstance(offsets, torch.Tensor) and offsets.is_cuda
        if on_dev:
            off, col, lab = offsets.contiguous(), cols.contiguous(), labels.contiguous()
            assert col.dtype == torch.int32 and lab.dtype == torch.int32
            is64 = off.dtype == torch.int64
            p_off, p_col, p_lab = off.data_ptr(), col.data_ptr(), lab.data_ptr()
            n, nnz = off.numel() - 1, col.numel()
        else:
            off = np.ascontiguousarray(offsets)
            is64 = off.dtype == np.int64
            if not is64:
                off = np.ascontiguousarray(off, dtype=np.int32)
            col = np.ascontiguousarray(cols, dtype=np.int32)
            lab = np.ascontiguousarray(labels, dtype=np.int32)
            p_off, p_col, p_lab = off.ctypes.data, col.ctypes.data, lab.ctypes.data
            n, nnz = off.shape[0] - 1, col.shape[0]
        h = ctypes.c_void_p()
        s = _stream(stream)
        _check(lib().rs_build_graph(n, nnz, ctypes.c_void_p(p_off), 1 if is64 else 0,
                                    ctypes.c_void_p(p_col if nnz else None), ctypes.c_void_p(p_lab if n else None),
                                    int(k), 1 if on_dev else 0,
                                    (RS_VALIDATE if validate else 0) | (RS_ALG2_COMPAT if alg2 else 0)
                                    | (RS_TRIAD_STRICT if strict else 0) | (RS_REORDER if reorder else 0), s,
                                    ctypes.byref(h)))
        return cls(h, n, k)

    @classmethod
    def build_batch(cls, graph_node_offsets, graph_k, offsets, cols, labels, validate=True, stream=None):
        """rs_build_batch from host numpy arrays: graphs packed into one CSR, local labels."""
        gno = np.ascontiguousarray(graph_node_offsets, dtype=np.int64)
        gk = np.ascontiguousarray(graph_k, dtype=np.int32)
        off = np.ascontiguousarray(offsets, dtype=np.int64)
        col = np.ascontiguousarray(cols, dtype=np.int32)
        lab = np.ascontiguousarray(labels, dtype=np.int32)
        n, nnz = off.shape[0] - 1, col.shape[0]
        h = ctypes.c_void_p()
        _check(lib().rs_build_batch(gk.shape[0], gno.ctypes.data, gk.ctypes.data, nnz, ctypes.c_void_p(off.ctypes.data), 1,
                                    ctypes.c_void_p(col.ctypes.data if nnz else None),
                                    ctypes.c_void_p(lab.ctypes.data if n else None), 0,
                                    RS_VALIDATE if validate else 0, _stream(stream), ctypes.byref(h)))
        G = cls(h, n, int(gk.sum()))
        G.n_graphs = int(gk.shape[0])
        return G

    def batch_omega_max(self, stream=None):
        """w_max of every graph of the batch (numpy float64[n_graphs])."""
        out = np.zeros(getattr(self, "n_graphs", 1), np.float64)
        _check(lib().rs_batch_omega_max(self._h, out.ctypes.data, _stream(stream)))
        return out

    @classmethod
    def from_generated(cls, g, validate=True, stream=None, alg2=False, strict=False, reorder=False):
        return cls.build(g.offsets, g.cols, g.labels, g.k, validate=validate, stream=stream, alg2=alg2,
                         strict=strict, reorder=reorder)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().rs_free_graph(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        n, nnz, k, dmax = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32()
        _check(lib().rs_graph_info(self._h, ctypes.byref(n), ctypes.byref(nnz), ctypes.byref(k), ctypes.byref(dmax)))
        return {"n": n.value, "nnz_capacity": nnz.value, "k": k.value, "max_degree": dmax.value}

    def score_into(self, out, stream=None):
        """rs_score into a preallocated float64 CUDA tensor (no host synchronisation)."""
        _check(lib().rs_score(self._h, _ptr(out), None, _stream(stream)))
        return out

    def topk_into(self, scores, k, ids, vals, stream=None):
        """rs_topk into preallocated int32 / float64 CUDA tensors."""
        _check(lib().rs_topk(self._h, _ptr(scores), int(k), _ptr(ids), _ptr(vals), _stream(stream)))
        return ids, vals

    def score(self, out=None, stream=None, want_omega_max=False):
        """rs_score: R(u) for every node as a float64 CUDA tensor (and w_max if asked)."""
        import torch
        if out is None:
            out = torch.empty(self.n, dtype=torch.float64, device="cuda")
        wm = ctypes.c_double(0.0)
        _check(lib().rs_score(self._h, _ptr(out), ctypes.byref(wm) if want_omega_max else None, _stream(stream)))
        return (out, wm.value) if want_omega_max else out

    def topk(self, scores, k, stream=None):
        """rs_topk: (ids int32[k], scores float64[k]) ordered by (score desc, id asc)."""
        import torch
        ids = torch.empty(k, dtype=torch.int32, device="cuda")
        vals = torch.empty(k, dtype=torch.float64, device="cuda")
        _check(lib().rs_topk(self._h, _ptr(scores), int(k), _ptr(ids), _ptr(vals), _stream(stream)))
        return ids, vals

    def interaction(self, stream=None):
        """rs_get_interaction: (row_ptr int64[n+1], comm int32[t], count int32[t]) CUDA tensors."""
        import torch
        t = ctypes.c_int64(0)
        s = _stream(stream)
        _check(lib().rs_get_interaction(self._h, ctypes.byref(t), None, None, None, s))
        rp = torch.empty(self.n + 1, dtype=torch.int64, device="cuda")
        comm = torch.empty(max(t.value, 1), dtype=torch.int32, device="cuda")
        cnt = torch.empty(max(t.value, 1), dtype=torch.int32, device="cuda")
        _check(lib().rs_get_interaction(self._h, ctypes.byref(t), _ptr(rp), _ptr(comm), _ptr(cnt), s))
        return rp, comm[: t.value], cnt[: t.value]

    def apply_removals(self, nodes=(), edges=(), stream=None):
        """rs_apply_removals from host lists; returns the number of effective removals."""
        nodes = np.ascontiguousarray(np.asarray(nodes, dtype=np.int32).reshape(-1))
        e = np.asarray(edges, dtype=np.int32).reshape(-1, 2) if len(edges) else np.zeros((0, 2), np.int32)
        es, ed = np.ascontiguousarray(e[:, 0]), np.ascontiguousarray(e[:, 1])
        applied = ctypes.c_int64(0)
        _check(lib().rs_apply_removals(self._h, ctypes.c_void_p(nodes.ctypes.data if nodes.size else None),
                                       nodes.size, ctypes.c_void_p(es.ctypes.data if es.size else None),
                                       ctypes.c_void_p(ed.ctypes.data if ed.size else None), es.size,
                                       ctypes.byref(applied), _stream(stream)))
        return applied.value

    def profile_enable(self, enable=True):
        """Start (or stop) recording per-kernel device times; clears the record."""
        _check(lib().rs_profile_enable(self._h, 1 if enable else 0))

    def profile_read(self):
        """[(name, ms, is_kernel)] for every operation recorded since profile_enable."""
        n = ctypes.c_int32(0)
        _check(lib().rs_profile_read(self._h, ctypes.byref(n), None, None, None, 0))
        cap = n.value
        names = (ctypes.c_char_p * max(cap, 1))()
        ms = (ctypes.c_float * max(cap, 1))()
        isk = (ctypes.c_int32 * max(cap, 1))()
        _check(lib().rs_profile_read(self._h, ctypes.byref(n), names, ms, isk, cap))
        return [(names[i].decode(), float(ms[i]), bool(isk[i])) for i in range(min(cap, n.value))]

    def device_errors(self, stream=None):
        """Internal consistency flags raised by the kernels of the last rs_score (0: none)."""
        f = ctypes.c_int32(0)
        _check(lib().rs_device_errors(self._h, ctypes.byref(f), _stream(stream)))
        return f.value

    def test_gx_stall(self, tile, spin_limit=1000):
        """Test hook: tile `tile` of the G_x offset scan withholds its words and the scan's
        waits give up after spin_limit reads (tile < 0: the normal scan)."""
        _check(lib().rs_test_gx_stall(self._h, int(tile), int(spin_limit)))

    def launch_count(self):
        c = ctypes.c_int64(0)
        _check(lib().rs_launch_count(self._h, ctypes.byref(c)))
        return c.value

    def awcc(self, nodes, deg_ref=None, stream=None):
        """rs_awcc: (AWCC of the node set, |zeta(v)| per node); deg_ref fixes d(v) (absolute AWCC)."""
        v = np.ascontiguousarray(np.asarray(nodes, dtype=np.int32).reshape(-1))
        d = None if deg_ref is None else np.ascontiguousarray(np.asarray(deg_ref, dtype=np.int64).reshape(-1))
        z = np.zeros(max(v.size, 1), np.int32)
        a = ctypes.c_double(0.0)
        _check(lib().rs_awcc(self._h, ctypes.c_void_p(v.ctypes.data if v.size else None), v.size,
                             ctypes.c_void_p(d.ctypes.data) if d is not None else None, ctypes.byref(a),
                             ctypes.c_void_p(z.ctypes.data), _stream(stream)))
        return a.value, z[: v.size]

    def target_subset(self, targets, stream=None):
        """rs_target_subset: a new Graph restricted to the target communities (target i -> community i)."""
        t = np.ascontiguousarray(np.asarray(targets, dtype=np.int32).reshape(-1))
        h = ctypes.c_void_p()
        _check(lib().rs_target_subset(self._h, ctypes.c_void_p(t.ctypes.data), t.size, _stream(stream), ctypes.byref(h)))
        return Graph(h, self.n, t.size)

    def clone(self, stream=None):
        h = ctypes.c_void_p()
        _check(lib().rs_clone_graph(self._h, ctypes.byref(h), _stream(stream)))
        return Graph(h, self.n, self.k)

    # ---- launch parameters, autotuner, captured steps ---------------------------------

    def tuning(self):
        t = Tuning()
        _check(lib().rs_get_tuning(self._h, ctypes.byref(t)))
        return t.as_dict()

    def set_tuning(self, stream=None, **fields):
        """rs_set_tuning with the current parameters updated by ``fields``."""
        cur = self.tuning()
        for k in fields:
            if k not in cur:
                raise KeyError(k)
        cur.update(fields)
        t = Tuning(**cur)
        _check(lib().rs_set_tuning(self._h, ctypes.byref(t), _stream(stream)))

    def autotune(self, topk=0, reps=5, stream=None):
        """rs_autotune: returns (chosen parameters, median step ms, candidates timed)."""
        import torch
        scores = torch.empty(max(self.n, 1), dtype=torch.float64, device="cuda")
        ids = torch.empty(max(topk, 1), dtype=torch.int32, device="cuda")
        vals = torch.empty(max(topk, 1), dtype=torch.float64, device="cuda")
        best = Tuning()
        ms = ctypes.c_float(0.0)
        tried = ctypes.c_int32(0)
        _check(lib().rs_autotune(self._h, _ptr(scores), int(topk), _ptr(ids), _ptr(vals), int(reps), _stream(stream),
                                 ctypes.byref(best), ctypes.byref(ms), ctypes.byref(tried)))
        return best.as_dict(), float(ms.value), int(tried.value)

    def capture_step(self, scores, k=0, ids=None, vals=None):
        """rs_step_capture: a CUDA graph of rs_score(scores) [+ rs_topk(k) into ids / vals]."""
        h = ctypes.c_void_p()
        _check(lib().rs_step_capture(self._h, _ptr(scores), int(k), _ptr(ids), _ptr(vals), ctypes.byref(h)))
        return Step(h, self, (scores, ids, vals))


class Step:
    """A captured scoring step (owns an rs_step); keeps its graph and buffers alive."""

    def __init__(self, handle, graph, buffers):
        self._h = handle
        self._graph = graph
        self._buffers = buffers

    def launch(self, stream=None):
        if self._h is None or self._graph._h is None:
            raise RSError(RS_EINVAL, "step or its graph is closed")
        _check(lib().rs_step_launch(self._h, _stream(stream)))

    def close(self):
        if self._h is not None and self._h.value:
            lib().rs_step_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- serving ------------------------------------------------------------------------------

RS_SERVE_INCREMENTAL, RS_SERVE_FULL = 0, 1


def _removal_arrays(nodes, edges):
    nodes = np.ascontiguousarray(np.asarray(nodes, dtype=np.int32).reshape(-1))
    e = np.asarray(edges, dtype=np.int32).reshape(-1, 2) if len(edges) else np.zeros((0, 2), np.int32)
    return nodes, np.ascontiguousarray(e[:, 0]), np.ascontiguousarray(e[:, 1])


def _cp(a):
    return ctypes.c_void_p(a.ctypes.data if a.size else None)


class Server:
    """rs_server: what-if removal requests served concurrently on resident graphs.

    Takes ownership of the given Graph objects (they must not be used afterwards)."""

    def __init__(self, graphs, max_slots=8, budget_bytes=120 << 30, max_top_k=100, mode="incremental"):
        handles = (ctypes.c_void_p * len(graphs))(*[g._h for g in graphs])
        h = ctypes.c_void_p()
        m = {"incremental": RS_SERVE_INCREMENTAL, "full": RS_SERVE_FULL}[mode]
        _check(lib().rs_server_create(ctypes.cast(handles, ctypes.c_void_p), len(graphs), int(max_slots),
                                      int(budget_bytes), int(max_top_k), m, ctypes.byref(h)))
        self._h = h
        self.n = [g.n for g in graphs]
        self.max_top_k = int(max_top_k)
        for g in graphs:                      # the server owns them now
            g._h = None

    def submit(self, graph, nodes=(), edges=(), top_k=100):
        nd, es, ed = _removal_arrays(nodes, edges)
        t = ctypes.c_int64(0)
        _check(lib().rs_server_submit(self._h, int(graph), _cp(nd), nd.size, _cp(es), _cp(ed), es.size, int(top_k),
                                      ctypes.byref(t)))
        return t.value

    def poll(self, max_results=256, block=False):
        """[(ticket, status, path, ids, scores)] of the requests that finished."""
        k = self.max_top_k
        tickets = np.zeros(max_results, np.int64)
        status = np.zeros(max_results, np.int32)
        path = np.zeros(max_results, np.int32)
        ids = np.zeros(max_results * k, np.int32)
        vals = np.zeros(max_results * k, np.float64)
        n = ctypes.c_int32(0)
        _check(lib().rs_server_poll(self._h, max_results, k, tickets.ctypes.data, status.ctypes.data,
                                    path.ctypes.data, ids.ctypes.data, vals.ctypes.data, ctypes.byref(n),
                                    1 if block else 0))
        return [(int(tickets[i]), int(status[i]), int(path[i]), ids[i * k:(i + 1) * k].copy(),
                 vals[i * k:(i + 1) * k].copy()) for i in range(n.value)]

    def info(self):
        sl, b, q, f = ctypes.c_int32(0), ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int32(0)
        _check(lib().rs_server_info(self._h, ctypes.byref(sl), ctypes.byref(b), ctypes.byref(q), ctypes.byref(f)))
        return {"slots": sl.value, "bytes": b.value, "queued": q.value, "in_flight": f.value}

    def whatif(self, graph, nodes=(), edges=(), full=False, out=None, stream=None):
        """The changed graph's scores for every node (a float64 CUDA tensor) and the path taken.

        full: False (as the server chooses), True (full rescoring) or "incremental" (the
        incremental path whenever a slot's buffers hold the request)."""
        import torch
        nd, es, ed = _removal_arrays(nodes, edges)
        if out is None:
            out = torch.empty(max(self.n[graph], 1), dtype=torch.float64, device="cuda")
        p = ctypes.c_int32(-1)
        _check(lib().rs_server_whatif(self._h, int(graph), _cp(nd), nd.size, _cp(es), _cp(ed), es.size,
                                      2 if full == "incremental" else (1 if full else 0), _ptr(out), ctypes.byref(p),
                                      _stream(stream)))
        return out[: self.n[graph]], p.value

    def base_scores(self, graph, stream=None):
        import torch
        out = torch.empty(max(self.n[graph], 1), dtype=torch.float64, device="cuda")
        _check(lib().rs_server_base_scores(self._h, int(graph), _ptr(out), _stream(stream)))
        torch.cuda.synchronize()
        return out[: self.n[graph]]

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().rs_server_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
