"""Parity on the full batched workload: 4,096 graphs with log-uniform sizes
(500 to 200,000 nodes) packed into one CSR of ~2.6e9 entries, past the 2^31
mark, so every CSR position on the path needs 64 bits.  Sampled graphs --
the smallest, the largest, the one whose entries straddle position 2^31 and
random others -- are checked against the oracle: their own w_max and sampled
node scores, including each graph's best nodes."""
import os

import numpy as np
import pytest

import graphgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2508_01485_gb300 as rsgpu
    b = graphgen.dcsbm_batch(4096, 500, 200_000, seed=4, dmax=5000, workers=min(16, os.cpu_count() or 1))
    G = rsgpu.Graph.build_batch(b.graph_node_offsets, b.graph_k, b.offsets, b.cols, b.labels, validate=False)
    s = G.score().cpu().numpy()
    flags = G.device_errors()
    wmax = G.batch_omega_max()
    G.close()
    return b, s, flags, wmax


def _sample(b):
    sizes = np.diff(b.graph_node_offsets)
    edge_start = b.offsets[b.graph_node_offsets[:-1]]
    edge_end = b.offsets[b.graph_node_offsets[1:]]
    straddle = np.flatnonzero((edge_start <= 2**31) & (edge_end > 2**31))
    rng = np.random.default_rng(404)
    pick = {int(np.argmin(sizes)), int(np.argmax(sizes))} | set(straddle.tolist())
    pick |= set(int(i) for i in rng.choice(b.n_graphs, 6, replace=False))
    # and the last graph, whose entries end at nnz
    pick.add(b.n_graphs - 1)
    return sorted(pick), straddle


def test_batch_crosses_2_31_entries(setup):
    b, s, flags, wmax = setup
    assert b.nnz > 2**31
    assert flags == 0


def test_sampled_graphs_full_batch(setup):
    b, s, flags, wmax = setup
    pick, straddle = _sample(b)
    assert len(straddle) == 1
    rng = np.random.default_rng(405)
    for i in pick:
        gi = b.graph(i)
        a0 = int(b.graph_node_offsets[i])
        o = oracle.Oracle.from_graph(gi, validate=False)
        assert abs(wmax[i] - o.wmax) <= 1e-13 * max(o.wmax, 1e-300), i
        local = s[a0:a0 + gi.n]
        best = np.argsort(-local, kind="stable")[:5]
        ids = np.concatenate([rng.integers(0, gi.n, size=40), best]).astype(np.int32)
        ref = o.scores(ids)
        got = local[ids]
        assert ((ref == 0) == (got == 0)).all(), i
        nz = ref != 0
        if nz.any():
            assert (np.abs(got[nz] - ref[nz]) / ref[nz]).max() <= 1e-12, i
        o.close()
