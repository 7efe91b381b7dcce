"""Batched scoring: independent graphs packed into one CSR give each graph the
scores (and w_max) it gets alone -- against the oracle per graph, and bit for
bit against the single-graph GPU path."""
import numpy as np
import pytest

import graphgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2508_01485_gb300 as rsgpu
    return rsgpu


def test_batch_matches_oracle_and_single_graphs(rs):
    b = graphgen.dcsbm_batch(24, 500, 20000, seed=9, dmax=2000)
    G = rs.Graph.build_batch(b.graph_node_offsets, b.graph_k, b.offsets, b.cols, b.labels)
    s = G.score().cpu().numpy()
    assert G.device_errors() == 0
    wmax = G.batch_omega_max()
    koff = np.concatenate([[0], np.cumsum(b.graph_k)[:-1]])
    rp, comm, cnt = [x.cpu().numpy() for x in G.interaction()]
    for i in range(b.n_graphs):
        gi = b.graph(i)
        a, z = int(b.graph_node_offsets[i]), int(b.graph_node_offsets[i + 1])
        o = oracle.Oracle.from_graph(gi)
        assert abs(wmax[i] - o.wmax) <= 1e-13 * max(o.wmax, 1e-300)
        ref = o.scores()
        got = s[a:z]
        assert ((ref == 0) == (got == 0)).all()
        nz = ref != 0
        if nz.any():
            assert (np.abs(got[nz] - ref[nz]) / ref[nz]).max() <= 1e-12
        # the same bits as scoring the graph alone
        alone = rs.Graph.from_generated(gi).score().cpu().numpy()
        np.testing.assert_array_equal(got.view(np.uint64), alone.view(np.uint64))
        # counts, with community ids offset by the graphs before
        ptr, ocomm, ocnt = o.table()
        np.testing.assert_array_equal(rp[a:z + 1] - rp[a], ptr)
        np.testing.assert_array_equal(comm[rp[a]:rp[z]], ocomm + koff[i])
        np.testing.assert_array_equal(cnt[rp[a]:rp[z]], ocnt)


def test_batch_rejects_cross_graph_edges(rs):
    g1, g2 = graphgen.sbm(2, 10, 0.5, 0.2, 1), graphgen.sbm(2, 10, 0.5, 0.2, 2)
    b = graphgen.pack([g1, g2])
    cols = b.cols.copy()
    # rewire one edge of graph 0 into graph 1 (both directions, so symmetry holds)
    u = 0
    v = int(cols[b.offsets[u]])
    w = 25                                             # a node of graph 1 not adjacent to u
    from tests.conftest import csr_from_edges
    edges = [(x, int(y)) for x in range(b.n) for y in b.cols[b.offsets[x]:b.offsets[x + 1]] if x < y]
    edges = [(a, c) for a, c in edges if (a, c) != (u, v)] + [(u, w)]
    off, cols = csr_from_edges(b.n, edges)
    with pytest.raises(rs.RSError) as e:
        rs.Graph.build_batch(b.graph_node_offsets, b.graph_k, off, cols, b.labels)
    assert e.value.status == 1
    labels = b.labels.copy(); labels[25] = 2           # graph 1 has k = 2
    with pytest.raises(rs.RSError):
        rs.Graph.build_batch(b.graph_node_offsets, b.graph_k, b.offsets, b.cols, labels)
