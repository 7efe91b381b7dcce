"""The Alg. 2 weight convention (RS_ALG2_COMPAT: |L| = L_all - 1 for every
column) against the oracle with the same option, and through the serving
path (incremental = full rescoring, bit for bit)."""
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


@pytest.mark.parametrize("gen", [lambda: graphgen.sbm_2000(),
                                 lambda: graphgen.dcsbm_small(20000, seed=3, dmax=800),
                                 lambda: graphgen.dcsbm(30000, 3000, 5.0, 2.1, 4, 4000, 0.5, seed=45)])
def test_alg2_matches_oracle(rs, gen):
    g = gen()
    G = rs.Graph.from_generated(g, alg2=True)
    s, wmax = G.score(want_omega_max=True)
    s = s.cpu().numpy()
    o = oracle.Oracle.from_graph(g, alg2=True)
    assert abs(wmax - o.wmax) <= 1e-13 * max(o.wmax, 1e-300)
    rng = np.random.default_rng(3)
    ids = np.concatenate([rng.integers(0, g.n, 2000), np.argsort(-s)[:50]]).astype(np.int32)
    ref = o.scores(ids)
    assert ((ref == 0) == (s[ids] == 0)).all()
    nz = ref != 0
    assert (np.abs(s[ids][nz] - ref[nz]) / ref[nz]).max() <= 1e-12


def test_alg2_pendant_triangle_closed_form(rs):
    """The absent own-community column becomes w_max = 2 log2 3: R = 1 / (3 log2 3)."""
    from tests.conftest import csr_from_edges
    import math
    off, cols = csr_from_edges(6, [(0, 1), (1, 2), (0, 2), (0, 3), (1, 4), (2, 5)])
    labels = np.array([0, 1, 2, 3, 3, 3], np.int32)
    s, wmax = rs.Graph.build(off, cols, labels, 4, alg2=True).score(want_omega_max=True)
    assert wmax == pytest.approx(2.0 * math.log2(3.0), rel=1e-15)
    np.testing.assert_allclose(s.cpu().numpy(), [1.0 / (3.0 * math.log2(3.0))] * 3 + [0, 0, 0], rtol=1e-13, atol=0)
    s0, w0 = rs.Graph.build(off, cols, labels, 4).score(want_omega_max=True)
    assert w0 == pytest.approx(3.0 * math.log2(3.0), rel=1e-15)


def test_alg2_serving_incremental_equals_full(rs):
    g = graphgen.dcsbm_small(20000, seed=3, dmax=800)
    srv = rs.Server([rs.Graph.from_generated(g, alg2=True)], max_slots=1, max_top_k=10)
    base = srv.base_scores(0).cpu().numpy()
    top = np.argsort(-base)[:20]
    for nodes, edges in [((int(top[0]),), ()), (tuple(int(x) for x in top[:5]), ((1, int(g.cols[g.offsets[1]])),))]:
        inc, p = srv.whatif(0, nodes, edges, full="incremental")
        full, _ = srv.whatif(0, nodes, edges, full=True)
        assert p == 1
        np.testing.assert_array_equal(inc.cpu().numpy().view(np.uint64), full.cpu().numpy().view(np.uint64))
    srv.close()
