"""Target-community subset mode: the graph restricted to the k largest
communities (the paper's experimental setting) equals, score for score, the
definition evaluated by the oracle on the induced subgraph with the targets
relabelled 0..k-1; the subset of all communities is the graph itself."""
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


def induced(g, targets):
    """Host definition: edges with both endpoints in the targets, target i -> community i."""
    m = -np.ones(g.k, np.int64)
    m[np.asarray(targets)] = np.arange(len(targets))
    keep_node = m[g.labels] >= 0
    rows = np.repeat(np.arange(g.n), np.diff(g.offsets))
    keep = keep_node[rows] & keep_node[g.cols]
    off = np.concatenate([[0], np.cumsum(np.bincount(rows[keep], minlength=g.n))]).astype(np.int64)
    return off, g.cols[keep].astype(np.int32), np.where(keep_node, m[g.labels], 0).astype(np.int32), keep_node


@pytest.mark.parametrize("k_top", [4, 7, 40])
def test_top_k_communities_match_oracle(rs, k_top):
    g = graphgen.dcsbm_small(20000, seed=3, dmax=800)
    targets = np.argsort(-np.bincount(g.labels, minlength=g.k), kind="stable")[:k_top]
    S = rs.Graph.from_generated(g).target_subset(targets)
    s, wmax = S.score(want_omega_max=True)
    s = s.cpu().numpy()
    off, cols, labels, inside = induced(g, targets)
    o = oracle.Oracle(off, cols, labels, k_top)
    assert abs(wmax - o.wmax) <= 1e-13 * max(o.wmax, 1e-300)
    ref = o.scores()
    assert (s[~inside] == 0).all()
    assert ((ref == 0) == (s == 0)).all()
    nz = ref != 0
    assert (np.abs(s[nz] - ref[nz]) / ref[nz]).max() <= 1e-12
    rp, comm, cnt = [x.cpu().numpy() for x in S.interaction()]
    ptr, ocomm, ocnt = o.table()
    np.testing.assert_array_equal(rp, ptr)
    np.testing.assert_array_equal(comm, ocomm)
    np.testing.assert_array_equal(cnt, ocnt)
    ids, _ = S.topk(torch.from_numpy(s).cuda(), 50)
    np.testing.assert_array_equal(ids.cpu().numpy(), oracle.topk(s, 50))


def test_all_communities_is_the_graph(rs):
    g = graphgen.dcsbm_small(20000, seed=4, dmax=800)
    G = rs.Graph.from_generated(g)
    base = G.score().cpu().numpy()
    S = G.target_subset(np.arange(g.k))
    np.testing.assert_array_equal(S.score().cpu().numpy().view(np.uint64), base.view(np.uint64))


def test_bad_targets_are_rejected(rs):
    G = rs.Graph.from_generated(graphgen.sbm_2000())
    for bad in ([0, 0], [-1], [20], []):
        with pytest.raises(rs.RSError):
            G.target_subset(bad)
