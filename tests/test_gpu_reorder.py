"""RS_REORDER: the library renumbers the nodes internally (by community, then
degree), and every id the caller sees or passes stays the caller's own.  Scores
must match the oracle in the caller's ids (1e-12 relative: the orientation of
G_x follows the internal ids, so a triangle's terms may be formed in another
operand order), and everything else -- top-K of the returned scores, the
interaction table, removals, AWCC, clones, target subsets, captured steps --
must match the same graph built without the flag."""
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


def _graphs():
    return {"sbm": graphgen.sbm_2000(),
            "dcsbm": graphgen.dcsbm_small(50000, seed=8, dmax=3000),
            "hubs": graphgen.dcsbm(30000, 3000, 5.0, 2.1, 4, 4000, 0.5, seed=45)}


def _close(got, ref):
    assert ((ref == 0) == (got == 0)).all()
    nz = ref != 0
    assert (np.abs(got[nz] - ref[nz]) / ref[nz]).max() <= 1e-12


@pytest.mark.parametrize("which", ["sbm", "dcsbm", "hubs"])
def test_reordered_scores_match_the_oracle(rs, which):
    g = _graphs()[which]
    R = rs.Graph.from_generated(g, reorder=True)
    got = R.score().cpu().numpy()
    assert R.device_errors() == 0
    ref = oracle.Oracle.from_graph(g).scores()
    _close(got, ref)
    ids, vals = R.topk(torch.as_tensor(got, device="cuda"), 100)
    assert ids.cpu().numpy().tolist() == oracle.topk(got, 100).tolist()
    R.close()


def test_reordered_interaction_table_is_in_the_callers_rows(rs):
    g = _graphs()["dcsbm"]
    P = rs.Graph.from_generated(g)
    R = rs.Graph.from_generated(g, reorder=True)
    for a, b in zip(P.interaction(), R.interaction()):
        np.testing.assert_array_equal(a.cpu().numpy(), b.cpu().numpy())
    P.close()
    R.close()


def test_reordered_removals_awcc_clone_subset_and_step(rs):
    g = _graphs()["hubs"]
    P = rs.Graph.from_generated(g)
    R = rs.Graph.from_generated(g, reorder=True)
    base = P.score().cpu().numpy()
    _close(R.score().cpu().numpy(), base)
    # AWCC of the same node set, in the caller's ids
    nodes = np.argsort(-base)[:200].astype(np.int32)
    a_p, z_p = P.awcc(nodes)
    a_r, z_r = R.awcc(nodes)
    assert a_p == a_r
    np.testing.assert_array_equal(z_p, z_r)
    # a clone keeps the numbering
    C = R.clone()
    _close(C.score().cpu().numpy(), base)
    C.close()
    # a target subset of a reordered graph
    targets = np.arange(0, g.k, 3, dtype=np.int32)[:40]
    SP = P.target_subset(targets)
    SR = R.target_subset(targets)
    _close(SR.score().cpu().numpy(), SP.score().cpu().numpy())
    SP.close()
    SR.close()
    # removals given in the caller's ids
    deg = np.diff(g.offsets)
    hub = int(np.argmax(deg))
    edges = np.array([[hub, g.cols[g.offsets[hub]]], [int(nodes[5]), g.cols[g.offsets[nodes[5]]]]], np.int32)
    for G in (P, R):
        assert G.apply_removals(nodes=nodes[:10], edges=edges) > 0
    after = P.score().cpu().numpy()
    _close(R.score().cpu().numpy(), after)
    off, col, _ = oracle.remove(g.offsets, g.cols, np.zeros(g.n, np.uint8), nodes[:10], [tuple(e) for e in edges])
    _close(R.score().cpu().numpy(), oracle.Oracle(off, col, g.labels, g.k).scores())
    # a captured step on the reordered graph writes the same scores
    scores = torch.zeros(R.n, dtype=torch.float64, device="cuda")
    st = R.capture_step(scores)
    st.launch()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(scores.cpu().numpy().view(np.uint64), R.score().cpu().numpy().view(np.uint64))
    st.close()
    P.close()
    R.close()


def test_server_refuses_reordered_graphs(rs):
    R = rs.Graph.from_generated(graphgen.sbm_2000(), reorder=True)
    with pytest.raises(rs.RSError) as e:
        rs.Server([R], max_slots=1)
    assert e.value.status == 1
