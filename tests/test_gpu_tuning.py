"""Launch parameters, the autotuner and captured steps.

Every sum of the score is accumulated in exact fixed point, so any valid
setting of the row split points, CTA sizes and grid sizes must give the same
bits; a captured step must give the same bits as the direct calls, and must
refuse to run once the graph it recorded has changed."""
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


EXTREMES = [
    # every row above degree 1 is a hub of the global-table path, in tiny chunks
    dict(small_max=1, warp_cap=64, cta_cap=64, hub_chunk=512, p2_cta_dx=32, p1_cta_threads=128,
         p2_cta_threads=256, ctas_per_sm=1, p3_mirror=1, p1_stage=1, rows_streams=2),
    dict(small_max=16, warp_cap=128, cta_cap=512, hub_chunk=1024, p2_cta_dx=64, p1_cta_threads=512,
         p2_cta_threads=512, ctas_per_sm=16, p3_mirror=0, p1_stage=1, rows_streams=1),
    dict(small_max=32, warp_cap=512, cta_cap=512, hub_chunk=65536, p2_cta_dx=256, p1_cta_threads=256,
         p2_cta_threads=1024, ctas_per_sm=32, p3_mirror=1, p1_stage=1, rows_streams=0),
    dict(small_max=24, warp_cap=256, cta_cap=2048, hub_chunk=2048, p2_cta_dx=100, p1_cta_threads=128,
         p2_cta_threads=256, ctas_per_sm=3, p3_mirror=0, p1_stage=0, rows_streams=-1),
]


def _bits(t):
    return t.cpu().numpy().view(np.uint64)


@pytest.mark.parametrize("which", ["hubs", "dcsbm"])
def test_any_tuning_gives_the_same_bits(rs, which):
    if which == "hubs":
        g = graphgen.dcsbm(60000, 5000, 5.0, 2.1, 4, 8000, 0.5, seed=44)
    else:
        g = graphgen.dcsbm_small(50000, seed=8, dmax=3000)
    G = rs.Graph.from_generated(g)
    assert G.tuning() == rs.default_tuning()
    base = G.score()
    assert G.device_errors() == 0
    ids0, vals0 = G.topk(base, 500)
    ref = _bits(base)
    for t in EXTREMES:
        G.set_tuning(**t)
        assert G.tuning() == t
        s = G.score()
        assert G.device_errors() == 0
        np.testing.assert_array_equal(_bits(s), ref)
        ids, vals = G.topk(s, 500)
        np.testing.assert_array_equal(ids.cpu().numpy(), ids0.cpu().numpy())
    G.close()


@pytest.mark.parametrize("which", [0, 1])
def test_extreme_tuning_matches_oracle(rs, which):
    g = graphgen.sbm_2000()
    o = oracle.Oracle.from_graph(g)
    G = rs.Graph.from_generated(g)
    G.set_tuning(**EXTREMES[which])
    got = G.score().cpu().numpy()
    assert G.device_errors() == 0
    ref = o.scores()
    assert ((ref == 0) == (got == 0)).all()
    nz = ref != 0
    assert (np.abs(got[nz] - ref[nz]) / ref[nz]).max() <= 1e-12


@pytest.mark.parametrize("which", ["hubs", "dcsbm", "batch"])
def test_reverse_values_by_lookup_or_mirror_give_the_same_bits(rs, which):
    """P3 takes the reverse value of a triangle edge from the in-list of its
    higher-ranked end, or from the array the mirror pass fills: the six values
    of every triangle, hence every bit of the scores, must agree."""
    if which == "hubs":
        g = graphgen.dcsbm(60000, 5000, 5.0, 2.1, 4, 8000, 0.5, seed=44)
        G = rs.Graph.from_generated(g)
    elif which == "dcsbm":
        G = rs.Graph.from_generated(graphgen.dcsbm_small(50000, seed=8, dmax=3000))
    else:
        b = graphgen.dcsbm_batch(12, 500, 20000, seed=5, dmax=2000)
        G = rs.Graph.build_batch(b.graph_node_offsets, b.graph_k, b.offsets, b.cols, b.labels)
    assert G.tuning()["p3_mirror"] == 1
    mir = _bits(G.score())
    assert G.device_errors() == 0
    G.set_tuning(p3_mirror=0)
    look = _bits(G.score())
    assert G.device_errors() == 0
    np.testing.assert_array_equal(look, mir)
    G.set_tuning(p3_mirror=1)
    np.testing.assert_array_equal(_bits(G.score()), mir)
    G.close()


@pytest.mark.parametrize("bad", [
    dict(small_max=0), dict(small_max=33), dict(warp_cap=100), dict(warp_cap=32), dict(warp_cap=1024),
    dict(warp_cap=512, cta_cap=256), dict(cta_cap=4096), dict(hub_chunk=256), dict(hub_chunk=3000),
    dict(p2_cta_dx=31), dict(p2_cta_dx=257), dict(p1_cta_threads=64), dict(p2_cta_threads=128),
    dict(ctas_per_sm=0), dict(ctas_per_sm=33), dict(p3_mirror=2), dict(p3_mirror=-1),
    dict(p1_stage=2), dict(p1_stage=-1), dict(rows_streams=3), dict(rows_streams=-2),
])
def test_invalid_tuning_is_rejected(rs, bad):
    G = rs.Graph.from_generated(graphgen.sbm_2000())
    before = G.tuning()
    with pytest.raises(rs.RSError) as e:
        G.set_tuning(**bad)
    assert e.value.status == 1
    assert G.tuning() == before


def test_autotune_keeps_results(rs):
    g = graphgen.dcsbm_small(50000, seed=8, dmax=3000)
    G = rs.Graph.from_generated(g)
    ref = _bits(G.score())
    best, ms, tried = G.autotune(topk=100, reps=3)
    assert ms > 0 and tried >= 1
    assert G.tuning() == best
    np.testing.assert_array_equal(_bits(G.score()), ref)


def test_captured_step_matches_direct_calls(rs):
    g = graphgen.dcsbm(60000, 5000, 5.0, 2.1, 4, 8000, 0.5, seed=44)
    G = rs.Graph.from_generated(g)
    ref = G.score()
    rid, rval = G.topk(ref, 100)
    scores = torch.zeros(G.n, dtype=torch.float64, device="cuda")
    ids = torch.zeros(100, dtype=torch.int32, device="cuda")
    vals = torch.zeros(100, dtype=torch.float64, device="cuda")
    st = G.capture_step(scores, 100, ids, vals)
    l0 = G.launch_count()
    for _ in range(2):
        scores.zero_()
        ids.zero_()
        st.launch()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(_bits(scores), _bits(ref))
        np.testing.assert_array_equal(ids.cpu().numpy(), rid.cpu().numpy())
        np.testing.assert_array_equal(_bits(vals), _bits(rval))
    assert G.launch_count() > l0
    # the recorded graph changes: the step refuses to run
    G.apply_removals(nodes=rid[:5].cpu().numpy())
    with pytest.raises(rs.RSError):
        st.launch()
    st.close()
    # a new capture runs the changed graph
    ref2 = G.score()
    st2 = G.capture_step(scores)
    scores.zero_()
    st2.launch()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(_bits(scores), _bits(ref2))
    G.set_tuning(ctas_per_sm=4)
    with pytest.raises(rs.RSError):
        st2.launch()
    st2.close()
    G.close()


def test_captured_batch_step(rs):
    b = graphgen.dcsbm_batch(12, 500, 20000, seed=5, dmax=2000)
    G = rs.Graph.build_batch(b.graph_node_offsets, b.graph_k, b.offsets, b.cols, b.labels)
    ref = G.score()
    scores = torch.zeros(G.n, dtype=torch.float64, device="cuda")
    st = G.capture_step(scores)
    st.launch()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(_bits(scores), _bits(ref))
    st.close()


def test_capture_refuses_while_profiling(rs):
    G = rs.Graph.from_generated(graphgen.sbm_2000())
    scores = torch.zeros(G.n, dtype=torch.float64, device="cuda")
    G.profile_enable(True)
    with pytest.raises(rs.RSError):
        G.capture_step(scores)
    G.profile_enable(False)
    st = G.capture_step(scores)
    st.launch()
    torch.cuda.synchronize()
    st.close()
