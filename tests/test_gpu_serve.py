"""Serving: what-if removal requests on resident graphs.

The incremental path updates the exact fixed-point sums by the terms that
change, so its scores must equal, bit for bit, a full rescoring of the changed
graph (the library's own full path) -- for node removals, edge removals,
mixes, duplicates, absent edges, hubs and the empty request -- and agree with
the oracle on the changed graph.  A request's result must be the same alone
and in a mix of concurrent requests, whichever path and slot serve it."""
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
    return [graphgen.sbm_2000(),
            graphgen.dcsbm_small(20000, seed=3, dmax=800),
            graphgen.dcsbm(30000, 3000, 5.0, 2.1, 4, 4000, 0.5, seed=45),   # hub rows, many communities
            graphgen.dcsbm_small(50000, seed=6, dmax=3000, mu=0.4)]


@pytest.fixture(scope="module")
def served(rs):
    gens = _graphs()
    srv = rs.Server([rs.Graph.from_generated(g) for g in gens], max_slots=4, max_top_k=100)
    yield srv, gens
    srv.close()


def _bits(t):
    return t.cpu().numpy().view(np.uint64)


def _edges_of(g, rng, m, hot=None):
    """m existing undirected edges (optionally incident to the nodes `hot`)."""
    deg = np.diff(g.offsets)
    out = []
    while len(out) < m:
        u = int(rng.choice(hot)) if hot is not None and rng.random() < 0.7 else int(rng.integers(0, g.n))
        if deg[u] == 0:
            continue
        v = int(g.cols[g.offsets[u] + rng.integers(0, deg[u])])
        out.append((u, v))
    return out


def _requests(g, base_scores, seed):
    rng = np.random.default_rng(seed)
    top = np.argsort(-base_scores, kind="stable")[: max(1, g.n // 100)]
    deg = np.diff(g.offsets)
    hub = int(np.argmax(deg))
    reqs = [
        ((), ()),                                                      # nothing removed
        ((int(top[0]),), ()),                                          # the best node
        ((hub,), ()),                                                  # the largest hub
        (tuple(int(x) for x in rng.choice(top, min(20, len(top)), replace=False)), ()),
        ((), tuple(_edges_of(g, rng, 1))),
        ((), tuple(_edges_of(g, rng, 60, hot=top))),
        (tuple(int(x) for x in rng.integers(0, g.n, 15)), tuple(_edges_of(g, rng, 30))),
        ((int(top[0]), int(top[0])), ((0, 0), (1, 1))),               # duplicates and self-pairs
        ((), ((0, int(g.n - 1)), (2, 3))),                             # likely absent edges
        (tuple(int(x) for x in g.cols[g.offsets[hub]:g.offsets[hub + 1]][:40]), ()),   # a hub's neighbours
    ]
    return reqs


def test_incremental_equals_full_rescoring(served):
    srv, gens = served
    for gi, g in enumerate(gens):
        base = srv.base_scores(gi).cpu().numpy()
        for ri, (nodes, edges) in enumerate(_requests(g, base, 100 + gi)):
            inc, p_inc = srv.whatif(gi, nodes, edges, full="incremental")
            assert p_inc == 1, (gi, ri)
            inc = _bits(inc)
            full, p_full = srv.whatif(gi, nodes, edges, full=True)
            assert p_full == 0
            np.testing.assert_array_equal(inc, _bits(full), err_msg="graph %d request %d" % (gi, ri))
            auto, p_auto = srv.whatif(gi, nodes, edges)
            np.testing.assert_array_equal(_bits(auto), inc)
            if ri in (0, 4, 8):                 # empty, one edge, absent edges: cheap, always incremental
                assert p_auto == 1, (gi, ri)


def test_empty_request_gives_base_scores(served):
    srv, gens = served
    for gi in range(len(gens)):
        s, p = srv.whatif(gi)
        assert p == 1
        np.testing.assert_array_equal(_bits(s), _bits(srv.base_scores(gi)))


def test_incremental_matches_oracle(served):
    srv, gens = served
    g = gens[1]
    base = srv.base_scores(1).cpu().numpy()
    rng = np.random.default_rng(7)
    for nodes, edges in _requests(g, base, 7)[1:7]:
        got, p = srv.whatif(1, nodes, edges, full="incremental")
        assert p == 1
        got = got.cpu().numpy()
        removed = np.zeros(g.n, np.uint8)
        off, col, _ = oracle.remove(g.offsets, g.cols, removed, nodes, edges)
        o = oracle.Oracle(off, col, g.labels, g.k)
        ids = np.concatenate([rng.integers(0, g.n, 300), np.argsort(-got)[:20]]).astype(np.int32)
        ref = o.scores(ids)
        assert ((ref == 0) == (got[ids] == 0)).all()
        nz = ref != 0
        assert (np.abs(got[ids][nz] - ref[nz]) / ref[nz]).max() <= 1e-12
        o.close()


def _drain(srv, want):
    res = {}
    while len(res) < want:
        for t, st, path, ids, vals in srv.poll(block=True):
            res[t] = (st, path, ids, vals)
    return res


def test_same_result_alone_and_in_the_mix(served):
    srv, gens = served
    rng = np.random.default_rng(11)
    base = [srv.base_scores(i).cpu().numpy() for i in range(len(gens))]
    probe = (3, _requests(gens[3], base[3], 5)[5])
    t0 = srv.submit(probe[0], *probe[1], top_k=100)
    alone = _drain(srv, 1)[t0]
    assert alone[0] == 0
    tickets = []
    for j in range(40):
        gi = int(rng.integers(0, len(gens)))
        reqs = _requests(gens[gi], base[gi], 200 + j)
        nodes, edges = reqs[int(rng.integers(0, len(reqs)))]
        tickets.append(srv.submit(gi, nodes, edges, top_k=int(rng.integers(1, 101))))
        if j == 20:
            tp = srv.submit(probe[0], *probe[1], top_k=100)
    res = _drain(srv, len(tickets) + 1)
    mixed = res[tp]
    assert mixed[0] == 0
    np.testing.assert_array_equal(mixed[2], alone[2])
    np.testing.assert_array_equal(mixed[3].view(np.uint64), alone[3].view(np.uint64))
    assert all(res[t][0] == 0 for t in tickets)


def test_topk_of_a_request_ranks_the_changed_scores(served):
    srv, gens = served
    g = gens[2]
    base = srv.base_scores(2).cpu().numpy()
    nodes, edges = _requests(g, base, 9)[6]
    t = srv.submit(2, nodes, edges, top_k=100)
    st, path, ids, vals = _drain(srv, 1)[t]
    assert st == 0
    s, _ = srv.whatif(2, nodes, edges)
    s = s.cpu().numpy()
    np.testing.assert_array_equal(ids, oracle.topk(s, 100))
    np.testing.assert_array_equal(vals.view(np.uint64), s[ids].view(np.uint64))


def test_full_mode_server_agrees(rs, served):
    srv, gens = served
    g = gens[1]
    full = rs.Server([rs.Graph.from_generated(g)], max_slots=2, max_top_k=50, mode="full")
    base = full.base_scores(0).cpu().numpy()
    reqs = _requests(g, base, 31)
    t_full = [full.submit(0, n, e, top_k=50) for n, e in reqs]
    r_full = _drain(full, len(reqs))
    inc = rs.Server([rs.Graph.from_generated(g)], max_slots=2, max_top_k=50)
    t_inc = [inc.submit(0, n, e, top_k=50) for n, e in reqs]
    r_inc = _drain(inc, len(reqs))
    for a, b in zip(t_full, t_inc):
        assert r_full[a][0] == 0 and r_inc[b][0] == 0
        assert r_full[a][1] == 0
        np.testing.assert_array_equal(r_full[a][2], r_inc[b][2])
        np.testing.assert_array_equal(r_full[a][3].view(np.uint64), r_inc[b][3].view(np.uint64))
    full.close()
    inc.close()


def test_memory_budget(rs):
    g = graphgen.dcsbm_small(20000, seed=3, dmax=800)
    with pytest.raises(rs.RSError) as e:
        rs.Server([rs.Graph.from_generated(g)], max_slots=2, budget_bytes=1 << 20)
    assert e.value.status == 5
    # a budget that holds the incremental slots but no full copy: full requests are refused
    srv = rs.Server([rs.Graph.from_generated(g)], max_slots=1, budget_bytes=120 << 30, mode="full")
    used = srv.info()["bytes"]
    srv.close()
    srv = rs.Server([rs.Graph.from_generated(g)], max_slots=1, budget_bytes=used + (1 << 20), mode="full")
    t = srv.submit(0, (1, 2), (), top_k=10)
    st = _drain(srv, 1)[t][0]
    assert st == 5
    srv.close()


def test_bad_requests_are_rejected(served, rs):
    srv, gens = served
    with pytest.raises(rs.RSError):
        srv.submit(0, (gens[0].n,), ())
    with pytest.raises(rs.RSError):
        srv.submit(0, (), ((0, -1),))
    with pytest.raises(rs.RSError):
        srv.submit(9, (), ())
    with pytest.raises(rs.RSError):
        srv.submit(0, (), (), top_k=101)
