"""GPU tests of the C ABI beyond scoring parity: removals, validation,
determinism, cloning, degenerate graphs and device-resident inputs."""
import numpy as np
import pytest

import graphgen
import oracle
from tests.conftest import csr_from_edges, random_tiny_graph

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL = 1e-12


@pytest.fixture(scope="module")
def rs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2508_01485_gb300 as rsgpu
    return rsgpu


def assert_scores(got, ref, rtol=RTOL):
    got, ref = np.asarray(got), np.asarray(ref)
    assert ((ref == 0) == (got == 0)).all(), "zero pattern differs"
    nz = ref != 0
    if nz.any():
        assert (np.abs(got[nz] - ref[nz]) / ref[nz]).max() <= rtol


def table_of(G):
    rp, comm, cnt = G.interaction()
    return rp.cpu().numpy(), comm.cpu().numpy(), cnt.cpu().numpy()


def test_removals_match_oracle(rs):
    g = graphgen.dcsbm_small(20000, seed=31, dmax=800)
    G = rs.Graph.from_generated(g)
    rng = np.random.default_rng(5)
    removed = np.zeros(g.n, np.uint8)
    off, cols = g.offsets, g.cols
    for step in range(3):
        nodes = rng.integers(0, g.n, size=200).tolist()
        nodes += nodes[:20]                                   # duplicates in one call
        deg = np.diff(off)
        srcs = rng.choice(np.flatnonzero(deg > 0), size=300)
        edges = [(int(s), int(cols[off[s] + rng.integers(0, deg[s])])) for s in srcs]
        edges += [(b, a) for a, b in edges[:30]]              # both directions listed
        edges += [(int(rng.integers(0, g.n)), int(rng.integers(0, g.n))) for _ in range(50)]  # mostly absent
        applied = G.apply_removals(nodes, edges)
        off, cols, expect = oracle.remove(off, cols, removed, nodes, edges)
        assert applied == expect
        o = oracle.Oracle(off, cols, g.labels, g.k)
        rp, comm, cnt = table_of(G)
        ptr, ocomm, ocnt = o.table()
        np.testing.assert_array_equal(rp, ptr)
        np.testing.assert_array_equal(comm, ocomm)
        np.testing.assert_array_equal(cnt, ocnt)
        s, wmax = G.score(want_omega_max=True)
        assert abs(wmax - o.wmax) <= 1e-13 * o.wmax
        assert_scores(s.cpu().numpy(), o.scores())
    # removed nodes score zero and removing them again counts nothing
    assert G.apply_removals(np.flatnonzero(removed)[:10].tolist(), []) == 0


def test_removal_ids_out_of_range_rejected(rs):
    g = graphgen.sbm_2000()
    G = rs.Graph.from_generated(g)
    with pytest.raises(rs.RSError) as e:
        G.apply_removals([5, g.n], [])
    assert e.value.status == 1
    with pytest.raises(rs.RSError):
        G.apply_removals([], [(0, -1)])
    # nothing was applied by the failed calls
    rp, _, _ = table_of(G)
    assert int(rp[-1]) > 0 and G.apply_removals([], []) == 0


@pytest.mark.parametrize("case", ["asym", "unsorted", "dup", "self", "label", "offsets", "colrange"])
def test_validation_rejects(rs, case):
    off, cols = csr_from_edges(5, [(0, 1), (1, 2), (2, 3), (3, 4), (0, 4)])
    labels = np.array([0, 1, 2, 0, 1], np.int32)
    k = 3
    off, cols = off.copy(), cols.copy()
    if case == "asym":
        cols[off[0]] = 2                      # 0-2 without 2-0 (and 0-1 now one-sided)
        cols[off[0]:off[1]] = np.sort(cols[off[0]:off[1]])
    elif case == "unsorted":
        cols[off[0]:off[1]] = cols[off[0]:off[1]][::-1].copy()
    elif case == "dup":
        cols[off[0] + 1] = cols[off[0]]
    elif case == "self":
        cols[off[1]] = 1
    elif case == "label":
        labels = labels.copy(); labels[2] = 3
    elif case == "offsets":
        off[2] = off[1] - 1
    elif case == "colrange":
        cols[-1] = 5
    with pytest.raises(rs.RSError) as e:
        rs.Graph.build(off, cols, labels, k, validate=True)
    assert e.value.status == 1


def test_validation_finds_one_sided_edges_in_a_large_graph(rs):
    """The symmetry check must catch a single one-sided entry among millions: an edge
    dropped in one direction, and one entry re-pointed (every degree unchanged)."""
    g = graphgen.dcsbm_small(50000, seed=8, dmax=3000)
    rs.Graph.build(g.offsets, g.cols, g.labels, g.k, validate=True).close()
    rng = np.random.default_rng(3)
    deg = np.diff(g.offsets)
    for case in ("dropped", "repointed"):
        u = int(rng.choice(np.nonzero(deg >= 3)[0]))
        row = g.cols[g.offsets[u]:g.offsets[u + 1]]
        if case == "dropped":
            cols = np.delete(g.cols, g.offsets[u] + 1)
            off = g.offsets.copy()
            off[u + 1:] -= 1
        else:
            # replace one neighbour v of u by a non-neighbour w, keeping the row sorted
            v = int(row[1])
            w = next(x for x in range(row[0] + 1, row[2]) if x != u and x not in row) if row[2] - row[0] > 2 \
                else None
            if w is None:
                continue
            cols = g.cols.copy()
            new_row = np.sort(np.where(row == v, w, row))
            cols[g.offsets[u]:g.offsets[u + 1]] = new_row
            off = g.offsets
        with pytest.raises(rs.RSError) as e:
            rs.Graph.build(off, cols, g.labels, g.k, validate=True)
        assert e.value.status == 1 and "reverse" in str(e.value)


def test_deterministic_and_clone(rs):
    g = graphgen.dcsbm_small(50000, seed=8, dmax=3000)
    G = rs.Graph.from_generated(g)
    a = G.score().cpu().numpy()
    b = G.score().cpu().numpy()
    np.testing.assert_array_equal(a.view(np.uint64), b.view(np.uint64))
    C = G.clone()
    c = C.score().cpu().numpy()
    np.testing.assert_array_equal(a.view(np.uint64), c.view(np.uint64))
    # the clone is independent of later removals on the original
    G.apply_removals([0, 1, 2], [])
    np.testing.assert_array_equal(C.score().cpu().numpy().view(np.uint64), a.view(np.uint64))


def test_degenerate_graphs(rs):
    # isolated nodes only
    G = rs.Graph.build(np.zeros(6, np.int64), np.zeros(0, np.int32), np.arange(5, dtype=np.int32), 5)
    s, wmax = G.score(want_omega_max=True)
    assert (s.cpu().numpy() == 0).all() and wmax == 0.0
    ids, vals = G.topk(s, 5)
    assert ids.cpu().numpy().tolist() == [0, 1, 2, 3, 4]
    # one community: every weight is zero
    off, cols = csr_from_edges(4, [(0, 1), (1, 2), (2, 3), (3, 0)])
    G = rs.Graph.build(off, cols, np.zeros(4, np.int32), 1)
    assert (G.score().cpu().numpy() == 0).all()
    # a single node
    G = rs.Graph.build(np.zeros(2, np.int64), np.zeros(0, np.int32), np.zeros(1, np.int32), 1)
    assert G.score().cpu().numpy().tolist() == [0.0]
    # an empty graph
    G = rs.Graph.build(np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0, np.int32), 1)
    assert G.score().numel() == 0
    with pytest.raises(rs.RSError):
        G.topk(G.score(), 1)


def test_device_inputs_and_int32_offsets(rs):
    rng = np.random.default_rng(77)
    off, cols, labels = random_tiny_graph(rng, 300, 6, 0.05)
    ref = oracle.Oracle(off, cols, labels, 6).scores()
    d_off = torch.as_tensor(off.astype(np.int32), device="cuda")
    d_col = torch.as_tensor(cols, device="cuda")
    d_lab = torch.as_tensor(labels, device="cuda")
    G = rs.Graph.build(d_off, d_col, d_lab, 6)
    assert_scores(G.score().cpu().numpy(), ref)
    G2 = rs.Graph.build(off.astype(np.int32), cols, labels, 6)
    assert_scores(G2.score().cpu().numpy(), ref)


def test_high_community_count_hubs(rs):
    """Hub rows with many distinct communities (k = 5000, degrees up to 8000)."""
    g = graphgen.dcsbm(60000, 5000, 5.0, 2.1, 4, 8000, 0.5, seed=44)
    o = oracle.Oracle.from_graph(g)
    G = rs.Graph.from_generated(g)
    s, wmax = G.score(want_omega_max=True)
    assert abs(wmax - o.wmax) <= 1e-13 * o.wmax
    assert_scores(s.cpu().numpy(), o.scores())
    info = G.info()
    assert info["max_degree"] == int(np.diff(g.offsets).max())


def test_profile_and_launch_count(rs):
    g = graphgen.sbm_2000()
    G = rs.Graph.from_generated(g)
    G.profile_enable(True)
    before = G.launch_count()
    s = G.score()
    G.topk(s, 10)
    prof = G.profile_read()
    G.profile_enable(False)
    kernels = [p for p in prof if p[2]]
    assert G.launch_count() - before == len(kernels) > 5
    assert all(ms >= 0 for _, ms, _ in prof)
