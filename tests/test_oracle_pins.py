"""Pins of the CPU oracle to facts fixed outside the oracle itself.

* the worked examples the paper prints (Sec. V-B), stored in
  tests/golden/paper_worked_example.json with their citation;
* closed forms derived by hand from Eq. cont / entropy / weight / RSI for two
  small graphs (a Type-I-only and a Type-II-only configuration);
* special cases the definitions fix (no cross-community neighbour, d < 2,
  k <= 2, the entropy maximum), and invariants (community relabelling, node
  permutation);
* brute force: a pure-Python enumeration of node triples (oracle/brute.py)
  on random tiny graphs;
* each pin is shown to catch a planted mistake in the brute-force statement.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import brute
from tests.conftest import csr_from_edges, random_tiny_graph

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_worked_example.json")
LOG2_3 = math.log2(3.0)


def golden():
    with open(GOLDEN) as f:
        return json.load(f)


# ---- the paper's worked examples (Sec. V-B) ------------------------------

def star3_graph(k=5):
    """Node 0 in community 0 with one neighbour in each of communities 1, 2, 3."""
    off, cols = csr_from_edges(4, [(0, 1), (0, 2), (0, 3)])
    labels = np.array([0, 1, 2, 3], np.int32)
    return off, cols, labels, k


def test_worked_example_weights():
    ex = golden()["weights_example"]
    off, cols, labels, k = star3_graph()
    o = oracle.Oracle(off, cols, labels, k)
    # removing C1 leaves counts {1, 1}: H = 1, |L| = 2 -> w = 2
    assert o.omega(0, 1) == pytest.approx(ex["omega_unnormalised_C1"], abs=1e-15)
    assert o.omega(0, 1) / ex["omega_unnormalised_C1"] * 1.0 == pytest.approx(ex["H_L1"] * 1.0)
    # a community absent from N(u) keeps all three: 3 log2 3 = 4.7549 (printed 4.754)
    w_abs = o.omega(0, 0)
    assert w_abs == pytest.approx(3 * LOG2_3, rel=1e-15)
    assert math.floor(w_abs * 1000) / 1000 == ex["omega_max_printed"]
    assert o.wmax == pytest.approx(3 * LOG2_3, rel=1e-15)
    assert round(ex["omega_unnormalised_C1"] / ex["omega_max_printed"], 2) == ex["omega_normalised_C1_printed"]
    assert round(o.omega(0, 1) / o.wmax, 2) == ex["omega_normalised_C1_printed"]


def test_worked_example_score_assembly():
    ex = golden()["score_example"]
    total = sum(oracle.triad_term(*t) for t in ex["triads"])
    r = oracle.finish(total, ex["degree"], 1.0)   # the printed weights are already normalised
    assert round(r, 3) == ex["R_printed"]
    # the pin rejects the nearby alternatives: square root, 1/d^2, unordered pairs
    assert round(sum(math.sqrt(a * b * c) for a, b, c in ex["triads"]) / 6, 3) != ex["R_printed"]
    assert round(total / 9, 3) != ex["R_printed"]
    assert round(total / 3, 3) != ex["R_printed"]


# ---- closed forms -----------------------------------------------------------

def pendant_triangle():
    """a, b, c (communities 0, 1, 2) form a triangle; each has a pendant in community 3."""
    off, cols = csr_from_edges(6, [(0, 1), (0, 2), (1, 2), (0, 3), (1, 4), (2, 5)])
    labels = np.array([0, 1, 2, 3, 3, 3], np.int32)
    return off, cols, labels, 4


# Every cross weight of a triangle node is 2 (counts {1,1} left), the absent own
# column gives w_max = 3 log2 3, each apex has two ordered Type-I triads of
# weight cbrt(8) = 2, so R = 4 / 6 / (3 log2 3) = 2 / (9 log2 3).
PENDANT_R = 2.0 / (9.0 * LOG2_3)


def open_triad():
    """u(0,C0) - w(1,C1) - v(2,C0), u not adjacent to v; w also sees C2, C3; v sees C2."""
    edges = [(0, 1), (1, 2), (1, 3), (1, 4), (2, 5), (0, 6)]
    off, cols = csr_from_edges(7, edges)
    labels = np.array([0, 1, 0, 2, 3, 2, 0], np.int32)
    return off, cols, labels, 4


# R(u): one Type-II triad (u, w, v) with w_v(C0) = 2 ({C1:1, C2:1}) and
# w_w(C0) = 2 ({C2:1, C3:1}) -> term 2; d(u) = 2; w_max = 4.5 (node w's absent
# own column, counts {2,1,1}: H = 1.5, |L| = 3).  Every other node scores 0.
OPEN_R = [2.0 / 2.0 / 4.5, 0, 0, 0, 0, 0, 0]


def test_pendant_triangle_closed_form():
    off, cols, labels, k = pendant_triangle()
    s = oracle.Oracle(off, cols, labels, k).scores()
    np.testing.assert_allclose(s, [PENDANT_R] * 3 + [0, 0, 0], rtol=1e-14, atol=0)


def test_open_triad_closed_form():
    off, cols, labels, k = open_triad()
    o = oracle.Oracle(off, cols, labels, k)
    assert o.wmax == pytest.approx(4.5, rel=1e-15)
    np.testing.assert_allclose(o.scores(), OPEN_R, rtol=1e-14, atol=0)


def test_no_cross_neighbour_scores_zero():
    # node 0 has neighbours only in its own community; its neighbours reach others
    edges = [(0, 1), (0, 2), (1, 3), (2, 4), (1, 2), (3, 4)]
    off, cols = csr_from_edges(5, edges)
    labels = np.array([0, 0, 0, 1, 2], np.int32)
    s = oracle.Oracle(off, cols, labels, 3).scores()
    assert s[0] == 0.0


def test_degree_below_two_scores_zero():
    off, cols, labels, k = pendant_triangle()
    s = oracle.Oracle(off, cols, labels, k).scores()
    assert (s[3:] == 0.0).all()          # degree-1 pendants
    off2, cols2 = csr_from_edges(3, [(0, 1)])
    s2 = oracle.Oracle(off2, cols2, np.array([0, 1, 2], np.int32), 3).scores()
    assert (s2 == 0.0).all()             # isolated node 2, degree-1 nodes 0, 1


def test_two_communities_all_zero():
    rng = np.random.default_rng(7)
    for _ in range(20):
        off, cols, labels = random_tiny_graph(rng, 10, 2, 0.5)
        o = oracle.Oracle(off, cols, labels, 2)
        assert o.wmax == 0.0
        assert (o.scores() == 0.0).all()


def test_entropy_maximum_and_uniform_equality():
    # node 0 with counts over 4 communities; w_v(c) <= |L| log2 |L|, equality iff uniform
    for counts, uniform in [((2, 2, 2, 2), True), ((3, 1, 1, 1), False), ((1, 1, 1, 5), False)]:
        edges, labels, nxt = [], [4], 1
        for c, f in enumerate(counts):
            for _ in range(f):
                edges.append((0, nxt)); labels.append(c); nxt += 1
        off, cols = csr_from_edges(nxt, edges)
        o = oracle.Oracle(off, cols, np.array(labels, np.int32), 5)
        w = o.omega(0, 4)            # community 4 is absent from N(0): all counts kept
        bound = 4 * 2.0
        assert w <= bound + 1e-15
        assert (abs(w - bound) < 1e-14) == uniform


# ---- invariants ---------------------------------------------------------------

def test_community_relabelling_invariance():
    rng = np.random.default_rng(11)
    for _ in range(10):
        off, cols, labels = random_tiny_graph(rng, 40, 6, 0.15)
        perm = rng.permutation(6).astype(np.int32)
        a = oracle.Oracle(off, cols, labels, 6)
        b = oracle.Oracle(off, cols, perm[labels], 6)
        np.testing.assert_array_equal(a.scores(), b.scores())
        assert a.wmax == b.wmax


def test_node_permutation_equivariance():
    rng = np.random.default_rng(12)
    off, cols, labels = random_tiny_graph(rng, 50, 5, 0.15)
    n = 50
    p = rng.permutation(n)           # new id of old node i is p[i]
    edges = [(p[v], p[int(x)]) for v in range(n) for x in cols[off[v]:off[v + 1]] if v < x]
    off2, cols2 = csr_from_edges(n, edges)
    labels2 = np.empty(n, np.int32); labels2[p] = labels
    s1 = oracle.Oracle(off, cols, labels, 5).scores()
    s2 = oracle.Oracle(off2, cols2, labels2, 5).scores()
    np.testing.assert_allclose(s2[p], s1, rtol=1e-13, atol=0)


# ---- brute force ---------------------------------------------------------------

@pytest.mark.parametrize("seed", range(6))
def test_oracle_matches_brute_force(seed):
    rng = np.random.default_rng(100 + seed)
    for trial in range(40):
        n = int(rng.integers(3, 13))
        k = int(rng.integers(2, 6))
        p = float(rng.uniform(0.15, 0.8))
        off, cols, labels = random_tiny_graph(rng, n, k, p)
        for strict in (False, True):
            ref, wmax = brute.scores(off, cols, labels, k, strict=strict)
            o = oracle.Oracle(off, cols, labels, k)
            assert o.wmax == pytest.approx(wmax, rel=1e-14, abs=0)
            np.testing.assert_allclose(o.scores(strict=strict), ref, rtol=1e-13, atol=1e-300)


def test_counts_match_definition():
    rng = np.random.default_rng(5)
    off, cols, labels = random_tiny_graph(rng, 30, 4, 0.3)
    ptr, comm, cnt = oracle.Oracle(off, cols, labels, 4).table()
    for v in range(30):
        expect = {}
        for x in cols[off[v]:off[v + 1]]:
            expect[int(labels[x])] = expect.get(int(labels[x]), 0) + 1
        got = dict(zip(comm[ptr[v]:ptr[v + 1]].tolist(), cnt[ptr[v]:ptr[v + 1]].tolist()))
        assert got == expect
        assert list(comm[ptr[v]:ptr[v + 1]]) == sorted(expect)


def test_rejects_invalid_graphs():
    off, cols = csr_from_edges(3, [(0, 1), (1, 2)])
    labels = np.array([0, 1, 2], np.int32)
    bad_cols = cols.copy(); bad_cols[0] = 2          # 0-2 without 2-0: asymmetric
    with pytest.raises(ValueError):
        oracle.Oracle(off, bad_cols, labels, 3)
    with pytest.raises(ValueError):
        oracle.Oracle(off, cols, np.array([0, 1, 3], np.int32), 3)   # label >= k


def test_topk_order():
    s = np.array([0.5, 0.7, 0.5, 0.0, 0.7, 0.1])
    assert oracle.topk(s, 4).tolist() == [1, 4, 0, 2]


def test_removals_match_definition():
    rng = np.random.default_rng(9)
    off, cols, labels = random_tiny_graph(rng, 25, 3, 0.3)
    removed = np.zeros(25, np.uint8)
    nodes = [3, 7, 3]
    edges = [(int(cols[off[0]]), 0)] if off[1] > off[0] else []
    edges += [(1, 1), (2, 2)]
    new_off, new_cols, applied = oracle.remove(off, cols, removed, nodes, edges)
    adj = brute.adjacency(off, cols)
    expect_applied = 2                                   # node 3 once, node 7
    for v in (3, 7):
        for x in list(adj[v]):
            adj[v].discard(x); adj[x].discard(v)
    for a, b in edges:
        if a != b and b in adj[a]:
            adj[a].discard(b); adj[b].discard(a); expect_applied += 1
    e_off, e_cols = csr_from_edges(25, [(v, x) for v in range(25) for x in adj[v]])
    np.testing.assert_array_equal(new_off, e_off)
    np.testing.assert_array_equal(new_cols, e_cols)
    assert applied == expect_applied
    assert removed[3] == 1 and removed[7] == 1
    # removing the same node again is a no-op
    _, _, again = oracle.remove(new_off, new_cols, removed, [3], [])
    assert again == 0


# ---- the pins catch planted mistakes in the brute-force statement ----------------

def _pins_pass(mod):
    """Re-evaluate the closed-form pins with the (possibly mutated) brute force."""
    ok = True
    off, cols, labels, k = pendant_triangle()
    s, _ = mod.scores(off, cols, labels, k)
    ok &= np.allclose(s, [PENDANT_R] * 3 + [0, 0, 0], rtol=1e-12, atol=0)
    off, cols, labels, k = open_triad()
    s, _ = mod.scores(off, cols, labels, k)
    ok &= np.allclose(s, OPEN_R, rtol=1e-12, atol=0)
    off, cols, labels, k = star3_graph()
    adj = mod.adjacency(off, cols)
    ok &= abs(mod.weight(adj, [int(x) for x in labels], 1, 0) - 2.0) < 1e-15
    return bool(ok)


def test_pins_hold_for_the_brute_force():
    assert _pins_pass(brute)


@pytest.mark.parametrize("mistake", ["natural_log", "no_absent_column", "sqrt", "include_v_eq_u",
                                     "swap_weight_operands", "drop_type2", "L_all_minus_1"])
def test_pins_catch_planted_mistake(monkeypatch, mistake):
    import types
    mod = types.ModuleType("mutant")
    mod.__dict__.update({k: v for k, v in brute.__dict__.items() if not k.startswith("__")})
    if mistake == "natural_log":
        mod.entropy_bits = lambda fr: -math.fsum((f / sum(fr)) * math.log(f / sum(fr)) for f in fr)
        mod.weight = lambda adj, lab, uc, v: (lambda L: 0.0 if len(L) < 2 else mod.entropy_bits(list(L.values())) * len(L))(mod.diversity(adj, lab, uc, v))
    elif mistake == "no_absent_column":
        orig = brute.scores
        def scores(off, cols, labels, k, strict=False):
            labels = [int(x) for x in labels]
            adj = brute.adjacency(off, cols)
            n = len(adj)
            present = {(v, labels[x]) for v in range(n) for x in adj[v]}
            wmax = max((brute.weight(adj, labels, c, v) for (v, c) in present), default=0.0)
            s, w_all = orig(off, cols, labels, k, strict)
            return [x * w_all / wmax if wmax else 0.0 for x in s], wmax
        mod.scores = scores
    elif mistake == "sqrt":
        mod.math = types.SimpleNamespace(**{**math.__dict__, "cbrt": math.sqrt})
    elif mistake == "include_v_eq_u":
        def tri(adj, labels, u, w, v, strict=False):
            if v == u and w in adj[u] and labels[u] != labels[w]:
                return True
            return brute.is_valid_triad(adj, labels, u, w, v, strict)
        mod.is_valid_triad = tri
    elif mistake == "swap_weight_operands":
        def weight(adj, labels, u_comm, v):
            return brute.weight(adj, labels, labels[v], v) if u_comm != labels[v] else brute.weight(adj, labels, u_comm, v)
        mod.weight = weight
    elif mistake == "drop_type2":
        def tri(adj, labels, u, w, v, strict=False):
            return brute.is_valid_triad(adj, labels, u, w, v, strict) and v in adj[u]
        mod.is_valid_triad = tri
    elif mistake == "L_all_minus_1":
        def weight(adj, labels, u_comm, v):
            L = brute.diversity(adj, labels, u_comm, v)
            allc = {labels[x] for x in adj[v]}
            size = len(allc) - 1
            return 0.0 if len(L) < 2 else brute.entropy_bits(list(L.values())) * size
        mod.weight = weight
    # rebind module-level functions so the mutant's helpers call each other
    src_scores = mod.scores
    if mistake not in ("no_absent_column",):
        def scores(offsets, cols, labels, k, strict=False, _m=mod):
            labels = [int(x) for x in labels]
            adj = _m.adjacency(offsets, cols)
            n = len(adj)
            wmax = max((_m.weight(adj, labels, c, v) for v in range(n) for c in range(k)), default=0.0)
            out = []
            for u in range(n):
                d = len(adj[u])
                if d < 2 or wmax == 0.0:
                    out.append(0.0); continue
                t = [_m.math.cbrt(_m.weight(adj, labels, labels[u], v) * _m.weight(adj, labels, labels[v], w)
                                  * _m.weight(adj, labels, labels[u], w))
                     for w in range(n) for v in range(n) if _m.is_valid_triad(adj, labels, u, w, v, strict)]
                out.append(math.fsum(t) / wmax / (d * (d - 1)))
            return out, wmax
        mod.scores = scores
    del src_scores
    assert not _pins_pass(mod)


def test_edge_only_removal_touches_no_node():
    """Removing only edges flags no node and deletes exactly those edges (both directions)."""
    rng = np.random.default_rng(19)
    off, cols, labels = random_tiny_graph(rng, 30, 3, 0.3)
    removed = np.zeros(30, np.uint8)
    u = int(np.flatnonzero(np.diff(off) > 0)[0])
    v = int(cols[off[u]])
    new_off, new_cols, applied = oracle.remove(off, cols, removed, (), [(u, v)])
    assert applied == 1
    assert not removed.any()
    adj = brute.adjacency(off, cols)
    adj[u].discard(v); adj[v].discard(u)
    e_off, e_cols = csr_from_edges(30, [(a, b) for a in range(30) for b in adj[a]])
    np.testing.assert_array_equal(new_off, e_off)
    np.testing.assert_array_equal(new_cols, e_cols)
    # and nothing at all removes nothing
    same_off, same_cols, none = oracle.remove(off, cols, np.zeros(30, np.uint8), (), ())
    assert none == 0
    np.testing.assert_array_equal(same_off, off)
    np.testing.assert_array_equal(same_cols, cols)


# Alg. 2 convention (|L| = L_all - 1 for every column).  In the pendant triangle the
# absent column of a, b, c (their own community) weighs H(1,1,1)(3 - 1) = 2 log2 3,
# which becomes w_max, and the triangle terms are unchanged (2 each, two per apex):
# R = 4 / (2 log2 3 * 3 * 2) = 1 / (3 log2 3).
ALG2_PENDANT_R = 1.0 / (3.0 * math.log2(3.0))


def test_alg2_pendant_triangle_closed_form():
    off, cols, labels, k = pendant_triangle()
    o = oracle.Oracle(off, cols, labels, k, alg2=True)
    assert o.wmax == pytest.approx(2.0 * math.log2(3.0), rel=1e-15)
    np.testing.assert_allclose(o.scores(), [ALG2_PENDANT_R] * 3 + [0, 0, 0], rtol=1e-14, atol=0)
    b, wmax = brute.scores(off, cols, labels, k, alg2=True)
    np.testing.assert_allclose(b, [ALG2_PENDANT_R] * 3 + [0, 0, 0], rtol=1e-13, atol=0)


def test_alg2_oracle_matches_brute_force():
    rng = np.random.default_rng(23)
    for _ in range(15):
        off, cols, labels = random_tiny_graph(rng, 12, 4, 0.35)
        o = oracle.Oracle(off, cols, labels, 4, alg2=True)
        b, wmax = brute.scores(off, cols, labels, 4, alg2=True)
        assert o.wmax == pytest.approx(wmax, rel=1e-13, abs=0)
        np.testing.assert_allclose(o.scores(), b, rtol=1e-12, atol=1e-300)


def test_alg2_changes_only_absent_columns():
    """With every community present around every node and no own-community gaps, the
    two conventions give the same weights."""
    off, cols = csr_from_edges(6, [(0, 1), (0, 2), (0, 3), (1, 2), (1, 4), (2, 5), (3, 4), (3, 5), (4, 5)])
    labels = np.array([0, 1, 2, 0, 1, 2], np.int32)
    a = oracle.Oracle(off, cols, labels, 3)
    b = oracle.Oracle(off, cols, labels, 3, alg2=True)
    np.testing.assert_array_equal(a.table()[0], b.table()[0])
    for v in range(6):
        for c in range(3):
            assert a.omega(v, c) == b.omega(v, c)
