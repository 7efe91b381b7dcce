"""AWCC of the paper's robustness analysis (Sec. VI-C): 1/|S| sum |zeta(v)|/d(v)
for the top scorers, before and after random edge removals (absolute AWCC keeps
the original degrees), against the definition evaluated on the host."""
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


def zeta(off, cols, labels, v):
    return len(set(int(labels[x]) for x in cols[off[v]:off[v + 1]]))


def awcc_host(off, cols, labels, S, deg):
    s = 0.0
    for v, d in zip(S, deg):
        if d > 0:
            s += zeta(off, cols, labels, v) / float(d)
    return s / len(S)


def test_awcc_of_top_scorers_under_edge_removal(rs):
    g = graphgen.dcsbm_small(20000, seed=3, dmax=800)
    G = rs.Graph.from_generated(g)
    s = G.score().cpu().numpy()
    S = oracle.topk(s, 25)
    deg0 = np.diff(g.offsets)[S]
    a0, z0 = G.awcc(S)
    assert list(z0) == [zeta(g.offsets, g.cols, g.labels, v) for v in S]
    assert a0 == awcc_host(g.offsets, g.cols, g.labels, S, deg0)
    rng = np.random.default_rng(12)
    off, cols = g.offsets, g.cols
    removed = np.zeros(g.n, np.uint8)
    for step in range(3):                      # 5% of the edges at a time
        deg = np.diff(off)
        src = rng.choice(np.flatnonzero(deg > 0), size=int(0.05 * len(cols) / 2))
        edges = [(int(u), int(cols[off[u] + rng.integers(0, deg[u])])) for u in src]
        G.apply_removals(edges=edges)
        off, cols, _ = oracle.remove(off, cols, removed, (), edges)
        with pytest.raises(rs.RSError):
            G.awcc(S)                          # not scored since the change
        G.score()
        a, z = G.awcc(S, deg_ref=deg0)
        assert list(z) == [zeta(off, cols, g.labels, v) for v in S]
        assert a == awcc_host(off, cols, g.labels, S, deg0)
        assert a <= a0 + 1e-15                 # removals only lose communities
