"""The strict triad reading (RS_TRIAD_STRICT: a closed triangle (u, w, v) with
C(v) = C(u) != C(w) is not a triad) against the oracle with the same reading,
on graphs that exercise every Type-II kernel (tiles, warps, tables, CTAs, hubs)."""
import numpy as np
import pytest

import graphgen
import oracle
from tests.conftest import random_tiny_graph

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2508_01485_gb300 as rsgpu
    return rsgpu


def _check(rs, off, cols, labels, k, sample=None, alg2=False):
    G = rs.Graph.build(off, cols, labels, k, strict=True, alg2=alg2)
    s, wmax = G.score(want_omega_max=True)
    assert G.device_errors() == 0
    s = s.cpu().numpy()
    o = oracle.Oracle(off, cols, labels, k, alg2=alg2)
    ids = np.arange(len(off) - 1, dtype=np.int32) if sample is None else sample
    ref = o.scores(ids, strict=True)
    got = s[ids]
    assert ((ref == 0) == (got == 0)).all()
    nz = ref != 0
    if nz.any():
        assert (np.abs(got[nz] - ref[nz]) / ref[nz]).max() <= 1e-12
    return s


def test_strict_tiny_graphs(rs):
    rng = np.random.default_rng(31)
    for _ in range(20):
        off, cols, labels = random_tiny_graph(rng, 40, 3, 0.25)
        _check(rs, off, cols, labels, 3)


@pytest.mark.parametrize("gen", [lambda: graphgen.sbm_2000(),
                                 lambda: graphgen.dcsbm_small(20000, seed=3, dmax=800),
                                 lambda: graphgen.dcsbm(30000, 3000, 5.0, 2.1, 4, 4000, 0.5, seed=45)])
def test_strict_matches_oracle(rs, gen):
    g = gen()
    rng = np.random.default_rng(5)
    base = rs.Graph.from_generated(g).score().cpu().numpy()
    sample = np.unique(np.concatenate([rng.integers(0, g.n, 1500), np.argsort(-base)[:50],
                                       np.argsort(-np.diff(g.offsets))[:10]])).astype(np.int32)
    s = _check(rs, g.offsets, g.cols, g.labels, g.k, sample)
    assert (s <= base * (1 + 1e-12) + 1e-300).all()      # strict only removes triads


def test_strict_with_alg2(rs):
    g = graphgen.dcsbm_small(20000, seed=9, dmax=800)
    _check(rs, g.offsets, g.cols, g.labels, g.k, np.arange(0, g.n, 7, dtype=np.int32), alg2=True)
