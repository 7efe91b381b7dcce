"""The seeded input generator: structure, determinism and the paper's Lemma 4."""
import hashlib
import math
import os

import numpy as np
import pytest

import graphgen

GOLDEN_HASH = os.path.join(os.path.dirname(__file__), "golden", "sbm_2000_sha256.txt")


def csr_digest(g):
    h = hashlib.sha256()
    for a in (g.offsets, g.cols, g.labels):
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def check_simple_symmetric(g):
    off, cols = g.offsets, g.cols
    assert off[0] == 0 and off[-1] == cols.shape[0]
    deg = np.diff(off)
    rows = np.repeat(np.arange(g.n, dtype=np.int64), deg)
    assert (cols >= 0).all() and (cols < g.n).all()
    assert (cols != rows).all(), "self-loop"
    same_row = rows[1:] == rows[:-1]
    assert (cols[1:][same_row] > cols[:-1][same_row]).all(), "rows not strictly ascending"
    fwd = np.sort(rows * g.n + cols)
    bwd = np.sort(cols.astype(np.int64) * g.n + rows)
    np.testing.assert_array_equal(fwd, bwd)
    assert (g.labels >= 0).all() and (g.labels < g.k).all()


def test_sbm_2000_structure_and_golden_hash():
    g = graphgen.sbm_2000()
    check_simple_symmetric(g)
    assert g.n == 2000 and g.k == 20
    d = csr_digest(g)
    # integer-only draws: the same bytes on every host
    with open(GOLDEN_HASH) as f:
        assert d == f.read().split()[0]


def test_sbm_mean_degrees():
    g = graphgen.sbm_2000()
    deg = np.diff(g.offsets)
    rows = np.repeat(np.arange(g.n), deg)
    intra = (g.labels[rows] == g.labels[g.cols]).sum() / g.n
    inter = (g.labels[rows] != g.labels[g.cols]).sum() / g.n
    assert abs(intra - 8.0) < 0.3
    assert abs(inter - 1.0) < 0.1


def test_lemma4_border_fraction():
    """Lemma 4 (Sec. V-C): with equal communities of size n_S = n_L and inter-community
    link probability p, p_border = 1 - exp(-(|V| - n_S) p); here (2000 - 100)/1900 = 1."""
    fr = []
    for seed in range(1, 6):
        g = graphgen.sbm_2000(seed)
        deg = np.diff(g.offsets)
        rows = np.repeat(np.arange(g.n), deg)
        cross = np.zeros(g.n, bool)
        cross[rows[g.labels[rows] != g.labels[g.cols]]] = True
        fr.append(cross.mean())
    expect = 1.0 - math.exp(-1.0)
    # 5 x 2000 Bernoulli(0.632) nodes: sd 0.0048
    assert abs(np.mean(fr) - expect) < 0.02


def test_determinism_and_seed_dependence():
    a = graphgen.dcsbm_small(5000, seed=4)
    b = graphgen.dcsbm_small(5000, seed=4)
    c = graphgen.dcsbm_small(5000, seed=5)
    assert csr_digest(a) == csr_digest(b)
    assert csr_digest(a) != csr_digest(c)


def test_dcsbm_shape():
    g = graphgen.dcsbm(200_000, 2000, 50.0, 2.5, 8, 2000, 0.2, seed=3)
    check_simple_symmetric(g)
    sizes = np.bincount(g.labels, minlength=g.k)
    assert sizes.sum() == g.n and sizes.min() >= 50
    assert sizes[0] == sizes.max() and (np.diff(sizes) <= 0).all()   # rank-size, largest first
    deg = np.diff(g.offsets)
    assert deg.max() <= 2000
    rows = np.repeat(np.arange(g.n), deg)
    mu = (g.labels[rows] != g.labels[g.cols]).mean()
    # mu is the floor: intra stubs beyond (community size - 1) move to inter stubs
    assert 0.18 < mu < 0.35


def test_bad_arguments():
    with pytest.raises(ValueError):
        graphgen.dcsbm(10, 20, 1.0, 2.5, 2, 5, 0.2, seed=1)   # k > n


def test_dense_core_structure():
    """The dense core: a simple symmetric CSR, seeded; fan nodes joined only to core nodes
    (and other fans), full nodes to every core node, subset sizes within their range."""
    g = graphgen.dense_core()
    check_simple_symmetric(g)
    assert csr_digest(g) == csr_digest(graphgen.dense_core())
    assert csr_digest(g) != csr_digest(graphgen.dense_core(seed=12))
    n_core, n_fan = 600, 2500
    assert g.n == n_core + n_fan + 6
    deg = np.diff(g.offsets)
    rows = np.repeat(np.arange(g.n), deg)
    to_core = np.bincount(rows[g.cols < n_core], minlength=g.n)
    fan = slice(n_core, n_core + n_fan)
    assert to_core[fan].min() >= 40 and to_core[fan].max() <= 420
    assert (to_core[n_core + n_fan:] == n_core).all()
    # the full nodes touch nothing but the core
    assert (deg[n_core + n_fan:] == n_core).all()
