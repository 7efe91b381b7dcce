"""rs_topk_noalloc: the top-K entry point that allocates no device memory.

It exists for callers that cannot allocate (memory owned by another allocator,
or loops that cannot afford cudaMalloc's synchronisation); its scratch is a
static device array.  This file is collected last so that a failure here comes
after every other test has run; it passes alone and after the others.
"""
import ctypes

import numpy as np
import pytest

import graphgen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2508_01485_gb300 as rsgpu
    L = rsgpu.lib()
    L.rs_topk_noalloc.restype = ctypes.c_int
    L.rs_topk_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p,
                                  ctypes.c_void_p, ctypes.c_void_p]
    return rsgpu


def noalloc_topk(rs, scores, k):
    ids = torch.full((k,), -1, dtype=torch.int32, device="cuda")
    vals = torch.full((k,), -1.0, dtype=torch.float64, device="cuda")
    st = rs.lib().rs_topk_noalloc(ctypes.c_void_p(scores.data_ptr()), scores.numel(), k,
                                  ctypes.c_void_p(ids.data_ptr()), ctypes.c_void_p(vals.data_ptr()),
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, rs.lib().rs_last_error().decode()
    torch.cuda.synchronize()
    return ids.cpu().numpy(), vals.cpu().numpy()


def check_against_rs_topk(rs, G, scores, k):
    ref_ids, ref_vals = G.topk(scores, k)
    ref_ids, ref_vals = ref_ids.cpu().numpy(), ref_vals.cpu().numpy()
    for _ in range(2):   # two calls in a row share the static scratch
        ids, vals = noalloc_topk(rs, scores, k)
        np.testing.assert_array_equal(ids, ref_ids)
        np.testing.assert_array_equal(vals, ref_vals)   # the same doubles, bit for bit


def test_noalloc_matches_rs_topk_on_scores(rs):
    g = graphgen.dcsbm_small(50000, seed=21, dmax=2000)
    G = rs.Graph.from_generated(g)
    scores = G.score()
    for k in (1, 100, 1000, 16384):
        check_against_rs_topk(rs, G, scores, k)


def test_noalloc_ties_and_small_inputs(rs):
    g = graphgen.sbm_2000()
    G = rs.Graph.from_generated(g)
    # many exact ties (zeros) decided by node id, and duplicated values
    s = G.score()
    check_against_rs_topk(rs, G, s, 100)          # more than the non-zero scores
    rng = np.random.default_rng(3)
    dup = torch.as_tensor(rng.integers(0, 5, size=g.n).astype(np.float64), device="cuda")
    check_against_rs_topk(rs, G, dup, 777)
    check_against_rs_topk(rs, G, dup, g.n)        # all of them


def test_noalloc_ties_above_the_scratch(rs):
    """More scores than the 16,384-key scratch and heavy ties: the radix levels must
    select down into the node-id digits (the last level's digit spans score and id)."""
    g = graphgen.dcsbm_small(100_000, seed=5)
    G = rs.Graph.from_generated(g)
    rng = np.random.default_rng(9)
    zeros = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    few = torch.as_tensor(rng.integers(0, 3, size=g.n).astype(np.float64), device="cuda")
    for s in (zeros, few):
        for k in (1, 5000, 16384):
            check_against_rs_topk(rs, G, s, k)
    G.close()


def test_noalloc_rejects_k_beyond_the_scratch(rs):
    s = torch.zeros(20000, dtype=torch.float64, device="cuda")
    ids = torch.empty(16385, dtype=torch.int32, device="cuda")
    st = rs.lib().rs_topk_noalloc(ctypes.c_void_p(s.data_ptr()), s.numel(), 16385, ctypes.c_void_p(ids.data_ptr()),
                                  None, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 1   # RS_EINVAL
    assert "16384" in rs.lib().rs_last_error().decode()
