"""Comparison rules shared by the GPU parity tests (host code only).

Scores: within a relative tolerance, with the same zero pattern.
Top-K: the order is (score descending, node id ascending).  GPU and oracle
scores agree to ~1e-14, not bit for bit, so two nodes whose oracle scores lie
within the tolerance of each other may legitimately come out in either order.
The rule (reading c15 of the design notes): chain the oracle's ranking into
near-tie groups (neighbours within rtol); every position outside a multi-node
group must hold the same id on both sides, a group that lies wholly inside the
first K positions must hold the same set of ids, and the group cut by position
K may hold any of its members.
"""
import numpy as np

RTOL = 1e-12


def assert_scores(got, ref, rtol=RTOL):
    got, ref = np.asarray(got), np.asarray(ref)
    assert got.shape == ref.shape
    assert ((ref == 0) == (got == 0)).all(), "zero pattern differs"
    nz = ref != 0
    rel = np.abs(got[nz] - ref[nz]) / ref[nz]
    assert rel.size == 0 or rel.max() <= rtol, "max rel err %.3e" % rel.max()
    return float(rel.max()) if rel.size else 0.0


def rank_order(ids, scores):
    """ids ordered by (score descending, id ascending)."""
    ids = np.asarray(ids, dtype=np.int64)
    s = np.asarray(scores, dtype=np.float64)
    return ids[np.lexsort((ids, -s))]


def near_tie_groups(sorted_scores, rtol=RTOL):
    """Group index of each position of a descending score list: a new group starts
    where a score is more than rtol (relative) below its predecessor."""
    s = np.asarray(sorted_scores, dtype=np.float64)
    if s.size == 0:
        return np.zeros(0, np.int64)
    scale = np.maximum(np.abs(s[:-1]), np.finfo(np.float64).tiny)
    new = (s[:-1] - s[1:]) > rtol * scale
    return np.concatenate([[0], np.cumsum(new)])


def assert_topk(gpu_ids, cand_ids, cand_ref, K, rtol=RTOL):
    """Check the GPU's top-K ids against the oracle's ranking of the candidates.

    cand_ids / cand_ref: node ids and their oracle scores; they must include every
    node that can rank in the top K (all nodes, or a superset of both lists' ids).
    Returns (number of multi-node near-tie groups met, positions that differ)."""
    gpu_ids = np.asarray(gpu_ids, dtype=np.int64)
    K = min(K, len(cand_ids))
    assert gpu_ids.shape[0] == K, "the GPU list has %d ids, expected %d" % (gpu_ids.shape[0], K)
    order = rank_order(cand_ids, cand_ref)
    ref_of = dict(zip(np.asarray(cand_ids, dtype=np.int64).tolist(), np.asarray(cand_ref).tolist()))
    missing = [int(i) for i in gpu_ids if int(i) not in ref_of]
    assert not missing, "GPU ids without an oracle score: %s" % missing[:10]
    s_sorted = np.array([ref_of[int(i)] for i in order])
    grp = near_tie_groups(s_sorted, rtol)
    sizes = np.bincount(grp)
    last = grp[K - 1]
    differ = 0
    for g in np.unique(grp[:K]):
        pos = np.flatnonzero(grp[:K] == g)
        want = order[grp == g]
        got = gpu_ids[pos]
        if sizes[g] == 1:
            assert got[0] == want[0], "position %d: GPU id %d, oracle id %d (scores %r, %r)" % (
                pos[0], got[0], want[0], ref_of.get(int(got[0])), ref_of[int(want[0])])
            continue
        if g != last:
            assert set(got.tolist()) == set(want.tolist()), "near-tie group at positions %d-%d differs" % (pos[0], pos[-1])
        else:
            assert set(got.tolist()) <= set(want.tolist()), "boundary group at positions %d-%d differs" % (pos[0], pos[-1])
        differ += int((got != want[:len(got)]).sum())
    return int((sizes[np.unique(grp[:K])] > 1).sum()), differ
