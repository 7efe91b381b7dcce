"""Crafted rows with skewed community counts, where Eq. H_optimal's form
H = log2 Y - (sum f log2 f) / Y cancels (reading c14): a centre node v whose
neighbour counts are (d-1, 1), (d-2, 1, 1) or (d/2, d/2-1, 1) for d = 1e3, 1e4
and 1e5, with v's own community absent from its neighbours or present.

Leaving one community out of such a row leaves counts like (d-2, 1), whose
entropy is ~(log2 d)/d, 1.8e-4 at d = 1e5.  The graph is built so that some
scores consist only of terms carrying these weights:

* the count-1 leaves (and, for (d-1, 1), one leaf of the large community) form
  triangles with v, so their scores hold w_v(c) of the left-out columns;
* when v's own community is among its neighbours' (the second community of the
  pattern), those triangles carry s_v = w_v(C(v))^(1/3) of the own column;
* a witness node in C(v), not adjacent to v, shares two large-community leaves
  with v, so its score holds s_v as a Type-II term.

Every touched leaf has two private neighbours in fresh communities, so that its
own weights are not degenerate.  The GPU's scores (table rows up to the hub
path at d = 1e5) must match the oracle's within 1e-12 and the interaction
table bit for bit."""
import numpy as np
import pytest

import oracle
from tests.parity import RTOL, assert_scores

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

A, B, C, V = 0, 1, 2, 3
FRESH = 40                     # pairs of fresh communities for private neighbours


def patterns(d):
    return {"d-1,1": [(A, d - 1), (B, 1)],
            "d-2,1,1": [(A, d - 2), (B, 1), (C, 1)],
            "d/2,d/2-1,1": [(A, d // 2), (B, d // 2 - 1), (C, 1)]}


def skewed_graph(ds=(1000, 10_000, 100_000)):
    edges, labels = [], []
    fresh = [0]

    def node(c):
        labels.append(c)
        return len(labels) - 1

    def private_pair(x):
        j = fresh[0] % FRESH
        fresh[0] += 1
        for c in (4 + 2 * j, 5 + 2 * j):
            edges.append((x, node(c)))

    centres = []
    for d in ds:
        for name, pat in patterns(d).items():
            for own in ("absent", "present"):
                v = node(V if own == "absent" else B)
                centres.append((d, name, own, v))
                leaves = {}
                for c, cnt in pat:
                    leaves[c] = [node(c) for _ in range(cnt)]
                    edges.extend((v, x) for x in leaves[c])
                ones = [leaves[c][0] for c, cnt in pat if cnt == 1]
                tri = ones if len(ones) >= 2 else ones + [leaves[A][0]]
                if name == "d/2,d/2-1,1":
                    tri = [leaves[C][0], leaves[A][0], leaves[B][0]]
                for i in range(len(tri)):
                    for j in range(i + 1, len(tri)):
                        edges.append((tri[i], tri[j]))
                for x in tri:
                    private_pair(x)
                wit = node(labels[v])
                for x in leaves[A][-2:]:
                    edges.append((wit, x))
                    private_pair(x)
    n = len(labels)
    e = np.array(edges, dtype=np.int64)
    e = np.concatenate([e, e[:, ::-1]])
    e = e[np.lexsort((e[:, 1], e[:, 0]))]
    off = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(e[:, 0], minlength=n), out=off[1:])
    return off, e[:, 1].astype(np.int32), np.array(labels, np.int32), 4 + 2 * FRESH, centres


@pytest.fixture(scope="module")
def rs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2508_01485_gb300 as rsgpu
    return rsgpu


def test_skewed_rows_match_oracle(rs):
    off, cols, labels, k, centres = skewed_graph()
    assert np.diff(off).max() == 100_000
    G = rs.Graph.build(off, cols, labels, k)
    s, wmax = G.score(want_omega_max=True)
    s = s.cpu().numpy()
    oracle.set_threads(0)
    o = oracle.Oracle(off, cols, labels, k)
    ref = o.scores()
    assert abs(wmax - o.wmax) <= 1e-13 * o.wmax
    # the skewed weights are tiny: each centre's left-out columns carry ~(log2 d)/d
    for d, name, own, v in centres:
        if name == "d-2,1,1":
            w = o.omega(v, C)
            assert 0 < w < 4 * np.log2(d) / d
    assert (ref > 0).sum() >= 3 * len(centres)
    err = assert_scores(s, ref, RTOL)
    print("max relative error %.2e over %d non-zero scores" % (err, int((ref > 0).sum())))
    rp, comm, cnt = G.interaction()
    ptr, ocomm, ocnt = o.table()
    np.testing.assert_array_equal(rp.cpu().numpy(), ptr)
    np.testing.assert_array_equal(comm.cpu().numpy(), ocomm)
    np.testing.assert_array_equal(cnt.cpu().numpy(), ocnt)
    G.close()
