"""rs_topk on synthetic score vectors: the K best nodes by (score descending,
id ascending) must be exactly those of a stable host sort, whatever the value
distribution -- all scores equal (every radix level down to the id bits), few
distinct values, zeros, values over many binades, K at its limits, n at and
around the size the selection sorts directly."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2508_01485_gb300 as rsgpu
    return rsgpu


def _isolated(rs, n):
    """A graph of n isolated nodes: its workspace serves score vectors of length n."""
    return rs.Graph.build(np.zeros(n + 1, np.int64), np.zeros(0, np.int32), np.zeros(n, np.int32), 1)


def _scores(dist, n, rng):
    if dist == "ties":
        return np.full(n, 0.25)
    if dist == "zeros":
        s = np.zeros(n)
        s[rng.choice(n, min(n, 7), replace=False)] = rng.random(min(n, 7))
        return s
    if dist == "few":
        return rng.choice(np.array([0.0, 1e-3, 0.5, 0.5000000000000001, 1.0]), n)
    if dist == "binades":
        return np.ldexp(rng.random(n) + 0.5, rng.integers(-300, 300, n))
    return rng.random(n)


@pytest.mark.parametrize("n", [1, 1000, 16384, 16385, 300000, 1000000])
@pytest.mark.parametrize("dist", ["ties", "zeros", "few", "binades", "uniform"])
def test_topk_equals_stable_sort(rs, n, dist):
    rng = np.random.default_rng(n * 7 + len(dist))
    s = _scores(dist, n, rng)
    G = _isolated(rs, n)
    d = torch.as_tensor(s, device="cuda")
    for K in sorted({1, min(n, 1000), min(n, 16384)}):
        ids, vals = G.topk(d, K)
        want = oracle.topk(s, K)
        np.testing.assert_array_equal(ids.cpu().numpy(), want)
        np.testing.assert_array_equal(vals.cpu().numpy().view(np.uint64), s[want].view(np.uint64))
    G.close()
