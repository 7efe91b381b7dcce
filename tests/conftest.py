import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: full-size workload")


def csr_from_edges(n, edges):
    """Symmetric CSR (int64 offsets, sorted int32 cols) from an undirected edge list."""
    import numpy as np
    adj = [set() for _ in range(n)]
    for a, b in edges:
        if a != b:
            adj[a].add(b)
            adj[b].add(a)
    off = np.zeros(n + 1, np.int64)
    cols = []
    for v in range(n):
        row = sorted(adj[v])
        cols.extend(row)
        off[v + 1] = off[v] + len(row)
    return off, np.asarray(cols, dtype=np.int32)


def random_tiny_graph(rng, n, k, p):
    """Erdos-Renyi graph with uniform random labels (test helper)."""
    import numpy as np
    edges = [(i, j) for i in range(n) for j in range(i + 1, n) if rng.random() < p]
    off, cols = csr_from_edges(n, edges)
    labels = rng.integers(0, k, size=n).astype(np.int32)
    return off, cols, labels
