"""Pure-Python brute force of the Robust Spanning Index -- TEST INFRASTRUCTURE ONLY.

A second, independent statement of the paper's definitions (Sec. III-B), for
tiny graphs.  It enumerates every ordered node triple and builds every
diversity vector from scratch, so it shares no structure with ``rs_oracle.c``
(no per-node tables, no memoised weights, no sorted-row searches):

* ``L(u, v)``: the communities of v's neighbours other than C(u), with their
  frequencies (Eq. cont);
* ``H(L)``: Shannon entropy in bits of those frequencies (Eq. entropy);
* ``w_v(u) = H(L(u, v)) |L(u, v)|`` (Eq. weight), 0 when |L| < 2;
* ``R(u)``: sum over ordered (w, v) with u-w and w-v edges and the indicator
  (Type-I closed triad / Type-II augmented edge, C(v) != C(w), C(u) != C(w))
  of the cube root of w_v(u) w_w(v) w_w(u), divided by w_max and d(d-1)
  (Eq. RSI).
"""
from __future__ import annotations

import math
from collections import Counter


def adjacency(offsets, cols):
    n = len(offsets) - 1
    return [set(int(x) for x in cols[offsets[v]:offsets[v + 1]]) for v in range(n)]


def diversity(adj, labels, u_comm, v):
    """L(u, v) as a Counter of community -> frequency, excluding community u_comm."""
    return Counter(labels[x] for x in adj[v] if labels[x] != u_comm)


def entropy_bits(freqs):
    total = sum(freqs)
    if total == 0:
        return 0.0
    return -math.fsum((f / total) * math.log2(f / total) for f in freqs)


def weight(adj, labels, u_comm, v, alg2=False):
    """w_v(u) with |L| = the communities left (Eq. weight), or, with alg2, the number of
    communities in N(v) minus one for every column (the convention of Alg. 2)."""
    L = diversity(adj, labels, u_comm, v)
    size = len(set(labels[x] for x in adj[v])) - 1 if alg2 else len(L)
    if size < 2:
        return 0.0
    return entropy_bits(list(L.values())) * size


def is_valid_triad(adj, labels, u, w, v, strict=False):
    """1(u, w, v) with the triad types of Sec. III-A."""
    if v == u or w == u or v == w:
        return False
    if w not in adj[u] or v not in adj[w]:
        return False
    cu, cw, cv = labels[u], labels[w], labels[v]
    if cv == cw or cu == cw:
        return False
    closed = v in adj[u]
    type1 = closed and len({cu, cw, cv}) == 3
    type2 = (not closed) and cu == cv
    same_comm_closed = closed and cu == cv and not strict
    return type1 or type2 or same_comm_closed


def scores(offsets, cols, labels, k, strict=False, alg2=False):
    """All R(u) by enumeration of node triples (tiny graphs only)."""
    labels = [int(x) for x in labels]
    adj = adjacency(offsets, cols)
    n = len(adj)
    wmax = max((weight(adj, labels, c, v, alg2) for v in range(n) for c in range(k)), default=0.0)
    out = []
    for u in range(n):
        d = len(adj[u])
        if d < 2 or wmax == 0.0:
            out.append(0.0)
            continue
        terms = []
        for w in range(n):
            for v in range(n):
                if is_valid_triad(adj, labels, u, w, v, strict):
                    a = weight(adj, labels, labels[u], v, alg2)   # w_v(u)
                    b = weight(adj, labels, labels[v], w, alg2)   # w_w(v)
                    c = weight(adj, labels, labels[u], w, alg2)   # w_w(u)
                    terms.append(math.cbrt(a * b * c))
        out.append(math.fsum(terms) / wmax / (d * (d - 1)))
    return out, wmax
