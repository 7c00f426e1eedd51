"""The seeded input generators: the vertex shuffle is an isomorphism, and
PageRank follows the vertices (the oracle on the shuffled graph equals the
oracle on the original, permuted)."""
import numpy as np

import cpaa_inputs as ci
from oracle import oracle as O


def _edge_set(g):
    rp, cx = g.numpy()
    rows = np.repeat(np.arange(g.n), np.diff(rp))
    return rows, cx


def test_shuffle_is_an_isomorphism():
    g = ci.chung_lu(3000, 20000, seed=4)
    h = ci.shuffled(g, seed=2)
    assert h.n == g.n and h.nnz == g.nnz
    rp, _ = g.numpy()
    rp2, cx2 = h.numpy()
    # rows ascending and symmetric
    for u in range(h.n):
        row = cx2[rp2[u]:rp2[u + 1]]
        assert np.all(np.diff(row) > 0)
    r2, c2 = _edge_set(h)
    s2 = set(zip(r2.tolist(), c2.tolist()))
    assert all((b, a) in s2 for a, b in s2)
    # the degree multiset is preserved (PageRank below checks the edges map)
    d1 = np.diff(rp)
    d2 = np.diff(rp2)
    assert sorted(d1.tolist()) == sorted(d2.tolist())


def test_pagerank_follows_the_vertices():
    g = ci.chung_lu(1500, 9000, seed=5)
    h = ci.shuffled(g, seed=7)
    rp, cx = g.numpy()
    rp2, cx2 = h.numpy()
    n = g.n
    a = O.lapack_pagerank(rp, cx, np.full(n, 1.0 / n), 0.85)
    b = O.lapack_pagerank(rp2, cx2, np.full(n, 1.0 / n), 0.85)
    # same multiset of values, and degree-matched vertices carry matching values
    assert np.allclose(np.sort(a), np.sort(b), atol=1e-14)
    d1 = np.diff(rp)
    d2 = np.diff(rp2)
    for d in (int(d1.max()), int(np.median(d1))):
        assert np.allclose(np.sort(a[d1 == d]), np.sort(b[d2 == d]), atol=1e-14)


def test_shuffle_is_seeded():
    g = ci.chung_lu(500, 3000, seed=1)
    a = ci.shuffled(g, seed=3)
    b = ci.shuffled(g, seed=3)
    c = ci.shuffled(g, seed=4)
    assert np.array_equal(a.col_idx.numpy(), b.col_idx.numpy())
    assert not np.array_equal(a.col_idx.numpy(), c.col_idx.numpy())
