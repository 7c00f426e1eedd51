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


def test_chung_lu_distinct_keeps_the_first_distinct_pairs():
    """chung_lu(distinct=True): exactly the first E distinct non-loop pairs in
    draw order, plus the ring; the same graph whatever the draw chunk."""
    import torch
    from cpaa_inputs import rng
    n, E = 5000, 30000
    g = ci.chung_lu(n, E, seed=3, distinct=True, chunk=1 << 12)
    w = np.arange(1, n + 1, dtype=np.float64) ** (-1.0 / 1.1)
    cum = np.cumsum(w)
    cum_int = np.floor(cum / cum[-1] * float(2 ** 53)).astype(np.int64)
    cum_int[-1] = 2 ** 53
    cum_t = torch.as_tensor(cum_int)
    idx = rng.arange(0, 4 * E, "cpu")
    u = torch.searchsorted(cum_t, rng.u53(3, 0, idx), right=True).tolist()
    v = torch.searchsorted(cum_t, rng.u53(3, 1, idx), right=True).tolist()
    seen, order = set(), []
    for a, b in zip(u, v):
        if a != b and (min(a, b), max(a, b)) not in seen:
            seen.add((min(a, b), max(a, b)))
            order.append((min(a, b), max(a, b)))
            if len(order) == E:
                break
    assert len(order) == E
    ring = {(min(i, (i + 1) % n), max(i, (i + 1) % n)) for i in range(n)}
    rows, cx = _edge_set(g)
    got = set(zip(rows[rows < cx].tolist(), cx[rows < cx].tolist()))
    assert got == set(order) | ring
    h = ci.chung_lu(n, E, seed=3, distinct=True, chunk=1 << 15)
    assert torch.equal(g.row_ptr, h.row_ptr) and torch.equal(g.col_idx, h.col_idx)


def test_with_self_loops_adds_one_loop_per_vertex():
    """Every vertex gains exactly one self-loop (none doubled where one was
    already present); the other entries are unchanged."""
    g = ci.from_edges(6, [(0, 1), (1, 2), (2, 2), (3, 4), (4, 5), (5, 0)])
    h = ci.with_self_loops(g)
    rp, cx = g.numpy()
    rp2, cx2 = h.numpy()
    for u in range(g.n):
        old = set(cx[rp[u]:rp[u + 1]].tolist())
        new = cx2[rp2[u]:rp2[u + 1]].tolist()
        assert new == sorted(old | {u})
