"""Sparse-frontier early rounds (CPAA_SPARSE_FRONTIER).

T_k p vanishes outside the k-hop ball of p's support (the recurrence of
Sec. 4.1 adds one hop per round), so the early rounds may skip every work item
outside that ball.  The results must be the same bits as without the
frontier, and match the oracle within the usual bounds, for seeds of degree 1
and 2 and for a hub seed, in every number format, alone, in a batch and in the
server."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import cpaa_inputs as ci
from oracle import oracle as O
from tests.gpu_util import solve, upload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2112_01743_gb300 as pkg
    return pkg


def _pendant_graph():
    """Chung-Lu (60k vertices) plus three pendant vertices (degree 1) hung on
    a hub, a middling vertex and a light one."""
    g = ci.chung_lu(60000, 700000, seed=15)
    rp, cx = g.numpy()
    rows = np.repeat(np.arange(g.n), np.diff(rp))
    keep = rows < cx
    e = np.stack([rows[keep], cx[keep]], 1)
    extra = np.array([[g.n, 0], [g.n + 1, 30000], [g.n + 2, 59999]])
    return ci.from_edges(g.n + 3, np.concatenate([e, extra]), name="chung_lu_pendants")


@pytest.fixture(scope="module")
def graphs(pkg):
    gl = {"pendants": _pendant_graph(), "grid": ci.grid_deleted(600, 700, 0.2, seed=8)}
    up = {k: upload(pkg, g) for k, g in gl.items()}
    yield gl, up
    for G in up.values():
        G.close()


PRECS = [("F64", 1e-12, False), ("DF64", 1e-12, False), ("F32", 1e-6, True), ("BF16", None, True)]


def _seeds(name, g):
    rp, _ = g.numpy()
    deg = np.diff(rp)
    if name == "pendants":
        n = g.n
        return {"degree 1": [n - 1], "degree 1 (on a hub)": [n - 3], "degree 2": [int(np.argmin(deg[:n - 3]))],
                "hub": [int(np.argmax(deg))], "mixed": [n - 2, 7, int(np.argmax(deg))]}
    return {"corner": [0], "middle": [350 * 700 + 300], "two": [5, 419_000]}


@pytest.mark.parametrize("name", ["pendants", "grid"])
@pytest.mark.parametrize("prec,bound,rel", PRECS, ids=[p[0] for p in PRECS])
def test_frontier_same_bits_and_oracle(pkg, graphs, name, prec, bound, rel):
    gl, up = graphs
    g, G = gl[name], up[name]
    rp, cx = g.numpy()
    P = getattr(pkg, "CPAA_" + prec)
    for what, seeds in _seeds(name, g).items():
        p = np.zeros(g.n)
        p[seeds] = 1.0 / len(seeds)
        a, ia = solve(pkg, G, p, 0.85, 1e-8, precision=P)
        b, ib = solve(pkg, G, p, 0.85, 1e-8, precision=P, frontier=True)
        assert ia.rounds == ib.rounds, what
        assert np.array_equal(a, b), (what, np.abs(a - b).max())
        if bound is not None:
            ref = O.cpaa(rp, cx, p, 0.85, ia.rounds)
            err = np.abs(b - ref).sum() / (np.abs(ref).sum() if rel else 1.0)
            assert err <= bound, (what, err)


def test_frontier_few_rounds_normalisations_and_history(pkg, graphs):
    """M below, at and above the frontier rounds; both normalisations; the
    a-posteriori rule (whose per-round sums read the skipped items' zero slots)
    and the per-round history."""
    gl, up = graphs
    g, G = gl["grid"], up["grid"]
    rp, cx = g.numpy()
    p = np.zeros(g.n)
    p[[1000, 1001]] = 0.5
    for M in (1, 2, 7, 8, 9, 20):
        for norm in (0, 1):
            a, _ = solve(pkg, G, p, 0.85, 0.0, fixed_rounds=M, normalize=norm)
            b, _ = solve(pkg, G, p, 0.85, 0.0, fixed_rounds=M, normalize=norm, frontier=True)
            assert np.array_equal(a, b), (M, norm)
            ref = O.cpaa(rp, cx, p, 0.85, M, normalize=norm)
            assert np.abs(b - ref).sum() <= 1e-12
    h1, h2 = np.zeros(400), np.zeros(400)
    a, ia = solve(pkg, G, p, 0.85, 1e-8, stop_rule=pkg.CPAA_STOP_POSTERIORI, history=h1)
    b, ib = solve(pkg, G, p, 0.85, 1e-8, stop_rule=pkg.CPAA_STOP_POSTERIORI, history=h2, frontier=True)
    assert ia.rounds == ib.rounds and np.array_equal(a, b) and np.array_equal(h1, h2)
    _, mass, l1 = O.cpaa(rp, cx, p, 0.85, ia.rounds, history=True)
    M = ia.rounds
    assert np.abs(h2[0:2 * (M + 1):2] - mass).max() < 1e-12
    # uniform p: the ball is everything from the start
    u = np.full(g.n, 1.0 / g.n)
    a, _ = solve(pkg, G, u, 0.85, 1e-8)
    b, _ = solve(pkg, G, u, 0.85, 1e-8, frontier=True)
    assert np.array_equal(a, b)


def test_frontier_batch_columns_equal_single(pkg, graphs):
    gl, up = graphs
    for name in ("pendants", "grid"):
        g, G = gl[name], up[name]
        seeds = ci.seed_vectors(g.n, 6, max_seeds=3, seed=21)
        P = ci.seed_dense(g.n, seeds)
        Pd = torch.as_tensor(P).cuda()
        for prec in (pkg.CPAA_F64, pkg.CPAA_F32):
            PI = torch.empty_like(Pd)
            infos = G.solve_batch(6, Pd, np.full(6, 0.85), 1e-7, PI, precision=prec, batch_width=4,
                                  frontier=True)
            torch.cuda.synchronize()
            for b in (0, 3, 5):
                single, info = solve(pkg, G, P[b], 0.85, 1e-7, precision=prec)
                assert infos[b].rounds == info.rounds
                assert np.array_equal(PI[b].cpu().numpy(), single), (name, prec, b)


@pytest.mark.parametrize("prec", ["F32", "F64"])
def test_frontier_server_alone_equals_mix_and_plain_server(pkg, prec):
    """A server with the frontier on (graphs of >= 2^22 entries): a query that
    starts an empty tile runs its early rounds on the frontier; it equals the
    same query in a mix (where it joins running ones) and on a server without
    the frontier, bit for bit, and matches the oracle."""
    gl = [ci.grid_deleted(1500, 1600, 0.2, seed=4), ci.chung_lu(300000, 2_600_000, seed=16)]
    G = [upload(pkg, x) for x in gl]
    assert all(x.nnz >= 1 << 22 for x in G)
    P = getattr(pkg, "CPAA_" + prec)
    queries = [(0, np.array([17], dtype=np.int32), 0.85), (0, np.array([1_200_000, 5], dtype=np.int32), 0.5),
               (1, np.array([299_999], dtype=np.int32), 0.85), (1, np.array([0, 4], dtype=np.int32), 0.95)]
    res = {}
    try:
        for fr in (False, True):
            S = pkg.Server(8 << 30, precision=P, frontier=fr)
            ids = [S.add_graph(x, 8) for x in G]
            alone = []
            for gi, sd, c in queries:  # one at a time: each starts an empty tile
                pi = np.empty(gl[gi].n)
                st, info = S.wait(S.submit(ids[gi], sd, None, c, 1e-7), pi, timeout_us=300_000_000)
                assert st == pkg.CPAA_OK
                alone.append((pi, info.rounds))
            # all at once, twice over: later ones join running tiles
            tickets = [S.submit(ids[gi], sd, None, c, 1e-7) for gi, sd, c in queries + queries]
            mix = []
            for (gi, sd, c), t in zip(queries + queries, tickets):
                pi = np.empty(gl[gi].n)
                st, info = S.wait(t, pi, timeout_us=300_000_000)
                assert st == pkg.CPAA_OK
                mix.append((pi, info.rounds))
            S.close()
            res[fr] = (alone, mix)
        for fr in (False, True):
            alone, mix = res[fr]
            for i in range(len(queries)):
                for pi, r in (mix[i], mix[i + len(queries)], res[not fr][0][i]):
                    assert r == alone[i][1]
                    assert np.array_equal(pi, alone[i][0]), (fr, i)
        tol = 1e-12 if prec == "F64" else 1e-6
        for i, (gi, sd, c) in enumerate(queries):
            rp, cx = gl[gi].numpy()
            p = np.zeros(gl[gi].n)
            p[sd] = 1.0 / len(sd)
            pi, M = res[True][0][i]
            ref = O.cpaa(rp, cx, p, c, M)
            err = np.abs(pi - ref).sum() / (1.0 if prec == "F64" else np.abs(ref).sum())
            assert err <= tol, (i, err)
    finally:
        for x in G:
            x.close()
