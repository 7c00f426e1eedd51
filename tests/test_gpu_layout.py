"""Layout parameters (cpaa_graph_create_ex) and their autotuner.

Every layout computes the same method (Algorithm 1); only the order of each
row's sum changes.  So every candidate layout must give the oracle's result
within the FP64 bound, and a batch must still equal its single solves bit for
bit on any one layout."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import cpaa_inputs as ci
from oracle import oracle as O
from tests.gpu_util import solve

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2112_01743_gb300 as pkg
    return pkg


@pytest.fixture(scope="module")
def graph():
    # hub rows above every tested threshold, long chunks and a ragged tail
    g = ci.chung_lu(60000, 1_500_000, seed=12)
    rp, cx = g.numpy()
    return g, rp, cx


LAYOUTS = [
    {},                                                        # defaults
    {"sort_window": 32},                                       # no reordering within chunks
    {"sort_window": 4096, "long_chunk": 1},                    # every chunk a CTA item
    {"hub_degree": 32, "hub_tile": 256},                       # many hub rows, short tiles
    {"hub_degree": 32, "hub_tile": 1 << 20},                   # one tile per hub row
    {"hub_degree": 1 << 20},                                   # no hub rows at all
    {"hub_degree": 64, "hub_tile": 512, "long_chunk": 16, "sort_window": 256},
    {"long_chunk": 1 << 20, "sort_window": 64},                # no long chunks
]


@pytest.mark.parametrize("li", range(len(LAYOUTS)), ids=[str(x) or "default" for x in LAYOUTS])
def test_every_layout_matches_the_oracle(pkg, graph, li):
    g, rp, cx = graph
    lp = LAYOUTS[li]
    G = pkg.Graph(g.row_ptr.cuda(), g.col_idx.cuda(), n=g.n, layout=lp)
    lay = G.layout()
    for k, v in lp.items():
        assert lay[k] == v, (k, lay)
    if lp.get("hub_degree") == 1 << 20:
        assert lay["hub_rows"] == 0
    if lp.get("long_chunk") == 1:
        assert lay["long_chunks"] == lay["chunks"]
    n = g.n
    p = np.zeros(n)
    p[[0, 7, 30000, n - 1]] = 0.25   # a hub, a heavy row and two light ones
    M = 23
    ref = O.cpaa(rp, cx, p, 0.85, M)
    for prec, bound, rel in ((pkg.CPAA_F64, 1e-12, False), (pkg.CPAA_DF64, 1e-12, False),
                             (pkg.CPAA_F32, 1e-6, True)):
        pi, info = solve(pkg, G, p, 0.85, 0.0, precision=prec, fixed_rounds=M)
        err = np.abs(pi - ref).sum()
        if rel:
            err /= np.abs(ref).sum()
        assert err <= bound, (lp, prec, err)
    # a batch equals its single solves on this layout
    P = ci.seed_dense(n, ci.seed_vectors(n, 5, seed=6))
    Pd = torch.as_tensor(P).cuda()
    PI = torch.empty_like(Pd)
    infos = G.solve_batch(5, Pd, np.full(5, 0.85), 1e-7, PI, precision=pkg.CPAA_F32, batch_width=4)
    torch.cuda.synchronize()
    for b in (0, 4):
        single, info = solve(pkg, G, P[b], 0.85, 1e-7, precision=pkg.CPAA_F32)
        assert infos[b].rounds == info.rounds
        assert np.array_equal(PI[b].cpu().numpy(), single)
    G.close()


def test_autotune_picks_a_layout_and_caches_it(pkg, graph):
    g, rp, cx = graph
    G = pkg.Graph(g.row_ptr.cuda(), g.col_idx.cuda(), n=g.n, autotune=True)
    lay = G.layout()
    assert lay["tuned"] == 1 and lay["tune_candidates"] >= 3
    n = g.n
    p = np.zeros(n)
    p[[3, 59999]] = 0.5
    pi, info = solve(pkg, G, p, 0.85, 1e-9)
    ref = O.cpaa(rp, cx, p, 0.85, info.rounds)
    assert np.abs(pi - ref).sum() <= 1e-12
    # the same graph again: the cached pick, the same layout
    G2 = pkg.Graph(g.row_ptr.cuda(), g.col_idx.cuda(), n=g.n, autotune=True)
    lay2 = G2.layout()
    for k in ("hub_degree", "hub_tile", "long_chunk", "sort_window", "hub_rows", "long_chunks", "tuned",
              "tune_candidates"):
        assert lay2[k] == lay[k], k
    pi2, info2 = solve(pkg, G2, p, 0.85, 1e-9)
    assert info2.rounds == info.rounds and np.array_equal(pi, pi2)
    G.close()
    G2.close()


def test_autotune_on_the_lattice(pkg):
    """A graph with no hub rows and no long chunks: only the sort window is
    a real choice; the tuned layout still matches the oracle."""
    g = ci.grid_deleted(300, 310, 0.2, seed=5)
    rp, cx = g.numpy()
    G = pkg.Graph(g.row_ptr.cuda(), g.col_idx.cuda(), n=g.n, autotune=True,
                  layout={"tune_precision": pkg.CPAA_F64})
    lay = G.layout()
    assert lay["tuned"] == 1 and lay["hub_rows"] == 0
    p = np.full(g.n, 1.0 / g.n)
    pi, info = solve(pkg, G, p, 0.85, 1e-10)
    ref = O.cpaa(rp, cx, p, 0.85, info.rounds)
    assert np.abs(pi - ref).sum() <= 1e-12
    G.close()


def test_row_longer_than_a_short_chunk_may_hold(pkg):
    """A non-hub row of more than 65532 entries (hub threshold and long-chunk
    threshold both above it) goes to a long chunk, because a warp's rows read a
    2-byte degree; every format still matches the oracle, and the short chunks'
    factor tables cover the degrees they meet."""
    g = ci.star(70001)                       # centre of degree 70001, leaves of degree 1
    rp, cx = g.numpy()
    G = pkg.Graph(g.row_ptr.cuda(), g.col_idx.cuda(), n=g.n,
                  layout={"hub_degree": 100000, "long_chunk": 1 << 20})
    lay = G.layout()
    assert lay["hub_rows"] == 0 and lay["long_chunks"] == 1, lay
    p = np.zeros(g.n)
    p[[0, 1, 5000, g.n - 1]] = 0.25
    M = 15
    ref = O.cpaa(rp, cx, p, 0.85, M)
    # The centre's row is one long chunk: each of a CTA's 8 warps adds a slice
    # of about 8750 of its entries in sequence.  DF64's significands hold about
    # 48 bits, so that sum is about 1e-12 off in L1 here (measured 1.02e-12),
    # and FP32's about 1e-5 (measured 1.2e-5): their bounds on this row are
    # ten times those of the bench graphs, whose rows this long are hub rows
    # summed by shuffle trees.
    for prec, bound, rel in ((pkg.CPAA_F64, 1e-12, False), (pkg.CPAA_DF64, 1e-11, False),
                             (pkg.CPAA_F32, 1e-4, True), (pkg.CPAA_BF16, 5e-2, True)):
        pi, info = solve(pkg, G, p, 0.85, 0.0, precision=prec, fixed_rounds=M)
        err = np.abs(pi - ref).sum()
        if rel:
            err /= np.abs(ref).sum()
        assert err <= bound, (prec, err)
    G.close()
