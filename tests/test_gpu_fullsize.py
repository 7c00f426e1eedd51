"""Parity at the benchmark configurations' full sizes (GPU + host oracle).

The oracle runs every row on the host cores for the same number of rounds the
GPU ran (rows are independent inside a round, Sec. 4.1), so the comparison is
element by element over the whole vector."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import cpaa_inputs as ci
from oracle import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2112_01743_gb300 as pkg
    return pkg


def _solve(pkg, G, p, c, tol, **kw):
    pi = torch.empty_like(p)
    info = G.solve(p, c, tol, pi, **kw)
    torch.cuda.synchronize()
    return pi, info


def _l1(a, ref):
    return float(np.abs(a.cpu().numpy() - ref).sum())


def test_config_10k_eq41_rounds(pkg):
    """10,000-vertex Chung-Lu, uniform p, c = 0.85, run until ERR_M < 1e-10
    (Eq. 41): 39 rounds; FP64 L1 <= 1e-12 against the oracle."""
    g = ci.chung_lu(10000, 100000, seed=0)
    rp, cx = g.numpy()
    G = pkg.Graph(g.row_ptr.cuda(), g.col_idx.cuda(), validate=True)
    p = torch.full((g.n,), 1.0 / g.n, dtype=torch.float64, device="cuda")
    M = next(m for m in range(1, 200) if O.err_bound(0.85, m) < 1e-10)
    pi, info = _solve(pkg, G, p, 0.85, 0.0, fixed_rounds=M)
    ref = O.cpaa(rp, cx, np.full(g.n, 1.0 / g.n), 0.85, M)
    assert M == 39 and info.rounds == 39
    assert _l1(pi, ref) <= 1e-12
    truth = O.power(rp, cx, np.full(g.n, 1.0 / g.n), 0.85, tol=1e-12)[0]
    assert _l1(pi, truth) <= 1e-10 * 10  # Eq. 41 is the paper's own (rough) bound
    G.close()


@pytest.fixture(scope="module")
def big_chung_lu(pkg):
    g = ci.chung_lu(1 << 24, 256_000_000, seed=0, device="cuda", distinct=True)
    G = pkg.Graph(g.row_ptr, g.col_idx, n=g.n, validate=True)
    rp, cx = g.numpy()
    del g
    torch.cuda.empty_cache()
    yield G, rp, cx
    G.close()


def test_config_16M_f64_and_f32(pkg, big_chung_lu):
    """16.7M-vertex Chung-Lu (256M distinct edges + ring), uniform p, c =
    0.85, tol 1e-6: FP64 within 1e-12 L1 and FP32 within 1e-6 relative L1 of
    the oracle run for the same M."""
    G, rp, cx = big_chung_lu
    n = len(rp) - 1
    p = torch.full((n,), 1.0 / n, dtype=torch.float64, device="cuda")
    pi64, i64 = _solve(pkg, G, p, 0.85, 1e-6, precision=pkg.CPAA_F64)
    pi32, i32 = _solve(pkg, G, p, 0.85, 1e-6, precision=pkg.CPAA_F32)
    pidf, idf = _solve(pkg, G, p, 0.85, 1e-6, precision=pkg.CPAA_DF64)
    assert i64.rounds == i32.rounds == idf.rounds
    hp = np.full(n, 1.0 / n)
    assert i64.rounds == O.rounds_needed(0.85, 1e-6, O.kappa(rp, hp))
    ref = O.cpaa(rp, cx, hp, 0.85, i64.rounds)
    e64 = _l1(pi64, ref)
    e32 = _l1(pi32, ref) / np.abs(ref).sum()
    edf = _l1(pidf, ref)
    print("16M: rounds %d, FP64 L1 %.3e, FP32 rel L1 %.3e, DF64 L1 %.3e" % (i64.rounds, e64, e32, edf))
    assert e64 <= 1e-12
    assert e32 <= 1e-6
    assert edf <= 1e-12


def test_config_16M_seeded_sample(pkg, big_chung_lu):
    """A 3-seed personalised vector on the same graph (high kappa)."""
    G, rp, cx = big_chung_lu
    n = len(rp) - 1
    hp = np.zeros(n)
    hp[[7, 123456, n - 5]] = 1.0 / 3
    p = torch.as_tensor(hp).cuda()
    pi64, i64 = _solve(pkg, G, p, 0.85, 1e-6, precision=pkg.CPAA_F64)
    pi32, i32 = _solve(pkg, G, p, 0.85, 1e-6, precision=pkg.CPAA_F32)
    pidf, idf = _solve(pkg, G, p, 0.85, 1e-6, precision=pkg.CPAA_DF64)
    ref = O.cpaa(rp, cx, hp, 0.85, i64.rounds)
    assert i64.rounds == O.rounds_needed(0.85, 1e-6, O.kappa(rp, hp))
    assert _l1(pi64, ref) <= 1e-12
    assert _l1(pi32, ref) / np.abs(ref).sum() <= 1e-6
    assert _l1(pidf, ref) <= 1e-12


def test_config_grid_precision_study(pkg):
    """4096 x 4096 lattice with 20% of edges deleted (spanning tree kept):
    FP64 / FP32 / BF16 against the oracle (BF16 is reported, loosely bounded)."""
    g = ci.grid_deleted(4096, 4096, 0.2, seed=0, device="cuda")
    assert g.nnz == 2 * (2 * 4096 * 4095 - round(0.2 * 2 * 4096 * 4095))
    G = pkg.Graph(g.row_ptr, g.col_idx, n=g.n, validate=True)
    rp, cx = g.numpy()
    n = g.n
    del g
    p = torch.full((n,), 1.0 / n, dtype=torch.float64, device="cuda")
    res = {}
    for name, prec in (("f64", pkg.CPAA_F64), ("f32", pkg.CPAA_F32), ("bf16", pkg.CPAA_BF16),
                       ("df64", pkg.CPAA_DF64)):
        res[name] = _solve(pkg, G, p, 0.85, 1e-6, precision=prec)
    M = res["f64"][1].rounds
    assert all(r[1].rounds == M for r in res.values())
    ref = O.cpaa(rp, cx, np.full(n, 1.0 / n), 0.85, M)
    errs = {k: _l1(v[0], ref) for k, v in res.items()}
    print("grid: rounds %d, L1 errors %s" % (M, errs))
    assert errs["f64"] <= 1e-12
    assert errs["df64"] <= 1e-12
    assert errs["f32"] <= 1e-6
    assert errs["bf16"] <= 5e-2
    G.close()


def test_config_batched_4M_sampled_columns(pkg):
    """4M-vertex Chung-Lu, 256 personalised vectors (1-16 uniform seeds), c =
    0.85, tol 1e-6, FP32 tiles: sampled columns against the oracle run for the
    same rounds, and every column normalised to 1."""
    g = ci.chung_lu(1 << 22, 64_000_000, seed=0, device="cuda", distinct=True)
    G = pkg.Graph(g.row_ptr, g.col_idx, n=g.n)
    rp, cx = g.numpy()
    n = g.n
    del g
    B = 256
    seeds = ci.seed_vectors(n, B, max_seeds=16, seed=0)
    P = torch.zeros((B, n), dtype=torch.float64, device="cuda")
    for b, (s, w) in enumerate(seeds):
        P[b, torch.as_tensor(s.astype(np.int64), device="cuda")] = torch.as_tensor(w, device="cuda")
    PI = torch.empty_like(P)
    infos = G.solve_batch(B, P, np.full(B, 0.85), 1e-6, PI, precision=pkg.CPAA_F32)
    torch.cuda.synchronize()
    sums = PI.sum(dim=1).cpu().numpy()
    assert np.abs(sums - 1.0).max() < 1e-9
    for b in (0, 131):
        p = P[b].cpu().numpy()
        ref = O.cpaa(rp, cx, p, 0.85, infos[b].rounds)
        rel = np.abs(PI[b].cpu().numpy() - ref).sum() / np.abs(ref).sum()
        print("batched column %d: rounds %d, rel L1 %.3e" % (b, infos[b].rounds, rel))
        assert rel <= 1e-6
    G.close()


def _with_hubs(n, edges, degrees, seed):
    """A Chung-Lu graph on n vertices plus one extra vertex per entry of
    `degrees`, joined to that many distinct vertices of the graph."""
    g = ci.chung_lu(n, edges, seed=seed)
    rp, cx = g.numpy()
    rows = np.repeat(np.arange(n), np.diff(rp))
    keep = rows < cx
    e = [np.stack([rows[keep], cx[keep]], 1)]
    rng = np.random.default_rng(seed)
    for i, d in enumerate(degrees):
        nb = rng.choice(n, size=d, replace=False)
        e.append(np.stack([np.full(d, n + i), nb], 1))
    return ci.from_edges(n + len(degrees), np.concatenate(e), name="chung_lu_with_hubs")


def test_large_graph_tile_boundaries(pkg):
    """A graph large enough for the 4096 hub threshold and 8192-entry hub
    tiles, with hub rows of exactly one tile, one tile plus one entry, and the
    threshold itself: FP64 against the oracle, FP32 and DF64 beside it, and a
    batch whose columns equal single solves."""
    degs = [4096, 4097, 8192, 8193, 16384]
    g = _with_hubs(1 << 20, 16_000_000, degs, seed=77)
    G = pkg.Graph(g.row_ptr.cuda(), g.col_idx.cuda(), n=g.n, validate=True)
    lay = G.layout()
    assert lay["hub_degree"] == 4096 and lay["hub_tile"] == 8192
    rp, cx = g.numpy()
    deg = np.diff(rp)
    hub = deg[deg > 4096]
    assert lay["hub_tiles"] == int(np.sum((hub + 8191) // 8192))
    n = g.n
    hp = np.zeros(n)
    hp[[n - 1, n - 3, 5, 77777]] = 0.25  # two of the added hubs among the seeds
    p = torch.as_tensor(hp).cuda()
    pi64, i64 = _solve(pkg, G, p, 0.85, 1e-9, precision=pkg.CPAA_F64)
    ref = O.cpaa(rp, cx, hp, 0.85, i64.rounds)
    assert _l1(pi64, ref) <= 1e-12
    pidf, idf = _solve(pkg, G, p, 0.85, 1e-9, precision=pkg.CPAA_DF64)
    assert _l1(pidf, ref) <= 1e-12
    pi32, _ = _solve(pkg, G, p, 0.85, 1e-9, precision=pkg.CPAA_F32, fixed_rounds=i64.rounds)
    assert _l1(pi32, ref) / np.abs(ref).sum() <= 1e-6
    P = torch.as_tensor(ci.seed_dense(n, ci.seed_vectors(n, 5, seed=3))).cuda()
    PI = torch.empty_like(P)
    infos = G.solve_batch(5, P, np.full(5, 0.85), 1e-7, PI, precision=pkg.CPAA_F32, batch_width=4)
    torch.cuda.synchronize()
    for b in (0, 4):
        single, info = _solve(pkg, G, P[b].contiguous(), 0.85, 1e-7, precision=pkg.CPAA_F32)
        assert infos[b].rounds == info.rounds
        assert torch.equal(PI[b], single)
    G.close()


def test_option_combinations(pkg):
    """Less common combinations: the (1 - c) scaling with DF64 and with the
    a-posteriori rule, per-round history under that rule, and every tile width
    in DF64."""
    g = ci.chung_lu(50000, 400000, seed=9)
    G = pkg.Graph(g.row_ptr.cuda(), g.col_idx.cuda(), n=g.n, validate=True)
    rp, cx = g.numpy()
    n = g.n
    hp = np.zeros(n)
    hp[[3, 40000]] = 0.5
    p = torch.as_tensor(hp).cuda()
    for prec, bound in ((pkg.CPAA_DF64, 1e-12), (pkg.CPAA_F64, 1e-12)):
        pi, info = _solve(pkg, G, p, 0.9, 1e-8, precision=prec, normalize=1,
                          stop_rule=pkg.CPAA_STOP_POSTERIORI)
        ref = O.cpaa(rp, cx, hp, 0.9, info.rounds, normalize=1)
        assert _l1(pi, ref) <= bound
    hist = np.zeros(2 * 200)
    pi, info = _solve(pkg, G, p, 0.85, 1e-8, stop_rule=pkg.CPAA_STOP_POSTERIORI, history=hist)
    _, mass, l1 = O.cpaa(rp, cx, hp, 0.85, info.rounds, history=True)
    M = info.rounds
    assert np.abs(hist[0:2 * (M + 1):2] - mass).max() < 1e-12
    assert np.abs(hist[1:2 * (M + 1):2] - l1).max() < 1e-10 * l1.max()
    P = torch.as_tensor(ci.seed_dense(n, ci.seed_vectors(n, 6, seed=4))).cuda()
    res = {}
    for W in (1, 2, 4, 8, 16):
        PI = torch.empty_like(P)
        infos = G.solve_batch(6, P, np.full(6, 0.85), 1e-8, PI, precision=pkg.CPAA_DF64, batch_width=W)
        torch.cuda.synchronize()
        res[W] = (PI.cpu().numpy(), [i.rounds for i in infos])
    for W in (2, 4, 8, 16):
        assert res[W][1] == res[1][1]
        assert np.array_equal(res[W][0], res[1][0])
    ref = O.cpaa(rp, cx, P[2].cpu().numpy(), 0.85, res[1][1][2])
    assert np.abs(res[1][0][2] - ref).sum() <= 1e-12
    G.close()
