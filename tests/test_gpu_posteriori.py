"""GPU tests of the a-posteriori stopping rule and of the per-round sums.

The rule (cpaa_options.stop_rule = CPAA_STOP_POSTERIORI) replaces kappa in
the L1 bound by twice the running maximum of ||T_j p||_1, which the rounds
reduce on the device in a fixed order; a vector stops after the first round
whose estimate passes, or at the rigorous M.  The oracle applies the same rule
to its own FP64 history, and the exact solution checks that the result is
within tol."""
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


def _graphs():
    return [ci.chung_lu(3000, 20000, seed=11), ci.chung_lu(60000, 1500000, seed=12),
            ci.grid_deleted(40, 75, seed=3)]


GRAPHS = _graphs()


@pytest.fixture(scope="module")
def uploaded(pkg):
    return [upload(pkg, g) for g in GRAPHS]


def _vectors(n):
    uni = np.full(n, 1.0 / n)
    one = np.zeros(n); one[n - 3] = 1.0
    few = np.zeros(n); few[[1, n // 3, n - 11]] = 1.0 / 3
    return {"uniform": uni, "one_seed": one, "three_seeds": few}


def _oracle_rounds(rp, cx, p, c, tol, normalize=0):
    k = O.kappa(rp, p)
    M1 = O.rounds_needed(c, tol, k, normalize)
    _, _, l1 = O.cpaa(rp, cx, p, c, M1, normalize=normalize, history=True)
    M2 = O.rounds_posteriori(c, tol, l1, normalize)
    M = M1 if M2 is None else min(M1, M2)
    # how far the deciding bound is from tol (a near tie could fall either way
    # under a different rounding of the sums)
    ml = np.maximum.accumulate(l1)
    gap = abs(O.l1_bound(c, M, 2 * ml[M], normalize) / tol - 1.0)
    return M, M1, gap


@pytest.mark.parametrize("gi", range(len(GRAPHS)), ids=[g.name for g in GRAPHS])
@pytest.mark.parametrize("c", [0.5, 0.85, 0.95])
def test_posteriori_f64_matches_oracle_rule(pkg, uploaded, gi, c):
    g, G = GRAPHS[gi], uploaded[gi]
    rp, cx = g.numpy()
    for pname, p in _vectors(g.n).items():
        if g.n <= 2500:
            truth = O.lapack_pagerank(rp, cx, p, c)
        else:
            truth, _ = O.power(rp, cx, p, c, tol=1e-11)
        for tol in (1e-6, 1e-9):
            pi, info = solve(pkg, G, p, c, tol, stop_rule=pkg.CPAA_STOP_POSTERIORI)
            M, M1, gap = _oracle_rounds(rp, cx, p, c, tol)
            if gap > 1e-9:
                assert info.rounds == M, (pname, tol, info.rounds, M)
            assert info.rounds <= M1
            ref = O.cpaa(rp, cx, p, c, info.rounds)
            assert np.abs(pi - ref).sum() <= 1e-12, (pname, tol)
            assert np.abs(pi - truth).sum() <= tol, (pname, tol)
            assert info.bound < tol


def test_posteriori_shortens_few_seed_solves(pkg, uploaded):
    """On the larger graph a single seed has kappa far above ||T_j p||_1, so the
    estimate stops well before the rigorous M."""
    g, G = GRAPHS[1], uploaded[1]
    p = _vectors(g.n)["one_seed"]
    _, r1 = solve(pkg, G, p, 0.85, 1e-6, precision=pkg.CPAA_F32)
    _, r2 = solve(pkg, G, p, 0.85, 1e-6, precision=pkg.CPAA_F32, stop_rule=pkg.CPAA_STOP_POSTERIORI)
    assert r2.rounds < r1.rounds


@pytest.mark.parametrize("gi", range(len(GRAPHS)), ids=[g.name for g in GRAPHS])
def test_posteriori_f32_matches_oracle(pkg, uploaded, gi):
    g, G = GRAPHS[gi], uploaded[gi]
    rp, cx = g.numpy()
    for pname, p in _vectors(g.n).items():
        pi, info = solve(pkg, G, p, 0.85, 1e-6, precision=pkg.CPAA_F32,
                         stop_rule=pkg.CPAA_STOP_POSTERIORI)
        M, M1, gap = _oracle_rounds(rp, cx, p, 0.85, 1e-6)
        if gap > 1e-4:  # FP32 sums: a looser tie margin
            assert info.rounds == M, (pname, info.rounds, M)
        ref = O.cpaa(rp, cx, p, 0.85, info.rounds)
        assert np.abs(pi - ref).sum() / np.abs(ref).sum() <= 1e-6, pname


@pytest.mark.parametrize("prec", ["F64", "F32", "DF64"])
def test_posteriori_batch_columns_equal_single(pkg, uploaded, prec):
    g, G = GRAPHS[1], uploaded[1]
    P = ci.seed_dense(g.n, ci.seed_vectors(g.n, 6, seed=21))
    cs = np.array([0.5, 0.85, 0.95, 0.85, 0.7, 0.95])
    pr = getattr(pkg, "CPAA_" + prec)
    Pd = torch.as_tensor(P).cuda()
    PI = torch.empty_like(Pd)
    infos = G.solve_batch(6, Pd, cs, 1e-7, PI, precision=pr, stop_rule=pkg.CPAA_STOP_POSTERIORI)
    torch.cuda.synchronize()
    for b in range(6):
        single, info = solve(pkg, G, P[b], cs[b], 1e-7, precision=pr, stop_rule=pkg.CPAA_STOP_POSTERIORI)
        assert infos[b].rounds == info.rounds
        assert infos[b].bound == info.bound
        assert np.array_equal(PI[b].cpu().numpy(), single)


def test_round_sums_are_deterministic(pkg, uploaded):
    """The per-round sums are added in a fixed order: a repeated solve and a
    batch column report the same bits as a single solve."""
    g, G = GRAPHS[1], uploaded[1]
    P = ci.seed_dense(g.n, ci.seed_vectors(g.n, 4, seed=5))
    for pr in (pkg.CPAA_F64, pkg.CPAA_F32):
        Pd = torch.as_tensor(P).cuda()
        PI = torch.empty_like(Pd)
        infos = G.solve_batch(4, Pd, np.full(4, 0.85), 1e-6, PI, precision=pr, batch_width=4)
        torch.cuda.synchronize()
        for b in range(4):
            _, i1 = solve(pkg, G, P[b], 0.85, 1e-6, precision=pr)
            _, i2 = solve(pkg, G, P[b], 0.85, 1e-6, precision=pr)
            assert (i1.mass, i1.l1) == (i2.mass, i2.l1)
            assert (infos[b].mass, infos[b].l1) == (i1.mass, i1.l1)


def test_stop_rule_invalid(pkg, uploaded):
    g, G = GRAPHS[0], uploaded[0]
    p = np.full(g.n, 1.0 / g.n)
    with pytest.raises(pkg.CpaaError, match="stop_rule"):
        solve(pkg, G, p, 0.85, 1e-6, stop_rule=7)
    pd = torch.as_tensor(p).cuda()
    out = torch.empty_like(pd)
    with pytest.raises(pkg.CpaaError, match="power method"):
        G.power_solve(pd, 0.85, 1e-6, out, stop_rule=pkg.CPAA_STOP_POSTERIORI)
    with pytest.raises(pkg.CpaaError, match="power method"):
        G.power_solve(pd, 0.85, 1e-6, out, precision=pkg.CPAA_BF16)
    with pytest.raises(pkg.CpaaError, match="precision"):
        pkg.Server(1 << 30, precision=7)
