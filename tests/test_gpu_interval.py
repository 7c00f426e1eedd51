"""The Chebyshev series on a narrower interval [lambda_lo, 1] on the GPU
(CPAA_INTERVAL / CPAA_CERTIFY_INTERVAL; Sec. 2.2's general-interval series).

On graphs with a self-loop on every vertex the library certifies
lambda_lo = -1 + 2/d_max by itself; the rounds must be the oracle's for that
interval, the result the oracle's interval truncation within the FP64 / FP32
bounds, and fewer rounds than the plain series must reach the same bound."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import cpaa_inputs as ci
from oracle import oracle as O
from tests.gpu_util import solve, upload
from tests.test_oracle_interval_pins import with_loops

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2112_01743_gb300 as pkg
    return pkg


@pytest.fixture(scope="module")
def looped(pkg):
    gl = {"lattice": with_loops(ci.grid_deleted(300, 310, 0.2, seed=6)),
          "chung_lu": with_loops(ci.chung_lu(60000, 700000, seed=17)),
          "bipartite": with_loops(ci.complete_bipartite(40, 70))}
    up = {k: upload(pkg, g) for k, g in gl.items()}
    yield gl, up
    for G in up.values():
        G.close()


@pytest.mark.parametrize("name", ["lattice", "chung_lu", "bipartite"])
@pytest.mark.parametrize("prec,bound,rel", [("F64", 1e-12, False), ("DF64", 1e-12, False), ("F32", 1e-6, True)])
def test_certified_interval_against_oracle(pkg, looped, name, prec, bound, rel):
    gl, up = looped
    g, G = gl[name], up[name]
    rp, cx = g.numpy()
    lo = O.lambda_lo_loops(rp, cx)
    assert lo > -1.0 and G.spectrum_bound() == lo
    P = getattr(pkg, "CPAA_" + prec)
    for seeds in ([0], [g.n // 2, 7], list(range(g.n))):
        p = np.zeros(g.n)
        p[seeds] = 1.0 / len(seeds)
        for norm in (0, 1):
            pi, info = solve(pkg, G, p, 0.85, 1e-8, precision=P, normalize=norm, certify_interval=True)
            assert info.lambda_lo == lo
            k = O.kappa(rp, p)
            assert info.rounds == O.rounds_needed_interval(0.85, lo, 1e-8, k, norm)
            assert info.rounds <= O.rounds_needed(0.85, 1e-8, k, norm)
            ref = O.cpaa_interval(rp, cx, p, 0.85, lo, info.rounds, norm)
            err = np.abs(pi - ref).sum() / (np.abs(ref).sum() if rel else 1.0)
            assert err <= bound, (name, seeds[:2], norm, err)


def test_interval_rounds_saved_and_exact_solution(pkg, looped):
    """On the looped lattice (d_max = 5: lambda_lo = -0.6) the interval series
    reaches the same L1 bound in fewer rounds, and both are within tol of the
    exact solution."""
    gl, up = looped
    g, G = gl["lattice"], up["lattice"]
    rp, cx = g.numpy()
    p = np.full(g.n, 1.0 / g.n)
    a, ia = solve(pkg, G, p, 0.85, 1e-9)
    b, ib = solve(pkg, G, p, 0.85, 1e-9, certify_interval=True)
    assert ib.lambda_lo == -0.6 and ia.lambda_lo == -1.0
    assert ib.rounds < ia.rounds
    truth, _ = O.power(rp, cx, p, 0.85, tol=1e-13)
    assert np.abs(a - truth).sum() < 1e-9 and np.abs(b - truth).sum() < 1e-9
    print("looped lattice: %d rounds on [-1, 1], %d on [-0.6, 1]" % (ia.rounds, ib.rounds))


def test_caller_interval_and_minus_one(pkg, looped):
    """A caller-certified looser lambda_lo works; CPAA_INTERVAL with -1 is the
    plain series bit for bit; without loops the graph certifies nothing."""
    gl, up = looped
    g, G = gl["chung_lu"], up["chung_lu"]
    rp, cx = g.numpy()
    p = np.zeros(g.n)
    p[[5, 50000]] = 0.5
    pi, info = solve(pkg, G, p, 0.9, 1e-9, lambda_lo=-0.95)
    assert info.lambda_lo == -0.95
    ref = O.cpaa_interval(rp, cx, p, 0.9, -0.95, info.rounds)
    assert np.abs(pi - ref).sum() <= 1e-12
    a, ia = solve(pkg, G, p, 0.9, 1e-9)
    b, ib = solve(pkg, G, p, 0.9, 1e-9, lambda_lo=-1.0)
    assert ia.rounds == ib.rounds and np.array_equal(a, b)
    plain = upload(pkg, ci.chung_lu(3000, 20000, seed=2))
    assert plain.spectrum_bound() == -1.0
    q = np.full(plain.n, 1.0 / plain.n)
    a, ia = solve(pkg, plain, q, 0.85, 1e-8)
    b, ib = solve(pkg, plain, q, 0.85, 1e-8, certify_interval=True)
    assert ib.lambda_lo == -1.0 and np.array_equal(a, b)
    with pytest.raises(pkg.CpaaError) as e:
        solve(pkg, plain, q, 0.85, 1e-8, lambda_lo=1.0)
    assert e.value.status == pkg.CPAA_EINVAL
    plain.close()


def test_interval_batch_and_frontier(pkg, looped):
    """Batch columns equal single solves on the interval series, and the
    sparse frontier gives the same bits on it."""
    gl, up = looped
    for name in ("lattice", "chung_lu"):
        g, G = gl[name], up[name]
        seeds = ci.seed_vectors(g.n, 5, max_seeds=4, seed=9)
        P = ci.seed_dense(g.n, seeds)
        Pd = torch.as_tensor(P).cuda()
        for prec in (pkg.CPAA_F64, pkg.CPAA_F32, pkg.CPAA_DF64, pkg.CPAA_BF16):
            PI = torch.empty_like(Pd)
            infos = G.solve_batch(5, Pd, np.array([0.5, 0.85, 0.95, 0.85, 0.7]), 1e-7, PI, precision=prec,
                                  batch_width=4, certify_interval=True)
            torch.cuda.synchronize()
            for b, cb in ((0, 0.5), (2, 0.95), (4, 0.7)):
                single, info = solve(pkg, G, P[b], cb, 1e-7, precision=prec, certify_interval=True)
                assert infos[b].rounds == info.rounds and infos[b].lambda_lo == info.lambda_lo
                assert np.array_equal(PI[b].cpu().numpy(), single), (name, prec, b)
                fr, finfo = solve(pkg, G, P[b], cb, 1e-7, precision=prec, certify_interval=True, frontier=True)
                assert finfo.rounds == info.rounds and np.array_equal(fr, single)
