"""Pins of the oracle's Chebyshev series on a narrower interval [lambda_lo, 1]
(Sec. 2.2's general-interval series; Sec. 6 names other approximations as
future work).

The series is pinned against things other than its own code: QUADPACK's
oscillatory quadrature of Sec. 2.2's coefficient integral on the interval,
the exact M-term truncation through eigh of S on graphs with a self-loop on
every vertex, LAPACK for the converged solution, explicit coefficient sums for
its error bound, and eigh again for the certified lower end of the spectrum
(-1 + 2/d_max when every vertex has a loop).  lambda_lo = -1 must give back
Algorithm 1 exactly."""
import math
import warnings

import numpy as np
import pytest
from scipy import integrate

import cpaa_inputs as ci
from oracle import oracle as O


def with_loops(g):
    """The same graph with a self-loop added on every vertex."""
    return ci.with_self_loops(g)


def looped_graphs():
    return [with_loops(ci.grid_deleted(6, 7, 0.2, seed=2)), with_loops(ci.random_small(40, 90, seed=4)),
            with_loops(ci.complete_bipartite(3, 5)), with_loops(ci.chung_lu(300, 1200, seed=5)),
            with_loops(ci.cycle(4)), with_loops(ci.star(9))]


def lam_min(g):
    rp, cx = g.numpy()
    _, A, d = O.dense_matrix_P(rp, cx)
    s = 1.0 / np.sqrt(d)
    return np.linalg.eigvalsh(s[:, None] * A * s[None, :]).min()


@pytest.mark.parametrize("c", [0.5, 0.85, 0.95])
@pytest.mark.parametrize("lo", [-1.0, -0.9, -0.6, -1.0 / 3.0, 0.0, 0.5])
def test_interval_coeffs_match_the_interval_integral(c, lo):
    """c_k = (2/pi) int_0^pi cos(k t) / (1 - c (mid + half cos t)) dt."""
    mid, half = 0.5 * (1 + lo), 0.5 * (1 - lo)
    ck = O.cheb_coeffs_interval(c, lo, 30)
    for k in range(0, 31, 3):
        with warnings.catch_warnings():
            warnings.simplefilter("ignore", integrate.IntegrationWarning)
            val, _ = integrate.quad(lambda t: 1.0 / (1.0 - c * (mid + half * math.cos(t))), 0.0, math.pi,
                                    weight="cos", wvar=k, limit=400, epsabs=1e-15, epsrel=1e-13)
        assert abs(ck[k] - 2.0 / math.pi * val) <= 1e-12 * max(1.0, ck[0]), (k, ck[k])
    # the full series at x = 1 (t = 1, every T_k(1) = 1) is f(1) = 1/(1 - c)
    long = O.cheb_coeffs_interval(c, lo, 3000)
    assert abs(long[0] / 2 + long[1:].sum() - 1.0 / (1.0 - c)) <= 1e-11 / (1 - c)


@pytest.mark.parametrize("c", [0.5, 0.85, 0.95])
def test_minus_one_is_algorithm_1(c):
    """lambda_lo = -1: the same coefficients, the same bound and the same
    iterates (mid = 0, half = 1 leave every operation unchanged)."""
    assert np.array_equal(O.cheb_coeffs_interval(c, -1.0, 40), O.cheb_coeffs(c, 40))
    for M in (1, 10, 40):
        assert abs(O.err_bound_interval(c, -1.0, M) - O.err_bound(c, M)) <= 1e-13 * O.err_bound(c, M)
    g = ci.chung_lu(500, 2500, seed=8)
    rp, cx = g.numpy()
    p = np.zeros(g.n)
    p[[3, 400]] = 0.5
    for M in (0, 1, 2, 9):
        for norm in (0, 1):
            assert np.array_equal(O.cpaa_interval(rp, cx, p, c, -1.0, M, norm), O.cpaa(rp, cx, p, c, M, norm))


@pytest.mark.parametrize("c", [0.5, 0.85, 0.95])
@pytest.mark.parametrize("lo", [-0.8, -0.5, 0.2])
def test_interval_err_bound_is_the_left_out_mass(c, lo):
    """ERR_M on the interval is (1-c) sum_{k>M} c_k, from explicit sums."""
    ck = O.cheb_coeffs_interval(c, lo, 4000)
    for M in (0, 1, 5, 20):
        tail = (1.0 - c) * ck[M + 1:].sum()
        assert abs(O.err_bound_interval(c, lo, M) - tail) <= 1e-12 * max(tail, 1e-300) + 1e-16


def test_certified_lower_end():
    """-1 + 2/d_max bounds the spectrum of S from below on every graph with a
    self-loop on every vertex, and is attained on the looped 4-cycle (d = 3,
    lambda_min = -1/3); with a vertex that has no loop the bound is the plain
    -1."""
    for g in looped_graphs():
        rp, cx = g.numpy()
        lo = O.lambda_lo_loops(rp, cx)
        assert lo == -1.0 + 2.0 / np.diff(rp).max()
        assert lam_min(g) >= lo - 1e-12, (g.name, lam_min(g), lo)
    c4 = with_loops(ci.cycle(4))
    rp, cx = c4.numpy()
    assert abs(lam_min(c4) - (-1.0 / 3.0)) <= 1e-12
    assert abs(O.lambda_lo_loops(rp, cx) - (-1.0 / 3.0)) <= 1e-15
    for g in (ci.cycle(4), ci.chung_lu(100, 300, seed=1)):
        rp, cx = g.numpy()
        assert O.lambda_lo_loops(rp, cx) == -1.0
    # one vertex without its loop: no bound beyond -1
    g = with_loops(ci.cycle(5))
    rp, cx = g.numpy()
    rows = np.repeat(np.arange(g.n), np.diff(rp))
    keep = ~((rows == 2) & (cx == 2))
    g2 = ci.from_edges(g.n, np.stack([rows[keep], cx[keep]], 1))
    rp2, cx2 = g2.numpy()
    assert O.lambda_lo_loops(rp2, cx2) == -1.0


@pytest.mark.parametrize("gi", range(6))
@pytest.mark.parametrize("norm", [0, 1])
def test_interval_truncation_matches_eigen_path(gi, norm):
    """After M rounds the interval recurrence equals the exact truncation of
    the interval series through eigh (pins the shift by mid, the scale by
    half, the coefficients and both normalisations), for the certified
    lambda_lo and for a looser one."""
    g = looped_graphs()[gi]
    rp, cx = g.numpy()
    n = g.n
    p = (np.arange(n) % 5 + 1.0)
    p /= p.sum()
    seed = np.zeros(n)
    seed[n // 3] = 1.0
    lo_cert = O.lambda_lo_loops(rp, cx)
    for lo in (lo_cert, 0.5 * (lo_cert - 1.0)):
        for c in (0.5, 0.9):
            for M in (0, 1, 2, 3, 6, 12):
                for q in (p, seed):
                    got = O.cpaa_interval(rp, cx, q, c, lo, M, norm)
                    want = O.eig_truncation_interval(rp, cx, q, c, lo, M, norm)
                    assert np.abs(got - want).sum() <= 1e-12, (g.name, lo, c, M)


@pytest.mark.parametrize("gi", range(6))
def test_interval_bound_holds_and_converges(gi):
    """The interval L1 bound holds after every M (exact error from LAPACK), and
    the rounds it asks for reach tol; the interval form needs no more rounds
    than Algorithm 1 on the same graph."""
    g = looped_graphs()[gi]
    rp, cx = g.numpy()
    n = g.n
    lo = O.lambda_lo_loops(rp, cx)
    for c in (0.5, 0.85, 0.95):
        for q in (np.full(n, 1.0 / n), np.eye(n)[n - 1]):
            truth = O.lapack_pagerank(rp, cx, q, c)
            k = O.kappa(rp, q)
            for norm in (0, 1):
                for M in (1, 3, 8, 15):
                    err = np.abs(O.cpaa_interval(rp, cx, q, c, lo, M, norm) - truth).sum()
                    assert err <= O.l1_bound_interval(c, lo, M, k, norm) * (1 + 1e-9) + 1e-14, (M, err)
                M = O.rounds_needed_interval(c, lo, 1e-10, k, norm)
                assert 1 <= M <= O.rounds_needed(c, 1e-10, k, norm)
                assert np.abs(O.cpaa_interval(rp, cx, q, c, lo, M, norm) - truth).sum() < 1e-10


def test_interval_saves_rounds_on_a_looped_lattice():
    """On a lattice with a loop on every vertex (d_max = 5, lambda_lo = -0.6)
    the series on [-0.6, 1] needs fewer rounds for the same bound."""
    g = with_loops(ci.grid_deleted(30, 30, 0.2, seed=1))
    rp, cx = g.numpy()
    lo = O.lambda_lo_loops(rp, cx)
    assert lo == -0.6
    p = np.full(g.n, 1.0 / g.n)
    k = O.kappa(rp, p)
    m_int = O.rounds_needed_interval(0.85, lo, 1e-6, k)
    m_std = O.rounds_needed(0.85, 1e-6, k)
    assert m_int < m_std
    truth = O.lapack_pagerank(rp, cx, p, 0.85)
    assert np.abs(O.cpaa_interval(rp, cx, p, 0.85, lo, m_int) - truth).sum() < 1e-6
