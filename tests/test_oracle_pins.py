"""Pins for the FP64 oracle: each test checks the oracle against something
other than itself -- numbers the paper prints, the defining integral of the
coefficients evaluated by quadrature, LAPACK, an eigen-decomposition, closed
forms derived by hand, invariants, and brute force on tiny graphs."""
import json
import math
import os
import warnings

import numpy as np
import pytest
from scipy import integrate

import cpaa_inputs as ci
from oracle import oracle as O

with open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")) as _f:
    GOLD = json.load(_f)
CS = [0.5, 0.85, 0.95]


# -- coefficients (Sec. 2.2, Proposition 1) -----------------------------------

@pytest.mark.parametrize("c", [0.1, 0.5, 0.85, 0.95, 0.99])
def test_coeffs_match_defining_integral(c):
    """c_k = (2/pi) int_0^pi cos(kt)/(1 - c cos t) dt, by adaptive quadrature."""
    ck = O.cheb_coeffs(c, 40)
    for k in range(0, 41, 3):
        # the oscillatory rule (weight cos(k t)) keeps its accuracy at large k,
        # where c_k is a tiny remainder of cancelling lobes; QUADPACK then
        # reports that no relative tolerance is reachable, while the assertion
        # below bounds the difference absolutely
        with warnings.catch_warnings():
            warnings.simplefilter("ignore", integrate.IntegrationWarning)
            val, err = integrate.quad(lambda t: 1.0 / (1.0 - c * math.cos(t)), 0.0, math.pi,
                                      weight="cos", wvar=k, limit=400, epsabs=1e-15, epsrel=1e-13)
        ref = 2.0 / math.pi * val
        assert abs(ck[k] - ref) <= 1e-12 * max(1.0, abs(ck[0])), (k, ck[k], ref)


@pytest.mark.parametrize("c", [0.1, 0.5, 0.85, 0.95, 0.99])
def test_coeffs_match_printed_closed_forms(c):
    """The proof of Proposition 1 (Sec. 4.2.1) prints c_0, c_1 and c_2 in closed
    form, and sigma_k as a ratio of two expressions in c; the oracle's first
    coefficients must equal the printed ones and its beta the printed sigma."""
    r = math.sqrt(1.0 - c * c)
    printed = [2.0 / r, 2.0 / c * (1.0 - r) / r, 2.0 / (c * c) * (2.0 * (1.0 - r) - c * c) / r]
    ck = O.cheb_coeffs(c, 2)
    for k in range(3):
        assert abs(ck[k] - printed[k]) <= 1e-13 * printed[0], (k, ck[k], printed[k])
    sigma = (c * c - (2.0 - c) * (1.0 - r)) / (c * c - c * (1.0 - r))
    assert abs(O.beta(c) - sigma) <= 1e-12 * sigma


@pytest.mark.parametrize("c", CS)
def test_coeff_three_term_relation(c):
    """c_{k-1} + c_{k+1} = (2/c) c_k (proof of Proposition 1)."""
    ck = O.cheb_coeffs(c, 60)
    for k in range(1, 60):
        assert abs(ck[k - 1] + ck[k + 1] - 2.0 / c * ck[k]) <= 1e-14 * ck[k - 1]


@pytest.mark.parametrize("c", CS)
def test_coeff_series_sums_to_f_at_one(c):
    """c_0/2 + sum_k c_k T_k(1) = f(1) = 1/(1-c): T_k(1) = 1 (Sec. 2.2)."""
    ck = O.cheb_coeffs(c, 2000)
    assert abs(ck[0] / 2 + ck[1:].sum() - 1.0 / (1.0 - c)) < 1e-11 / (1.0 - c)


def test_sigma_c_printed_value():
    """sigma_c = 0.5567 at c = 0.85 (printed after Proposition 1); sigma_k =
    (S - S_k)/(S - S_{k-1}) from explicit coefficient sums."""
    g = GOLD["sigma_c_at_0.85"]
    ck = O.cheb_coeffs(0.85, 3000)
    S = ck[0] / 2 + ck[1:].sum()
    for k in (1, 5, 20):
        Sk = ck[0] / 2 + ck[1:k + 1].sum()
        Skm1 = ck[0] / 2 + ck[1:k].sum()
        sig = (S - Sk) / (S - Skm1)
        assert round(sig, g["digits"]) == g["value"]
    assert round(O.beta(0.85), 4) == g["value"]


@pytest.mark.parametrize("c", CS)
def test_err_bound_matches_explicit_sums(c):
    """Eq. 41 against 1 - S_M/S summed from the coefficient table."""
    ck = O.cheb_coeffs(c, 3000)
    S = 1.0 / (1.0 - c)  # f(1)
    for M in (0, 1, 5, 12, 30):
        SM = ck[0] / 2 + ck[1:M + 1].sum()
        assert abs(O.err_bound(c, M) - (1.0 - SM / S)) < 1e-13


def test_err_bound_paper_claims():
    """ERR_M < 1e-4 within 20 rounds at c=0.85 (after Eq. 41) and 12 rounds reach
    1e-3 (Table 3's CPAA column), while 11 do not."""
    g = GOLD["err_M_below_1e-4_within_rounds"]
    assert O.err_bound(g["c"], g["rounds"]) < 1e-4
    r = GOLD["rounds_to_err_1e-3_cpaa"]["rounds"]
    assert O.err_bound(0.85, r) < 1e-3 <= O.err_bound(0.85, r - 1)


# -- the method against independent solvers ------------------------------------

def _graphs():
    return [ci.star(7), ci.cycle(9), ci.path(6), ci.complete(6), ci.complete_bipartite(3, 5),
            ci.random_small(40, 90, seed=1), ci.random_small(120, 500, seed=2),
            ci.chung_lu(300, 2000, seed=3)]


@pytest.mark.parametrize("gi", range(8))
@pytest.mark.parametrize("c", CS)
def test_converged_cpaa_equals_dense_solve(gi, c):
    """CPAA run to a 1e-14 L1 bound equals (1-c)(I - cP)^-1 p (Sec. 2.1, Eq. 31)
    solved by LAPACK, for uniform and single-seed p."""
    g = _graphs()[gi]
    rp, cx = g.numpy()
    n = g.n
    for p in (np.full(n, 1.0 / n), np.eye(n)[n // 3]):
        ref = O.lapack_pagerank(rp, cx, p, c)
        for norm in (0, 1):
            pi, M = O.solve(rp, cx, p, c, 1e-13, normalize=norm)
            assert np.abs(pi - ref).sum() < 1e-12, (g.name, c, norm, M)


@pytest.mark.parametrize("gi", range(8))
def test_c_dense_solver_matches_lapack(gi):
    g = _graphs()[gi]
    rp, cx = g.numpy()
    p = np.linspace(1.0, 2.0, g.n)
    p /= p.sum()
    assert np.abs(O.dense_pagerank(rp, cx, p, 0.85) - O.lapack_pagerank(rp, cx, p, 0.85)).sum() < 1e-13


def barbell(k):
    """Two k-cliques joined by one edge: a slowly mixing graph."""
    edges = [(i, j) for i in range(k) for j in range(i + 1, k)]
    edges += [(k + i, k + j) for i in range(k) for j in range(i + 1, k)]
    return ci.from_edges(2 * k, edges + [(k - 1, k)], name="barbell%d" % k)


def power_stop_failures():
    """The power method's stop test (c/(1-c)) ||x_{t+1} - x_t||_1 < tol bounds
    the distance to pi* (cP shrinks L1 distances by c).  On a barbell graph
    with one seed that bound is nearly attained (the error reaches 0.94 tol),
    so the returned x must be within tol of the exact solution; returns the
    failing (c, tol) cases."""
    bad = []
    g = barbell(20)
    rp, cx = g.numpy()
    p = np.zeros(g.n); p[0] = 1.0
    for c in (0.85, 0.95):
        ref = O.lapack_pagerank(rp, cx, p, c)
        for tol in (1e-3, 1e-5, 1e-7, 1e-9):
            x, _ = O.power(rp, cx, p, c, tol=tol)
            if not np.abs(x - ref).sum() <= tol:
                bad.append((c, tol))
    return bad


def test_power_method_ground_truth_rounds():
    """Sec. 5.1 takes 210 power-method rounds at c = 0.85 as the ground truth
    (0.85^210 is about 1.5e-15): after that many rounds the oracle's power
    method agrees with LAPACK to rounding, also on the slowly mixing barbell."""
    g0 = GOLD["ground_truth_power_rounds"]["value"]
    for g in (barbell(20), ci.chung_lu(300, 2000, seed=3)):
        rp, cx = g.numpy()
        p = np.zeros(g.n); p[0] = 1.0
        x, _ = O.power(rp, cx, p, 0.85, rounds=g0)
        assert np.abs(x - O.lapack_pagerank(rp, cx, p, 0.85)).sum() < 1e-13, g.name
    assert 0.85 ** g0 < 2e-15


def test_power_method_stop_rule_against_exact_error():
    assert power_stop_failures() == []


@pytest.mark.parametrize("gi", range(8))
def test_power_method_matches_lapack(gi):
    g = _graphs()[gi]
    rp, cx = g.numpy()
    p = np.full(g.n, 1.0 / g.n)
    # 1e-13: on some graphs the L1 change between rounds stalls near 2e-15
    # (rounding), which puts a 1e-14 bound out of reach.
    x, it = O.power(rp, cx, p, 0.85, tol=1e-13)
    assert np.abs(x - O.lapack_pagerank(rp, cx, p, 0.85)).sum() < 1e-13


@pytest.mark.parametrize("gi", range(8))
@pytest.mark.parametrize("M", [0, 1, 2, 3, 7, 15])
def test_truncation_matches_eigen_path(gi, M):
    """The recurrence after M rounds equals (1-c)[c_0/2 p + sum c_k T_k(P) p] with
    T_k(lambda) = cos(k arccos lambda) applied to S = D^-1/2 A D^-1/2's spectrum
    and coefficients from quadrature (pins the recurrence, the rotation, the
    coefficient indexing and both normalisations independently)."""
    g = _graphs()[gi]
    rp, cx = g.numpy()
    n = g.n
    p = (np.arange(n) % 5 + 1.0)
    p /= p.sum()
    for norm in (0, 1):
        a = O.cpaa(rp, cx, p, 0.85, M, normalize=norm)
        b = O.eig_truncation(rp, cx, p, 0.85, M, normalize=norm)
        assert np.abs(a - b).sum() < 1e-12, (g.name, M, norm)


def negative_entry_truncation_failures():
    """For c > 0.943 (beta^2 > 1/2) the degree-2 truncation's constant term
    c_0/2 - c_2 is negative, so on K_50 with one seed (every neighbour of the
    seed has degree 49) pibar_2 has a negative entry at the seed.  The
    recurrence must still equal the eigen path there, in both normalisations
    (Algorithm 1's last line divides by the signed sum)."""
    bad = []
    g = ci.complete(50)
    rp, cx = g.numpy()
    p = np.zeros(50); p[0] = 1.0
    if not O.cpaa(rp, cx, p, 0.95, 2, normalize=1).min() < -1e-4:
        bad.append("no_negative_entry")
    for norm in (0, 1):
        if np.abs(O.cpaa(rp, cx, p, 0.95, 2, normalize=norm)
                  - O.eig_truncation(rp, cx, p, 0.95, 2, normalize=norm)).sum() > 1e-13:
            bad.append("norm%d" % norm)
    return bad


def test_truncation_with_a_negative_entry():
    assert negative_entry_truncation_failures() == []


@pytest.mark.parametrize("c", CS)
def test_truncated_sum_is_one_minus_err(c):
    """With (1-c) scaling the M-term result sums to exactly 1 - ERR_M (mass view of
    Sec. 4.1: e^T T_k(P) p = e^T p, and Eq. 41)."""
    g = ci.chung_lu(500, 4000, seed=5)
    rp, cx = g.numpy()
    p = np.full(g.n, 1.0 / g.n)
    for M in (1, 4, 10, 25):
        pi = O.cpaa(rp, cx, p, c, M, normalize=1)
        assert abs(pi.sum() - (1.0 - O.err_bound(c, M))) < 1e-13


def test_mass_invariant_every_round():
    """sum_u T_k[u] stays e^T p for every k (Sec. 4.1)."""
    g = ci.chung_lu(2000, 15000, seed=4)
    rp, cx = g.numpy()
    p = np.zeros(g.n)
    p[[3, 700, 1999]] = [0.5, 0.25, 0.25]
    _, mass, l1 = O.cpaa(rp, cx, p, 0.85, 40, history=True)
    assert np.all(np.abs(mass - 1.0) < 1e-12)
    assert np.all(l1 <= O.kappa(rp, p) * (1 + 1e-12))


@pytest.mark.parametrize("c", CS)
def test_l1_bound_holds(c):
    """The rigorous stopping bound really bounds the L1 error."""
    g = ci.chung_lu(800, 6000, seed=6)
    rp, cx = g.numpy()
    n = g.n
    ref_u = O.lapack_pagerank(rp, cx, np.full(n, 1.0 / n), c)
    e = np.zeros(n); e[n - 1] = 1.0
    ref_e = O.lapack_pagerank(rp, cx, e, c)
    for p, ref in ((np.full(n, 1.0 / n), ref_u), (e, ref_e)):
        k = O.kappa(rp, p)
        for M in (2, 5, 10, 20):
            for norm in (0, 1):
                err = np.abs(O.cpaa(rp, cx, p, c, M, normalize=norm) - ref).sum()
                assert err <= O.l1_bound(c, M, k, norm) * (1 + 1e-9) + 1e-15


def stopping_rule_truth_failures(c):
    """Pins of the rigorous stopping rule against the exact solution (LAPACK),
    sharper than soundness; returns the names of the checks that fail.

    - On a regular graph with uniform p every T_k p is p and kappa = 1, so the
      (1-c)-scaled truncation misses exactly the coefficient mass ERR_M: its L1
      error equals the normalize=1 bound ERR_M kappa (Eq. 41).
    - There, rounds_needed's M is the first whose measured error is below tol.
    - Dividing by the sum (Algorithm 1's last line) can cost more than
      ERR_M kappa: on K_5 with one seed, c = 0.05, M = 1 the error is 1.27 x
      ERR_M kappa, so the normalisation term of the normalize=0 bound is needed
      and must cover it."""
    bad = []
    g = ci.circulant(30, [1, 4, 7])
    rp, cx = g.numpy()
    n = g.n
    p = np.full(n, 1.0 / n)
    ref = O.lapack_pagerank(rp, cx, p, c)
    k = O.kappa(rp, p)
    if abs(k - 1.0) > 1e-14:
        bad.append("kappa_regular")
    err = {M: np.abs(O.cpaa(rp, cx, p, c, M, normalize=1) - ref).sum() for M in range(1, 80)}
    for M in (1, 2, 5, 13):
        if abs(err[M] - O.l1_bound(c, M, k, 1)) > 1e-9 * err[M] + 1e-14:
            bad.append("tight_M%d" % M)
    for tol in (1e-2, 1e-4, 1e-7):
        M = O.rounds_needed(c, tol, k, 1)
        if not (1 <= M < 80 and err[M] < tol and (M == 1 or err[M - 1] >= tol)):
            bad.append("minimal_%g" % tol)
    g5 = ci.complete(5)
    rp5, cx5 = g5.numpy()
    e = np.zeros(5); e[0] = 1.0
    k5 = O.kappa(rp5, e)
    err0 = np.abs(O.cpaa(rp5, cx5, e, 0.05, 1, normalize=0) - O.lapack_pagerank(rp5, cx5, e, 0.05)).sum()
    if not err0 > 1.2 * O.err_bound(0.05, 1) * k5:
        bad.append("norm_case")
    if not err0 <= O.l1_bound(0.05, 1, k5, 0):
        bad.append("norm_term")
    return bad


@pytest.mark.parametrize("c", CS)
def test_stopping_rule_against_exact_error(c):
    assert stopping_rule_truth_failures(c) == []


@pytest.mark.parametrize("c", CS)
def test_posteriori_rule_against_exact_solution(c):
    """The a-posteriori rule (kappa replaced by twice the running max of
    ||T_j p||_1) is an estimate: pin its M against the exact solution from
    LAPACK on uniform, single-seed and few-seed vectors, and check that it
    never asks for more rounds than the rigorous rule when 2 max ||T_j p|| <=
    kappa (so it can only shorten such solves)."""
    margins = []
    for gseed, (n, m) in enumerate(((600, 4000), (1500, 9000))):
        g = ci.chung_lu(n, m, seed=40 + gseed)
        rp, cx = g.numpy()
        ps = [np.full(n, 1.0 / n)]
        for s0 in ((n - 1,), (n // 2,), (3, 100, n - 7)):
            e = np.zeros(n); e[list(s0)] = 1.0 / len(s0)
            ps.append(e)
        for p in ps:
            ref = O.lapack_pagerank(rp, cx, p, c)
            k = O.kappa(rp, p)
            for tol in (1e-4, 1e-6, 1e-9):
                for norm in (0, 1):
                    M1 = O.rounds_needed(c, tol, k, norm)
                    _, _, l1 = O.cpaa(rp, cx, p, c, M1, normalize=norm, history=True)
                    M2 = O.rounds_posteriori(c, tol, l1, norm)
                    if 2 * l1.max() <= k:
                        assert M2 is not None and M2 <= M1
                    M = M1 if M2 is None else min(M1, M2)
                    err = np.abs(O.cpaa(rp, cx, p, c, M, normalize=norm) - ref).sum()
                    assert err <= tol, (n, tol, norm, M, err)
                    margins.append(err / tol)
    assert max(margins) < 1.0


def posteriori_hand_failures(rule):
    """Hand cases of the a-posteriori rule (kappa replaced by twice the running
    max of ||T_j p||_1 over j = 0..M); returns the names of the cases that
    ``rule`` (same signature as ``oracle.rounds_posteriori``) gets wrong."""
    c, tol = 0.85, 1e-6
    bad = []
    hist = np.ones(200)
    # all terms 1: the estimate is 2, so M is the first with l1_bound(c, M, 2) < tol
    want = next(M for M in range(1, 200) if O.l1_bound(c, M, 2.0) < tol)
    if rule(c, tol, hist) != want:
        bad.append("flat")
    # a larger term at round want - 1 keeps the estimate up from there on
    hist2 = hist.copy(); hist2[want - 1] = 50.0
    if not rule(c, tol, hist2) > want:
        bad.append("earlier_peak")
    # a larger term at round want itself counts in round want's test
    hist3 = hist.copy(); hist3[want] = 50.0
    if not rule(c, tol, hist3) > want:
        bad.append("peak_at_M")
    # ||T_0 p||_1 = ||p||_1 counts too (j = 0 is in the max)
    hist4 = hist.copy(); hist4[0] = 10.0
    if rule(c, tol, hist4) != next(M for M in range(1, 200) if O.l1_bound(c, M, 20.0) < tol):
        bad.append("T0")
    # no M within a history too short to pass
    if rule(c, tol, hist[:want]) is not None:
        bad.append("short")
    return bad


def test_posteriori_rule_hand_case():
    assert posteriori_hand_failures(O.rounds_posteriori) == []


# -- closed forms ------------------------------------------------------------------

@pytest.mark.parametrize("L", [1, 2, 5, 50])
@pytest.mark.parametrize("c", CS)
def test_star_closed_form(L, c):
    """K_{1,L}, uniform p: pi_centre = (1+cL)/(n(1+c)), pi_leaf = (L+c)/(nL(1+c))
    (solved by hand from (I - cP) pi = (1-c) p, Sec. 2.1).  Bipartite, so P has
    the eigenvalue -1 and T_k(-1) = (-1)^k is exercised."""
    g = ci.star(L)
    rp, cx = g.numpy()
    n = L + 1
    pi, _ = O.solve(rp, cx, np.full(n, 1.0 / n), c, 1e-14)
    assert abs(pi[0] - (1 + c * L) / (n * (1 + c))) < 1e-14
    assert np.all(np.abs(pi[1:] - (L + c) / (n * L * (1 + c))) < 1e-14)


@pytest.mark.parametrize("a,b", [(2, 3), (4, 4), (1, 9), (6, 2)])
def test_complete_bipartite_closed_form(a, b):
    """K_{a,b}, uniform p: pi_X = (a + cb)/(a n (1+c)), pi_Y = (b + ca)/(b n (1+c))."""
    c = 0.85
    g = ci.complete_bipartite(a, b)
    rp, cx = g.numpy()
    n = a + b
    pi, _ = O.solve(rp, cx, np.full(n, 1.0 / n), c, 1e-14)
    assert np.all(np.abs(pi[:a] - (a + c * b) / (a * n * (1 + c))) < 1e-14)
    assert np.all(np.abs(pi[a:] - (b + c * a) / (b * n * (1 + c))) < 1e-14)


@pytest.mark.parametrize("g", [ci.cycle(10), ci.complete(7), ci.circulant(30, [1, 4, 7])],
                         ids=lambda g: g.name)
def test_regular_graph_uniform_at_every_round(g):
    """On a regular graph P e = e, so T_k(P) e = e and the normalised result is
    uniform after any number of rounds."""
    rp, cx = g.numpy()
    p = np.full(g.n, 1.0 / g.n)
    for M in (0, 1, 2, 9):
        assert np.all(np.abs(O.cpaa(rp, cx, p, 0.85, M) - 1.0 / g.n) < 1e-15)


def test_personalized_reversibility_and_linearity():
    """(I - cP)^-1 = D (D - cA)^-1 with D - cA symmetric (Lemma 2's B), so
    pi_s(t)/d_t = pi_t(s)/d_s; and by linearity the mean of the single-seed
    results is the uniform result."""
    g = ci.random_small(60, 150, seed=9)
    rp, cx = g.numpy()
    n = g.n
    d = np.diff(rp).astype(float)
    cols = [O.solve(rp, cx, np.eye(n)[s], 0.85, 1e-14)[0] for s in range(n)]
    Pi = np.stack(cols, axis=1)  # Pi[t, s] = pi_s(t)
    lhs = Pi / d[:, None]
    assert np.abs(lhs - lhs.T).max() < 1e-14
    uni, _ = O.solve(rp, cx, np.full(n, 1.0 / n), 0.85, 1e-14)
    assert np.abs(Pi.mean(axis=1) - uni).sum() < 1e-13


@pytest.mark.parametrize("n", [2, 3, 4, 5])
def test_brute_force_all_tiny_graphs(n):
    """Every labelled graph with no isolated vertex on n <= 5 vertices: CPAA
    against LAPACK for a fixed non-uniform p."""
    p = np.arange(1, n + 1, dtype=float)
    p /= p.sum()
    for g in ci.all_graphs(n):
        rp, cx = g.numpy()
        pi, _ = O.solve(rp, cx, p, 0.85, 1e-14)
        assert np.abs(pi - O.lapack_pagerank(rp, cx, p, 0.85)).sum() < 1e-13, g.name


def test_thread_count_does_not_change_result():
    g = ci.chung_lu(20000, 150000, seed=8)
    rp, cx = g.numpy()
    p = np.full(g.n, 1.0 / g.n)
    a = O.cpaa(rp, cx, p, 0.85, 20, nthreads=1)
    b = O.cpaa(rp, cx, p, 0.85, 20, nthreads=7)
    assert np.array_equal(a, b)


# -- fuzzing: random small graphs, self-loops included ---------------------------

def _random_graph(n, density, loops, seed):
    """Random symmetric graph on n vertices; every vertex gets degree >= 1 (a
    self-loop is one entry and counts once in d_u, Sec. 2.1)."""
    rng = np.random.default_rng(seed)
    edges = [(u, v) for u in range(n) for v in range(u + 1, n) if rng.random() < density]
    edges += [(u, u) for u in range(n) if rng.random() < loops]
    deg = np.zeros(n, dtype=int)
    for u, v in edges:
        deg[u] += 1
        deg[v] += u != v
    edges += [(u, u) for u in range(n) if deg[u] == 0]
    return ci.from_edges(n, edges, name="fuzz")


def test_fuzz_truncation_and_solution_on_random_small_graphs():
    """Random graphs of 1-12 vertices with self-loops, random p on the simplex,
    c and M: the recurrence equals the eigen path after M rounds in both
    normalisations, and a converged solve equals LAPACK."""
    hyp = pytest.importorskip("hypothesis")
    st = pytest.importorskip("hypothesis.strategies")

    @hyp.settings(max_examples=80, deadline=None, derandomize=True)
    @hyp.given(n=st.integers(1, 12), density=st.floats(0.0, 1.0), loops=st.floats(0.0, 1.0),
               seed=st.integers(0, 2 ** 31 - 1), c=st.floats(0.05, 0.97), M=st.integers(0, 25),
               single=st.booleans())
    def check(n, density, loops, seed, c, M, single):
        g = _random_graph(n, density, loops, seed)
        rp, cx = g.numpy()
        rng = np.random.default_rng(seed + 1)
        if single:
            p = np.zeros(n); p[rng.integers(n)] = 1.0
        else:
            p = rng.dirichlet(np.ones(n))
        scale = O.cheb_coeffs(c, 0)[0]
        for norm in (0, 1):
            a = O.cpaa(rp, cx, p, c, M, normalize=norm)
            b = O.eig_truncation(rp, cx, p, c, M, normalize=norm)
            assert np.abs(a - b).sum() <= 1e-12 * max(1.0, scale), (n, c, M, norm)
        pi, _ = O.solve(rp, cx, p, c, 1e-12)
        assert np.abs(pi - O.lapack_pagerank(rp, cx, p, c)).sum() <= 1e-11

    check()
