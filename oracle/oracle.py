"""Python face of the CPAA oracle (test infrastructure only).

Two kinds of reference live here:

* ctypes wrappers around ``cpaa_oracle.c`` (plain FP64 loops in CSR order):
  the Chebyshev coefficients, the error bound of Eq. 41, CPAA as in
  Algorithm 1 (Sec. 4.1), the power method (the paper's ground truth,
  Sec. 5.1) and a dense Gaussian-elimination solve of (I - cP) x = (1-c) p
  (Sec. 2.1);
* numpy routines that reach the same quantities another way, used to pin the
  C code: LAPACK's dense solve and the eigen-decomposition of the symmetric
  S = D^-1/2 A D^-1/2 (similar to P = A D^-1, which is why P's spectrum is
  real, Lemma 2), which gives the exact M-term truncation for any M.

Only tests, the smoke check and the benchmark's CPU-baseline leg may use it.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None

_i64 = ctypes.c_int64
_int = ctypes.c_int
_dbl = ctypes.c_double
_pi32 = ctypes.POINTER(ctypes.c_int32)
_pf64 = ctypes.POINTER(ctypes.c_double)


def lib():
    """Load (building first if needed) the C oracle."""
    global _lib
    if _lib is None:
        _lib = configure(ctypes.CDLL(_build.build()))
    return _lib


def configure(L):
    """Declare the C signatures on a loaded oracle library."""
    if True:
        L.orc_beta.restype = _dbl
        L.orc_beta.argtypes = [_dbl]
        L.orc_cheb_coeffs.restype = None
        L.orc_cheb_coeffs.argtypes = [_dbl, _int, _pf64]
        L.orc_err_bound.restype = _dbl
        L.orc_err_bound.argtypes = [_dbl, _int]
        L.orc_kappa.restype = _dbl
        L.orc_kappa.argtypes = [_i64, _pi32, _pf64]
        L.orc_l1_bound.restype = _dbl
        L.orc_l1_bound.argtypes = [_dbl, _int, _dbl, _int]
        L.orc_rounds_needed.restype = _int
        L.orc_rounds_needed.argtypes = [_dbl, _dbl, _dbl, _int, _int]
        L.orc_cpaa.restype = _int
        L.orc_cpaa.argtypes = [_i64, _pi32, _pi32, _pf64, _dbl, _int, _int, _int,
                               _pf64, _pf64, _pf64]
        L.orc_power.restype = _int
        L.orc_power.argtypes = [_i64, _pi32, _pi32, _pf64, _dbl, _dbl, _int, _int, _pf64]
        L.orc_dense_pagerank.restype = _int
        L.orc_dense_pagerank.argtypes = [_i64, _pi32, _pi32, _pf64, _dbl, _pf64]
        L.orc_cheb_coeffs_interval.restype = None
        L.orc_cheb_coeffs_interval.argtypes = [_dbl, _dbl, _int, _pf64]
        L.orc_err_bound_interval.restype = _dbl
        L.orc_err_bound_interval.argtypes = [_dbl, _dbl, _int]
        L.orc_l1_bound_interval.restype = _dbl
        L.orc_l1_bound_interval.argtypes = [_dbl, _dbl, _int, _dbl, _int]
        L.orc_rounds_needed_interval.restype = _int
        L.orc_rounds_needed_interval.argtypes = [_dbl, _dbl, _dbl, _dbl, _int, _int]
        L.orc_lambda_lo_loops.restype = _dbl
        L.orc_lambda_lo_loops.argtypes = [_i64, _pi32, _pi32]
        L.orc_cpaa_interval.restype = _int
        L.orc_cpaa_interval.argtypes = [_i64, _pi32, _pi32, _pf64, _dbl, _dbl, _int, _int, _int, _pf64]
    return L


def _i32(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(_pi32)


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_pf64)


def default_threads():
    return max(1, min(64, os.cpu_count() or 1))


# -- coefficients and bounds (Sec. 2.2, Sec. 4.2) ---------------------------

def beta(c):
    return lib().orc_beta(float(c))


def cheb_coeffs(c, M):
    """c_0 .. c_M of 1/(1 - c x) (Sec. 2.2; ratio from Proposition 1's proof)."""
    out = np.empty(M + 1, dtype=np.float64)
    lib().orc_cheb_coeffs(float(c), int(M), out.ctypes.data_as(_pf64))
    return out


def err_bound(c, M):
    """ERR_M of Eq. 41."""
    return lib().orc_err_bound(float(c), int(M))


def kappa(row_ptr, p):
    rp, rpp = _i32(row_ptr)
    pv, pvp = _f64(p)
    return lib().orc_kappa(len(rp) - 1, rpp, pvp)


def l1_bound(c, M, kap, normalize=0):
    return lib().orc_l1_bound(float(c), int(M), float(kap), int(normalize))


def rounds_needed(c, tol, kap, normalize=0, max_rounds=10000):
    return lib().orc_rounds_needed(float(c), float(tol), float(kap), int(normalize),
                                   int(max_rounds))


def rounds_posteriori(c, tol, l1_hist, normalize=0, max_rounds=None):
    """The a-posteriori stopping rule: the first M >= 1 with
    l1_bound(c, M, 2 max_{j<=M} ||T_j p||_1) < tol, where l1_hist[j] is
    ||T_j p||_1 (j = 0 .. len - 1) from ``cpaa(..., history=True)``; None if no
    M within the history (or max_rounds) passes.

    Eq. 41's ERR_M bounds the neglected coefficient mass; the L1 error of pi is
    at most ERR_M times the size of the neglected T_k p.  The rigorous rule
    bounds that size by kappa; this rule estimates it from the terms already
    computed (twice their running maximum).  It is an estimate, not a proof,
    which is why the tests check its result against the exact solution.
    """
    last = len(l1_hist) - 1 if max_rounds is None else min(max_rounds, len(l1_hist) - 1)
    m = float(l1_hist[0])
    for M in range(1, last + 1):
        m = max(m, float(l1_hist[M]))
        if l1_bound(c, M, 2.0 * m, normalize) < tol:
            return M
    return None


# -- the method ---------------------------------------------------------------

def cpaa(row_ptr, col_idx, p, c, M, normalize=0, nthreads=None, history=False):
    """CPAA after M rounds (Algorithm 1 with the readings in cpaa_oracle.c).

    Returns pi (FP64) or (pi, mass[0..M], l1[0..M]) when ``history``.
    """
    rp, rpp = _i32(row_ptr)
    ci, cip = _i32(col_idx)
    pv, pvp = _f64(p)
    n = len(rp) - 1
    pi = np.empty(n, dtype=np.float64)
    mass = np.empty(M + 1, dtype=np.float64) if history else None
    l1 = np.empty(M + 1, dtype=np.float64) if history else None
    rc = lib().orc_cpaa(n, rpp, cip, pvp, float(c), int(M), int(normalize),
                        int(nthreads or default_threads()), pi.ctypes.data_as(_pf64),
                        mass.ctypes.data_as(_pf64) if history else None,
                        l1.ctypes.data_as(_pf64) if history else None)
    if rc != 0:
        raise ValueError("orc_cpaa failed")
    return (pi, mass, l1) if history else pi


def power(row_ptr, col_idx, p, c, tol=1e-14, max_iter=100000, nthreads=None, rounds=None):
    """Power method to an L1 bound of ``tol`` (the paper's SPI, Sec. 5.1), or for
    exactly ``rounds`` rounds when that is given."""
    rp, rpp = _i32(row_ptr)
    ci, cip = _i32(col_idx)
    pv, pvp = _f64(p)
    x = np.empty(len(rp) - 1, dtype=np.float64)
    if rounds is not None:  # a zero tolerance never stops early
        tol, max_iter = 0.0, int(rounds)
    it = lib().orc_power(len(rp) - 1, rpp, cip, pvp, float(c), float(tol), int(max_iter),
                         int(nthreads or default_threads()), x.ctypes.data_as(_pf64))
    if rounds is not None:
        return x, int(rounds)
    if it < 0:
        raise RuntimeError("power method did not reach tol")
    return x, it


def dense_pagerank(row_ptr, col_idx, p, c):
    """Gaussian elimination on (I - cP) x = (1-c) p (Sec. 2.1); n small."""
    rp, rpp = _i32(row_ptr)
    ci, cip = _i32(col_idx)
    pv, pvp = _f64(p)
    x = np.empty(len(rp) - 1, dtype=np.float64)
    if lib().orc_dense_pagerank(len(rp) - 1, rpp, cip, pvp, float(c),
                                x.ctypes.data_as(_pf64)) != 0:
        raise RuntimeError("dense solve failed")
    return x


def solve(row_ptr, col_idx, p, c, tol, normalize=0, nthreads=None):
    """CPAA run for the rounds the rigorous L1 bound asks for; returns (pi, M)."""
    M = rounds_needed(c, tol, kappa(row_ptr, p), normalize)
    return cpaa(row_ptr, col_idx, p, c, M, normalize, nthreads), M


# -- the series on a narrower interval [lambda_lo, 1] (Sec. 2.2's general
#    interval; see cpaa_oracle.c) ------------------------------------------------

def cheb_coeffs_interval(c, lambda_lo, M):
    out = np.empty(M + 1, dtype=np.float64)
    lib().orc_cheb_coeffs_interval(float(c), float(lambda_lo), int(M), out.ctypes.data_as(_pf64))
    return out


def err_bound_interval(c, lambda_lo, M):
    return lib().orc_err_bound_interval(float(c), float(lambda_lo), int(M))


def l1_bound_interval(c, lambda_lo, M, kap, normalize=0):
    return lib().orc_l1_bound_interval(float(c), float(lambda_lo), int(M), float(kap), int(normalize))


def rounds_needed_interval(c, lambda_lo, tol, kap, normalize=0, max_rounds=10000):
    return lib().orc_rounds_needed_interval(float(c), float(lambda_lo), float(tol), float(kap),
                                            int(normalize), int(max_rounds))


def lambda_lo_loops(row_ptr, col_idx):
    """-1 + 2/d_max when every vertex has a self-loop, else -1."""
    rp, rpp = _i32(row_ptr)
    ci, cip = _i32(col_idx)
    return lib().orc_lambda_lo_loops(len(rp) - 1, rpp, cip)


def cpaa_interval(row_ptr, col_idx, p, c, lambda_lo, M, normalize=0, nthreads=None):
    """CPAA after M rounds of the series on [lambda_lo, 1]."""
    rp, rpp = _i32(row_ptr)
    ci, cip = _i32(col_idx)
    pv, pvp = _f64(p)
    n = len(rp) - 1
    pi = np.empty(n, dtype=np.float64)
    if lib().orc_cpaa_interval(n, rpp, cip, pvp, float(c), float(lambda_lo), int(M), int(normalize),
                               int(nthreads or default_threads()), pi.ctypes.data_as(_pf64)) != 0:
        raise ValueError("orc_cpaa_interval failed")
    return pi


# -- numpy cross-checks (independent of the C code) ---------------------------

def dense_matrix_P(row_ptr, col_idx):
    """P = A D^-1 as a dense array (Sec. 2.1)."""
    n = len(row_ptr) - 1
    A = np.zeros((n, n))
    for i in range(n):
        for e in range(row_ptr[i], row_ptr[i + 1]):
            A[i, col_idx[e]] = 1.0
    d = A.sum(axis=0)
    return A / d[None, :], A, d


def lapack_pagerank(row_ptr, col_idx, p, c):
    """pi* = (1-c)(I - cP)^-1 p by numpy.linalg.solve."""
    P, _, _ = dense_matrix_P(row_ptr, col_idx)
    n = P.shape[0]
    return np.linalg.solve(np.eye(n) - c * P, (1.0 - c) * np.asarray(p, dtype=np.float64))


def eig_truncation(row_ptr, col_idx, p, c, M, normalize=0):
    """Exact M-term truncation (1-c)[c_0/2 p + sum_{k<=M} c_k T_k(P) p] through the
    eigen-decomposition of S = D^-1/2 A D^-1/2 (Eq. 31 with P's real spectrum,
    Lemma 2).  T_k(lambda) = cos(k arccos lambda) (Sec. 2.2); the coefficients
    come from the integral of Sec. 2.2 evaluated by numpy quadrature, not from
    the C code."""
    _, A, d = dense_matrix_P(row_ptr, col_idx)
    s = 1.0 / np.sqrt(d)
    S = s[:, None] * A * s[None, :]
    lam, U = np.linalg.eigh(S)
    lam = np.clip(lam, -1.0, 1.0)
    ck = quadrature_coeffs(c, M)
    theta = np.arccos(lam)
    f = ck[0] / 2.0 + sum(ck[k] * np.cos(k * theta) for k in range(1, M + 1))
    q = U.T @ (s * np.asarray(p, dtype=np.float64))
    v = np.sqrt(d) * (U @ (f * q))
    if normalize == 0:
        return v / v.sum()
    return (1.0 - c) * v


def quadrature_coeffs(c, M, nodes=8192):
    """c_k = (2/pi) int_0^pi cos(kt) / (1 - c cos t) dt (Sec. 2.2) by the
    composite trapezoid rule, which is spectrally accurate for this smooth
    periodic integrand."""
    t = np.linspace(0.0, np.pi, nodes + 1)
    w = np.full(nodes + 1, np.pi / nodes)
    w[0] = w[-1] = np.pi / (2 * nodes)
    g = 1.0 / (1.0 - c * np.cos(t))
    return np.array([(2.0 / np.pi) * np.sum(w * np.cos(k * t) * g) for k in range(M + 1)])


def quadrature_coeffs_interval(c, lambda_lo, M, nodes=8192):
    """c_k = (2/pi) int_0^pi f(mid + half cos t) cos(kt) dt for f(x) = 1/(1 - cx)
    on [lambda_lo, 1] (Sec. 2.2's general interval), composite trapezoid rule;
    independent of the reduction to 1/(1 - chat cos t) the C code uses."""
    mid, half = 0.5 * (1.0 + lambda_lo), 0.5 * (1.0 - lambda_lo)
    t = np.linspace(0.0, np.pi, nodes + 1)
    w = np.full(nodes + 1, np.pi / nodes)
    w[0] = w[-1] = np.pi / (2 * nodes)
    g = 1.0 / (1.0 - c * (mid + half * np.cos(t)))
    return np.array([(2.0 / np.pi) * np.sum(w * np.cos(k * t) * g) for k in range(M + 1)])


def eig_truncation_interval(row_ptr, col_idx, p, c, lambda_lo, M, normalize=0):
    """The exact M-term truncation on [lambda_lo, 1] through eigh of S: each
    eigenvalue lambda enters as c_0/2 + sum_k c_k T_k((lambda - mid)/half),
    T_k(t) = cos(k arccos t), coefficients by quadrature."""
    _, A, d = dense_matrix_P(row_ptr, col_idx)
    s = 1.0 / np.sqrt(d)
    S = s[:, None] * A * s[None, :]
    lam, U = np.linalg.eigh(S)
    mid, half = 0.5 * (1.0 + lambda_lo), 0.5 * (1.0 - lambda_lo)
    t = np.clip((lam - mid) / half, -1.0, 1.0)
    ck = quadrature_coeffs_interval(c, lambda_lo, M)
    theta = np.arccos(t)
    f = ck[0] / 2.0 + sum(ck[k] * np.cos(k * theta) for k in range(1, M + 1))
    q = U.T @ (s * np.asarray(p, dtype=np.float64))
    v = np.sqrt(d) * (U @ (f * q))
    if normalize == 0:
        return v / v.sum()
    return (1.0 - c) * v
