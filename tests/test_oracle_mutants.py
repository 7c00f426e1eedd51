"""Planted mistakes: each test copies the oracle's C source, plants one plausible
slip (a wrong sign, a dropped term, a wrong index, an off-by-one coefficient, a
skipped rotation, a wrong normalisation), builds it, and checks that the pins
reject the mutant.  Everything runs on the CPU."""
import ctypes
import math
import os
import subprocess

import numpy as np
import pytest

import cpaa_inputs as ci
from oracle import oracle as O
from oracle import build as B
from tests.test_oracle_pins import (negative_entry_truncation_failures, power_stop_failures,
                                    stopping_rule_truth_failures)

MUTANTS = {
    "recurrence_sign": ("s = 2.0 * s - j->T[u];", "s = 2.0 * s + j->T[u];"),
    "recurrence_factor": ("s = 2.0 * s - j->T[u];", "s = s - j->T[u];"),
    "first_round_degree_index": (
        "s = s + j->T[v] / (double)(rp[v + 1] - rp[v]);\n            }\n            j->Tpp[u] = s;\n            j->pibar[u] = j->pibar[u] + j->ck * s;\n        } else if",
        "s = s + j->T[v] / (double)(rp[u + 1] - rp[u]);\n            }\n            j->Tpp[u] = s;\n            j->pibar[u] = j->pibar[u] + j->ck * s;\n        } else if"),
    "later_round_degree_index": ("s = s + j->Tp[v] / (double)(rp[v + 1] - rp[v]);",
                                 "s = s + j->Tp[v] / (double)(rp[u + 1] - rp[u]);"),
    "gather_wrong_operand": ("s = s + j->Tp[v] / (double)(rp[v + 1] - rp[v]);",
                             "s = s + j->T[v] / (double)(rp[v + 1] - rp[v]);"),
    "c0_not_halved": ("pibar[i] = ck[0] / 2.0 * T[i];", "pibar[i] = ck[0] * T[i];"),
    "coeff_off_by_one": ("job.pibar = pibar; job.ck = ck[k];", "job.pibar = pibar; job.ck = ck[k - 1];"),
    "ratio_transposed": ("double ratio = c / (1.0 - s);", "double ratio = (1.0 - s) / c;"),
    "rotation_skipped": ("if (k >= 2) { /* rotate", "if (k >= 3) { /* rotate"),
    "scale_normalisation": ("pi[i] = (1.0 - c) * pibar[i];", "pi[i] = c * pibar[i];"),
    "err_bound_exponent": ("2.0 * pow(b, (double)(M + 1)) / (1.0 + b)", "2.0 * pow(b, (double)M) / (1.0 + b)"),
    "kappa_degree": ("q += p[i] * p[i] / d;", "q += p[i] * p[i] * d;"),
    "dense_wrong_degree": ("a[i * n + j] -= c / (double)(row_ptr[j + 1] - row_ptr[j]);",
                           "a[i * n + j] -= c / (double)(row_ptr[i + 1] - row_ptr[i]);"),
    "power_restart": ("job.T = x; job.Tpp = y; job.c = c; job.p = p;",
                      "job.T = p; job.Tpp = y; job.c = c; job.p = p;"),
    "bound_normalisation_term_dropped": (
        "double E = orc_err_bound(c, M);\n    if (normalize == 1) return E * kappa;\n"
        "    return E * kappa + (1.0 + E * kappa) * E / (1.0 - E);",
        "double E = orc_err_bound(c, M);\n    if (normalize == 1) return E * kappa;\n    return E * kappa;"),
    "rounds_needed_one_late": ("if (orc_l1_bound(c, M, kappa, normalize) < tol) return M;",
                               "if (orc_l1_bound(c, M, kappa, normalize) < tol) return M + 1;"),
    "power_stop_without_factor": ("if (c / (1.0 - c) * diff < tol) break;", "if (diff < tol) break;"),
    "normaliser_sums_magnitudes": ("for (int64_t i = 0; i < n; ++i) s += pibar[i];",
                                   "for (int64_t i = 0; i < n; ++i) s += fabs(pibar[i]);"),
}


# Slips in the series on [lambda_lo, 1] (the interval form): each must fail
# the interval pins below.
INTERVAL_MUTANTS = {
    "interval_first_round_no_shift": ("s = (s - j->mid * j->T[u]) / j->half;", "s = s / j->half;"),
    "interval_later_round_no_scale": ("s = 2.0 * (s - j->mid * j->Tp[u]) / j->half - j->T[u];",
                                      "s = 2.0 * (s - j->mid * j->Tp[u]) - j->T[u];"),
    "interval_shift_of_older_iterate": ("s = 2.0 * (s - j->mid * j->Tp[u]) / j->half - j->T[u];",
                                        "s = 2.0 * (s - j->mid * j->T[u]) / j->half - j->T[u];"),
    "interval_coeff_factor_dropped": ("for (int k = 0; k <= M; ++k) ck[k] = ck[k] / (1.0 - c * mid);",
                                      "for (int k = 0; k <= M; ++k) ck[k] = ck[k];"),
    "interval_chat_unscaled": ("*chat = c * *half / (1.0 - c * *mid);", "*chat = c * *half;"),
    "interval_err_tail_sign": ("pow(bh, (double)(M + 1)) / (1.0 - bh);", "pow(bh, (double)(M + 1)) / (1.0 + bh);"),
    "loops_bound_factor": ("return -1.0 + 2.0 / (double)dmax;", "return -1.0 + 4.0 / (double)dmax;"),
    "loops_missing_loop_ignored": ("if (!loop) return -1.0;", "if (!loop) continue;"),
}


def _interval_pins():
    """The interval pins on a few cases (O._lib as it is); names that failed."""
    from tests.test_oracle_interval_pins import lam_min, looped_graphs, with_loops
    failed = []
    c, lo = 0.85, -0.6
    mid, half = 0.5 * (1 + lo), 0.5 * (1 - lo)
    if np.abs(O.cheb_coeffs_interval(c, lo, 12) - O.quadrature_coeffs_interval(c, lo, 12)).max() > 1e-12:
        failed.append("interval_coeffs")
    ck = O.cheb_coeffs_interval(c, lo, 4000)
    for M in (1, 5):
        if abs(O.err_bound_interval(c, lo, M) - (1 - c) * ck[M + 1:].sum()) > 1e-12:
            failed.append("interval_err")
            break
    for g in looped_graphs()[:4]:
        rp, cx = g.numpy()
        l = O.lambda_lo_loops(rp, cx)
        if not (lam_min(g) >= l - 1e-12) or l != -1.0 + 2.0 / np.diff(rp).max():
            failed.append("interval_certified")
        p = np.zeros(g.n)
        p[g.n // 2] = 1.0
        for M in (1, 2, 5):
            if np.abs(O.cpaa_interval(rp, cx, p, c, l, M) - O.eig_truncation_interval(rp, cx, p, c, l, M)).sum() > 1e-12:
                failed.append("interval_eig")
    g = with_loops(ci.cycle(5))
    rp, cx = g.numpy()
    rows = np.repeat(np.arange(g.n), np.diff(rp))
    keep = ~((rows == 2) & (cx == 2))
    rp2, cx2 = ci.from_edges(g.n, np.stack([rows[keep], cx[keep]], 1)).numpy()
    if O.lambda_lo_loops(rp2, cx2) != -1.0:
        failed.append("interval_no_loop")
    return failed


def test_unmutated_oracle_passes_interval_pins():
    assert _interval_pins() == []


@pytest.mark.parametrize("name", sorted(INTERVAL_MUTANTS))
def test_planted_mistake_in_interval_form_is_caught(name, tmp_path):
    old, new = INTERVAL_MUTANTS[name]
    src = open(B.SRC).read()
    assert src.count(old) == 1, "mutation anchor not unique: " + name
    path = tmp_path / "mutant.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off",
                    "-o", str(so), str(path), "-lm", "-lpthread"], check=True)
    saved = O._lib
    try:
        O._lib = O.configure(ctypes.CDLL(str(so)))
        failed = _interval_pins()
    finally:
        O._lib = saved
    assert failed, "planted mistake %r passed every interval pin" % name


def _pins():
    """Run the core pins against whatever library O._lib holds; return the
    names of the pins that failed."""
    failed = []
    c = 0.85
    ck = O.cheb_coeffs(c, 12)
    if np.abs(ck - O.quadrature_coeffs(c, 12)).max() > 1e-12:
        failed.append("coeffs")
    S = 1.0 / (1.0 - c)
    for M in (1, 5, 12):
        SM = ck[0] / 2 + ck[1:M + 1].sum()
        if abs(O.err_bound(c, M) - (1.0 - SM / S)) > 1e-13:
            failed.append("err_bound")
            break
    for g in (ci.random_small(30, 70, seed=1), ci.star(5), ci.chung_lu(200, 900, seed=3)):
        rp, cx = g.numpy()
        n = g.n
        p = (np.arange(n) % 4 + 1.0)
        p /= p.sum()
        ref = O.lapack_pagerank(rp, cx, p, c)
        for M in (1, 2, 5):
            for norm in (0, 1):
                if np.abs(O.cpaa(rp, cx, p, c, M, norm) - O.eig_truncation(rp, cx, p, c, M, norm)).sum() > 1e-12:
                    failed.append("eig_truncation")
        for norm in (0, 1):
            M = O.rounds_needed(c, 1e-12, O.kappa(rp, p), norm)
            if M < 0 or np.abs(O.cpaa(rp, cx, p, c, M, norm) - ref).sum() > 1e-12:
                failed.append("converged")
        # the stopping bound must hold and must not be loose by more than kappa
        k = O.kappa(rp, p)
        if not (1.0 <= k <= math.sqrt(rp[-1]) * np.sqrt((p * p).sum()) * (1 + 1e-12) + 1e-12):
            failed.append("kappa_range")
        d = np.diff(rp).astype(float)
        if abs(k - math.sqrt(d.sum()) * math.sqrt((p * p / d).sum())) > 1e-12 * k:
            failed.append("kappa_def")
        if np.abs(O.dense_pagerank(rp, cx, p, c) - ref).sum() > 1e-12:
            failed.append("dense")
        try:
            x, _ = O.power(rp, cx, p, c, tol=1e-13, max_iter=5000)
            if np.abs(x - ref).sum() > 1e-12:
                failed.append("power")
        except RuntimeError:
            failed.append("power")
    failed += stopping_rule_truth_failures(c)
    if power_stop_failures():
        failed.append("power_stop")
    failed += negative_entry_truncation_failures()
    return failed


def test_unmutated_oracle_passes_core_pins():
    assert _pins() == []


def _interval_spans(src):
    """Where the interval form's code sits (its two worker branches and its
    section): the core mutants are planted outside these spans, where lines
    the interval copy repeats appear once."""
    a = src.index("} else if (j->kind == 3) {")
    b = src.index("    return NULL;", a)
    c = src.index("/* Chebyshev series on a narrower interval")
    d = src.index("/* Power method (the paper's SPI baseline")
    return [(a, b), (c, d)]


def _plant_outside_interval(src, old, new, name):
    spans = _interval_spans(src)
    hits = [i for i in range(len(src)) if src.startswith(old, i) and not any(a <= i < b for a, b in spans)]
    assert len(hits) == 1, "mutation anchor not unique: " + name
    i = hits[0]
    return src[:i] + new + src[i + len(old):]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(B.SRC).read()
    path = tmp_path / "mutant.c"
    path.write_text(_plant_outside_interval(src, old, new, name))
    so = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off",
                    "-o", str(so), str(path), "-lm", "-lpthread"], check=True)
    saved = O._lib
    try:
        O._lib = O.configure(ctypes.CDLL(str(so)))
        failed = _pins()
    finally:
        O._lib = saved
    assert failed, "planted mistake %r passed every pin" % name


# Slips in the a-posteriori rule (Python, in oracle.py): each copy of the
# function gets one and must fail the rule's hand cases.
PY_MUTANTS = {
    "posteriori_no_factor_2": ("l1_bound(c, M, 2.0 * m, normalize)", "l1_bound(c, M, m, normalize)"),
    "posteriori_skips_T0": ("m = float(l1_hist[0])", "m = 0.0"),
    "posteriori_current_term": ("m = max(m, float(l1_hist[M]))", "m = float(l1_hist[M])"),
    "posteriori_lagging_max": ("m = max(m, float(l1_hist[M]))", "m = max(m, float(l1_hist[M - 1]))"),
    "posteriori_reports_next_round": ("            return M\n", "            return M + 1\n"),
}


@pytest.mark.parametrize("name", sorted(PY_MUTANTS))
def test_planted_mistake_in_posteriori_rule_is_caught(name):
    import inspect
    import textwrap
    from tests.test_oracle_pins import posteriori_hand_failures
    src = textwrap.dedent(inspect.getsource(O.rounds_posteriori))
    old, new = PY_MUTANTS[name]
    assert src.count(old) == 1, name
    ns = {"l1_bound": O.l1_bound}
    exec(src.replace(old, new), ns)
    assert posteriori_hand_failures(ns["rounds_posteriori"]) != [], name
