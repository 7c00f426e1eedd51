/*
 * cpaa_oracle.c -- plain FP64 CPU oracle for CPAA, the Chebyshev Polynomial
 * Approximation Algorithm for PageRank on undirected graphs (Zhang, Tang, Yao,
 * Zhang, "A Parallel PageRank Algorithm For Undirected Graph").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct reference
 * that the GPU library is checked against.  Only the test suite, the smoke
 * check and the benchmark's CPU-baseline leg may load it; the library itself
 * never does.  It shares no code, header or constant with the CUDA path.
 *
 * Conventions (Sec. 2.1): A is the symmetric 0/1 adjacency matrix held as CSR
 * (row_ptr[n+1], col_idx[nnz], int32), d_i = number of CSR entries of row i
 * (a self-loop is one entry and counts once), P = A D^-1 (column stochastic),
 * and the PageRank vector is pi* = (1-c)(I - cP)^-1 p.
 *
 * Arithmetic is IEEE FP64 with no contraction (built with -ffp-contract=off);
 * every sum runs in ascending CSR order.  Rows may be split over worker threads
 * (the vertex sets S_j of Algorithm 1); each row is still summed by one thread
 * in the same order, so the result does not depend on the thread count.
 *
 * Every function states the passage of the paper it follows.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* Chebyshev coefficients of f(x) = 1/(1 - c x) (Sec. 2.2, Sec. 4.2.1) */
/* ------------------------------------------------------------------ */

/* beta = (1 - sqrt(1 - c^2)) / c : the constant ratio c_k / c_{k-1}
 * (Proposition 1's proof gives c_{k-1}/c_k = c / (1 - sqrt(1 - c^2))), and
 * the beta of Eq. 41. */
double orc_beta(double c) { return (1.0 - sqrt(1.0 - c * c)) / c; }

/* c_0 .. c_M.  c_0 = 2 / sqrt(1 - c^2) is printed in the proof of
 * Proposition 1; every later coefficient is the previous one divided by the
 * constant ratio c_{k-1}/c_k proved there.  (The defining integral,
 * c_k = (2/pi) int_0^pi cos(kt)/(1 - c cos t) dt, Sec. 2.2, is the test pin.) */
void orc_cheb_coeffs(double c, int M, double *ck) {
    double s = sqrt(1.0 - c * c);
    double ratio = c / (1.0 - s); /* c_{k-1} / c_k */
    ck[0] = 2.0 / s;
    for (int k = 1; k <= M; ++k) ck[k] = ck[k - 1] / ratio;
}

/* ERR_M = 1 - S_M / S = 2 beta^(M+1) / (1 + beta)   (Eq. 41, Sec. 4.2.2). */
double orc_err_bound(double c, int M) {
    double b = orc_beta(c);
    return 2.0 * pow(b, (double)(M + 1)) / (1.0 + b);
}

/* kappa = sqrt(sum_i d_i) * || D^-1/2 p ||_2.
 * P = D^1/2 S D^-1/2 with S = D^-1/2 A D^-1/2 symmetric (the reason the
 * eigenvalues are real, Lemma 2), so ||T_k(P) p||_1 <= kappa for every k
 * (|T_k| <= 1 on [-1,1], Sec. 2.2 property (1), then Cauchy-Schwarz). */
double orc_kappa(int64_t n, const int32_t *row_ptr, const double *p) {
    double sum_d = 0.0, q = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double d = (double)(row_ptr[i + 1] - row_ptr[i]);
        sum_d += d;
        q += p[i] * p[i] / d;
    }
    return sqrt(sum_d) * sqrt(q);
}

/* Bound on || pi_M - pi* ||_1 after M rounds.
 * normalize = 1 ((1-c) scaling, Sec. 2.1): the truncation error is
 *   (1-c) sum_{k>M} c_k T_k(P) p, whose L1 norm is at most ERR_M * kappa
 *   (the coefficients are positive and (1-c) sum_{k>M} c_k = ERR_M).
 * normalize = 0 (divide by the sum, last line of Algorithm 1): the sum of the
 *   (1-c)-scaled iterate is exactly 1 - ERR_M (every T_k(P) keeps e^T p = 1),
 *   so dividing by it adds at most (1 + E kappa) E / (1 - E). */
double orc_l1_bound(double c, int M, double kappa, int normalize) {
    double E = orc_err_bound(c, M);
    if (normalize == 1) return E * kappa;
    return E * kappa + (1.0 + E * kappa) * E / (1.0 - E);
}

/* Smallest M >= 1 whose bound is below tol (at most max_rounds). */
int orc_rounds_needed(double c, double tol, double kappa, int normalize, int max_rounds) {
    for (int M = 1; M <= max_rounds; ++M)
        if (orc_l1_bound(c, M, kappa, normalize) < tol) return M;
    return -1;
}

/* ------------------------------------------------------------------ */
/* Worker threads over vertex sets S_j (Algorithm 1, second line)       */
/* ------------------------------------------------------------------ */

typedef struct {
    int kind; /* 0: first round, 1: later round, 2: power-method round,
                 3 / 4: first / later round of the interval form (below) */
    int64_t n, lo, hi;
    const int32_t *row_ptr, *col_idx;
    const double *T;   /* T_{k-1} (or the power iterate) */
    const double *Tp;  /* T_k                            */
    double *Tpp;       /* T_{k+1} (output)               */
    double *pibar;
    double ck, c;
    const double *p;
    double mid, half;  /* interval form: centre and half-width of [lambda_lo, 1] */
} orc_job;

static void *orc_worker(void *arg) {
    orc_job *j = (orc_job *)arg;
    const int32_t *rp = j->row_ptr, *ci = j->col_idx;
    for (int64_t u = j->lo; u < j->hi; ++u) {
        double s = 0.0;
        if (j->kind == 0) {
            /* k = 1: T'_u = sum_{v in N(u)} T_v / deg(v); pibar_u += c_1 T'_u */
            for (int32_t e = rp[u]; e < rp[u + 1]; ++e) {
                int32_t v = ci[e];
                s = s + j->T[v] / (double)(rp[v + 1] - rp[v]);
            }
            j->Tpp[u] = s;
            j->pibar[u] = j->pibar[u] + j->ck * s;
        } else if (j->kind == 1) {
            /* k >= 2: T''_u = 2 sum_{v in N(u)} T'_v / deg(v) - T_u;
             *         pibar_u += c_k T''_u                                 */
            for (int32_t e = rp[u]; e < rp[u + 1]; ++e) {
                int32_t v = ci[e];
                s = s + j->Tp[v] / (double)(rp[v + 1] - rp[v]);
            }
            s = 2.0 * s - j->T[u];
            j->Tpp[u] = s;
            j->pibar[u] = j->pibar[u] + j->ck * s;
        } else if (j->kind == 2) {
            /* power method (Jacobi) round: x'_u = c sum_v x_v / deg(v) + (1-c) p_u */
            for (int32_t e = rp[u]; e < rp[u + 1]; ++e) {
                int32_t v = ci[e];
                s = s + j->T[v] / (double)(rp[v + 1] - rp[v]);
            }
            j->Tpp[u] = j->c * s + (1.0 - j->c) * j->p[u];
        } else if (j->kind == 3) {
            /* interval form, k = 1: T'_u = ((P T)_u - mid T_u) / half */
            for (int32_t e = rp[u]; e < rp[u + 1]; ++e) {
                int32_t v = ci[e];
                s = s + j->T[v] / (double)(rp[v + 1] - rp[v]);
            }
            s = (s - j->mid * j->T[u]) / j->half;
            j->Tpp[u] = s;
            j->pibar[u] = j->pibar[u] + j->ck * s;
        } else {
            /* interval form, k >= 2: T''_u = 2 ((P T')_u - mid T'_u) / half - T_u */
            for (int32_t e = rp[u]; e < rp[u + 1]; ++e) {
                int32_t v = ci[e];
                s = s + j->Tp[v] / (double)(rp[v + 1] - rp[v]);
            }
            s = 2.0 * (s - j->mid * j->Tp[u]) / j->half - j->T[u];
            j->Tpp[u] = s;
            j->pibar[u] = j->pibar[u] + j->ck * s;
        }
    }
    return NULL;
}

/* One parallel round: rows split into K contiguous vertex sets; joining the
 * threads is the barrier between rounds (Sec. 4.1: rounds depend on each
 * other, vertices inside a round do not). */
static void orc_round(orc_job base, int nthreads) {
    if (nthreads <= 1 || base.n < 4096) {
        base.lo = 0;
        base.hi = base.n;
        orc_worker(&base);
        return;
    }
    pthread_t th[256];
    orc_job jobs[256];
    if (nthreads > 256) nthreads = 256;
    for (int t = 0; t < nthreads; ++t) {
        jobs[t] = base;
        jobs[t].lo = base.n * t / nthreads;
        jobs[t].hi = base.n * (t + 1) / nthreads;
        pthread_create(&th[t], NULL, orc_worker, &jobs[t]);
    }
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
}

/* ------------------------------------------------------------------ */
/* CPAA, Algorithm 1 (Sec. 4.1) with the readings listed below          */
/* ------------------------------------------------------------------ */
/*
 * Readings of Algorithm 1 (the printed listing has slips):
 *  - T_0 = p (the listing sets T_i = 1, i.e. p = e, and the result is
 *    normalised at the end; with a personalised p the start is p itself).
 *  - k = 1 computes T_1 = P p; k >= 2 computes T_k = 2 P T_{k-1} - T_{k-2}
 *    (Chebyshev property (3), Sec. 2.2, and the iteration of Sec. 4.1 (2)).
 *    The buffers rotate only once T_1 exists.
 *  - The accumulation adds c_k T_k to the accumulator of the row u being
 *    updated.
 *  - normalize = 0: pi = pibar / sum(pibar) (last line of Algorithm 1);
 *    normalize = 1: pi = (1-c) pibar (Sec. 2.1).
 * mass[k] = sum_u T_k[u] and l1[k] = sum_u |T_k[u]| for k = 0..M when the
 * pointers are non-NULL (the mass view of Sec. 4.1: the total stays e^T p).
 * Returns 0, or -1 on bad arguments / allocation failure.
 */
int orc_cpaa(int64_t n, const int32_t *row_ptr, const int32_t *col_idx, const double *p,
             double c, int M, int normalize, int nthreads, double *pi, double *mass, double *l1) {
    if (n <= 0 || M < 0 || !(c > 0.0 && c < 1.0)) return -1;
    double *ck = (double *)malloc(sizeof(double) * (size_t)(M + 1));
    double *T = (double *)malloc(sizeof(double) * (size_t)n);
    double *Tp = (double *)malloc(sizeof(double) * (size_t)n);
    double *Tpp = (double *)malloc(sizeof(double) * (size_t)n);
    if (!ck || !T || !Tp || !Tpp) {
        free(ck); free(T); free(Tp); free(Tpp);
        return -1;
    }
    orc_cheb_coeffs(c, M, ck);
    double *pibar = pi; /* accumulate in the output buffer */
    for (int64_t i = 0; i < n; ++i) {
        T[i] = p[i];
        pibar[i] = ck[0] / 2.0 * T[i];
    }
    if (mass || l1) {
        double m = 0.0, a = 0.0;
        for (int64_t i = 0; i < n; ++i) { m += T[i]; a += fabs(T[i]); }
        if (mass) mass[0] = m;
        if (l1) l1[0] = a;
    }
    for (int k = 1; k <= M; ++k) {
        orc_job job;
        memset(&job, 0, sizeof(job));
        job.n = n; job.row_ptr = row_ptr; job.col_idx = col_idx;
        job.pibar = pibar; job.ck = ck[k];
        double *out;
        if (k == 1) {
            job.kind = 0; job.T = T; job.Tpp = Tp; out = Tp;
        } else {
            job.kind = 1; job.T = T; job.Tp = Tp; job.Tpp = Tpp; out = Tpp;
        }
        orc_round(job, nthreads);
        if (mass || l1) {
            double m = 0.0, a = 0.0;
            for (int64_t i = 0; i < n; ++i) { m += out[i]; a += fabs(out[i]); }
            if (mass) mass[k] = m;
            if (l1) l1[k] = a;
        }
        if (k >= 2) { /* rotate: T <- T', T' <- T'' */
            double *t = T; T = Tp; Tp = Tpp; Tpp = t;
        }
    }
    if (normalize == 0) {
        double s = 0.0;
        for (int64_t i = 0; i < n; ++i) s += pibar[i];
        for (int64_t i = 0; i < n; ++i) pi[i] = pibar[i] / s;
    } else {
        for (int64_t i = 0; i < n; ++i) pi[i] = (1.0 - c) * pibar[i];
    }
    free(ck); free(T); free(Tp); free(Tpp);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Chebyshev series on a narrower interval [lambda_lo, 1]                */
/* (the general-interval series of Sec. 2.2; Sec. 6 names other        */
/*  approximations as future work)                                      */
/* ------------------------------------------------------------------ */
/*
 * Sec. 2.2 gives the Chebyshev series of f on a general interval [a, b]: the
 * expansion variable is t = (2x - (a+b)) / (b-a), which maps [a, b] onto
 * [-1, 1], and the coefficients are the integrals printed there.  Reading
 * (the printed series writes T_k(x) for T_k(t), and its coefficient integral
 * lacks the 1/pi of the [-1, 1] case given right after it): with the centre
 * mid = (a+b)/2 and half-width half = (b-a)/2, x = mid + half cos(theta),
 *     c_k = (2/pi) int_0^pi f(mid + half cos theta) cos(k theta) d theta.
 * Here [a, b] = [lambda_lo, 1] holds the whole spectrum of P (real, Lemma 2),
 * and f(x) = 1/(1 - c x) becomes
 *     f(mid + half cos theta) = 1/(1 - c mid) * 1/(1 - chat cos theta),
 *     chat = c half / (1 - c mid)  (< c when lambda_lo > -1),
 * so c_k = c_k(chat) / (1 - c mid) with the [-1, 1] coefficients of chat, and
 * the recurrence runs on Q = (P - mid I) / half, whose spectrum lies in
 * [-1, 1]: T_0 = p, T_1 = Q p, T_{k+1} = 2 Q T_k - T_{k-1}.  lambda_lo = -1
 * gives back Algorithm 1 exactly (mid = 0, half = 1, chat = c).
 */
static void orc_interval(double c, double lambda_lo, double *mid, double *half, double *chat) {
    *mid = 0.5 * (1.0 + lambda_lo);
    *half = 0.5 * (1.0 - lambda_lo);
    *chat = c * *half / (1.0 - c * *mid);
}

/* c_0 .. c_M of 1/(1 - c x) expanded on [lambda_lo, 1]. */
void orc_cheb_coeffs_interval(double c, double lambda_lo, int M, double *ck) {
    double mid, half, chat;
    orc_interval(c, lambda_lo, &mid, &half, &chat);
    orc_cheb_coeffs(chat, M, ck);
    for (int k = 0; k <= M; ++k) ck[k] = ck[k] / (1.0 - c * mid);
}

/* The interval form's ERR_M: (1-c) sum_{k>M} c_k, the mass the truncation
 * leaves out (every T_k(Q) keeps e^T p, because e^T Q = e^T).  With
 * c_k = c_0 betahat^k this is (1-c) c_0 betahat^(M+1) / (1 - betahat). */
double orc_err_bound_interval(double c, double lambda_lo, int M) {
    double mid, half, chat;
    orc_interval(c, lambda_lo, &mid, &half, &chat);
    double bh = orc_beta(chat);
    double c0 = 2.0 / sqrt(1.0 - chat * chat) / (1.0 - c * mid);
    return (1.0 - c) * c0 * pow(bh, (double)(M + 1)) / (1.0 - bh);
}

/* The L1 bound of orc_l1_bound with the interval form's ERR_M: kappa still
 * bounds ||T_k(Q) p||_1, since Q is similar to the symmetric
 * (S - mid I) / half, whose spectrum lies in [-1, 1]. */
double orc_l1_bound_interval(double c, double lambda_lo, int M, double kappa, int normalize) {
    double E = orc_err_bound_interval(c, lambda_lo, M);
    if (normalize == 1) return E * kappa;
    return E * kappa + (1.0 + E * kappa) * E / (1.0 - E);
}

int orc_rounds_needed_interval(double c, double lambda_lo, double tol, double kappa, int normalize,
                               int max_rounds) {
    for (int M = 1; M <= max_rounds; ++M)
        if (orc_l1_bound_interval(c, lambda_lo, M, kappa, normalize) < tol) return M;
    return -1;
}

/* A lower bound on the spectrum of S = D^-1/2 A D^-1/2 (hence of P) that holds
 * for every graph with a self-loop on every vertex: A = A' + I and D = D' + I
 * with the loop-free A', D', and D' + A' is positive semidefinite (its
 * quadratic form is the sum over edges of (x_i + x_j)^2), so A + D >= 2I and
 * S + I = D^-1/2 (A + D) D^-1/2 >= 2 D^-1 >= (2 / d_max) I.  Returns
 * -1 + 2 / d_max, or -1 (no bound beyond Lemma 2's) when a vertex has no loop. */
double orc_lambda_lo_loops(int64_t n, const int32_t *row_ptr, const int32_t *col_idx) {
    int32_t dmax = 0;
    for (int64_t u = 0; u < n; ++u) {
        int loop = 0;
        for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e)
            if (col_idx[e] == (int32_t)u) loop = 1;
        if (!loop) return -1.0;
        if (row_ptr[u + 1] - row_ptr[u] > dmax) dmax = row_ptr[u + 1] - row_ptr[u];
    }
    return -1.0 + 2.0 / (double)dmax;
}

/* CPAA on [lambda_lo, 1]: Algorithm 1 with the coefficients and the
 * recurrence above (same readings as orc_cpaa; lambda_lo = -1 is orc_cpaa).
 * normalize = 1 scales by (1-c) (Sec. 2.1), as the coefficients already hold
 * the 1/(1 - c mid). */
int orc_cpaa_interval(int64_t n, const int32_t *row_ptr, const int32_t *col_idx, const double *p,
                      double c, double lambda_lo, int M, int normalize, int nthreads, double *pi) {
    if (n <= 0 || M < 0 || !(c > 0.0 && c < 1.0) || !(lambda_lo >= -1.0 && lambda_lo < 1.0)) return -1;
    double mid, half, chat;
    orc_interval(c, lambda_lo, &mid, &half, &chat);
    double *ck = (double *)malloc(sizeof(double) * (size_t)(M + 1));
    double *T = (double *)malloc(sizeof(double) * (size_t)n);
    double *Tp = (double *)malloc(sizeof(double) * (size_t)n);
    double *Tpp = (double *)malloc(sizeof(double) * (size_t)n);
    if (!ck || !T || !Tp || !Tpp) {
        free(ck); free(T); free(Tp); free(Tpp);
        return -1;
    }
    orc_cheb_coeffs_interval(c, lambda_lo, M, ck);
    double *pibar = pi;
    for (int64_t i = 0; i < n; ++i) {
        T[i] = p[i];
        pibar[i] = ck[0] / 2.0 * T[i];
    }
    for (int k = 1; k <= M; ++k) {
        orc_job job;
        memset(&job, 0, sizeof(job));
        job.n = n; job.row_ptr = row_ptr; job.col_idx = col_idx;
        job.pibar = pibar; job.ck = ck[k]; job.mid = mid; job.half = half;
        if (k == 1) {
            job.kind = 3; job.T = T; job.Tpp = Tp;
        } else {
            job.kind = 4; job.T = T; job.Tp = Tp; job.Tpp = Tpp;
        }
        orc_round(job, nthreads);
        if (k >= 2) { /* rotate: T <- T', T' <- T'' */
            double *t = T; T = Tp; Tp = Tpp; Tpp = t;
        }
    }
    if (normalize == 0) {
        double s = 0.0;
        for (int64_t i = 0; i < n; ++i) s += pibar[i];
        for (int64_t i = 0; i < n; ++i) pi[i] = pibar[i] / s;
    } else {
        for (int64_t i = 0; i < n; ++i) pi[i] = (1.0 - c) * pibar[i];
    }
    free(ck); free(T); free(Tp); free(Tpp);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Power method (the paper's SPI baseline and ground truth, Sec. 5.1)   */
/* ------------------------------------------------------------------ */
/* x <- c P x + (1-c) p from x = p, until (c/(1-c)) ||x_{t+1} - x_t||_1 < tol
 * (cP has L1 norm c, so that quantity bounds the distance to pi*).
 * Returns the number of rounds, or -1 if max_iter was reached first. */
int orc_power(int64_t n, const int32_t *row_ptr, const int32_t *col_idx, const double *p,
              double c, double tol, int max_iter, int nthreads, double *x) {
    double *y = (double *)malloc(sizeof(double) * (size_t)n);
    if (!y) return -1;
    for (int64_t i = 0; i < n; ++i) x[i] = p[i];
    int t;
    for (t = 1; t <= max_iter; ++t) {
        orc_job job;
        memset(&job, 0, sizeof(job));
        job.kind = 2; job.n = n; job.row_ptr = row_ptr; job.col_idx = col_idx;
        job.T = x; job.Tpp = y; job.c = c; job.p = p;
        orc_round(job, nthreads);
        double diff = 0.0;
        for (int64_t i = 0; i < n; ++i) diff += fabs(y[i] - x[i]);
        memcpy(x, y, sizeof(double) * (size_t)n);
        if (c / (1.0 - c) * diff < tol) break;
    }
    free(y);
    return t <= max_iter ? t : -1;
}

/* ------------------------------------------------------------------ */
/* Dense solve of (I - cP) x = (1-c) p (Sec. 2.1), n small              */
/* ------------------------------------------------------------------ */
/* Gaussian elimination with partial pivoting on the dense n x n system.
 * Returns 0, or -1 on allocation failure / a zero pivot. */
int orc_dense_pagerank(int64_t n, const int32_t *row_ptr, const int32_t *col_idx,
                       const double *p, double c, double *x) {
    double *a = (double *)calloc((size_t)(n * n), sizeof(double));
    double *b = (double *)malloc(sizeof(double) * (size_t)n);
    if (!a || !b) { free(a); free(b); return -1; }
    for (int64_t i = 0; i < n; ++i) {
        a[i * n + i] = 1.0;
        b[i] = (1.0 - c) * p[i];
    }
    /* P_ij = a_ij / d_j; row i of A lists its neighbours j. */
    for (int64_t i = 0; i < n; ++i)
        for (int32_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            int32_t j = col_idx[e];
            a[i * n + j] -= c / (double)(row_ptr[j + 1] - row_ptr[j]);
        }
    for (int64_t k = 0; k < n; ++k) {
        int64_t piv = k;
        for (int64_t i = k + 1; i < n; ++i)
            if (fabs(a[i * n + k]) > fabs(a[piv * n + k])) piv = i;
        if (a[piv * n + k] == 0.0) { free(a); free(b); return -1; }
        if (piv != k) {
            for (int64_t j = 0; j < n; ++j) {
                double t = a[k * n + j]; a[k * n + j] = a[piv * n + j]; a[piv * n + j] = t;
            }
            double t = b[k]; b[k] = b[piv]; b[piv] = t;
        }
        for (int64_t i = k + 1; i < n; ++i) {
            double f = a[i * n + k] / a[k * n + k];
            if (f == 0.0) continue;
            for (int64_t j = k; j < n; ++j) a[i * n + j] -= f * a[k * n + j];
            b[i] -= f * b[k];
        }
    }
    for (int64_t i = n - 1; i >= 0; --i) {
        double s = b[i];
        for (int64_t j = i + 1; j < n; ++j) s -= a[i * n + j] * x[j];
        x[i] = s / a[i * n + i];
    }
    free(a); free(b);
    return 0;
}
