// status.cpp -- status strings, per-thread error text, defaults, and the
// host-side FP64 pieces of the method: the Chebyshev coefficient table and
// the stopping rule.
#include <cmath>
#include <cstring>

#include "internal.h"

namespace cpaa {

static thread_local std::string t_last_error;

cpaa_status fail(cpaa_status s, const std::string &msg) {
    t_last_error = msg;
    return s;
}

cpaa_status cuda_fail(cudaError_t e, const char *what) {
    t_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return CPAA_ENOMEM;
    return CPAA_ECUDA;
}

void clear_error() { t_last_error.clear(); }

cpaa_status dev_alloc(cpaa_graph *g, void **p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) return CPAA_OK;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        (void)cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? CPAA_ENOMEM : CPAA_ECUDA,
                    std::string("cudaMalloc(") + std::to_string(bytes) +
                        " bytes): " + cudaGetErrorString(e));
    }
    if (g) g->device_bytes += (int64_t)bytes;
    return CPAA_OK;
}

void dev_free(cpaa_graph *g, void **p, size_t bytes) {
    if (*p) {
        cudaFree(*p);
        if (g) g->device_bytes -= (int64_t)bytes;
    }
    *p = nullptr;
}

// c_0 = 2 / sqrt(1 - c^2) and c_{k-1}/c_k = c / (1 - sqrt(1 - c^2)) for all
// k (proof of Proposition 1), i.e. c_k = c_0 beta^k with beta the Eq. 41 base.
void cheb_coeffs(double c, int M, std::vector<double> &ck) {
    const double s = std::sqrt(1.0 - c * c);
    const double beta = (1.0 - s) / c;
    ck.resize((size_t)M + 1);
    ck[0] = 2.0 / s;
    for (int k = 1; k <= M; ++k) ck[k] = ck[k - 1] * beta;
}

double err_bound(double c, int M) {
    const double beta = (1.0 - std::sqrt(1.0 - c * c)) / c;
    return 2.0 * std::pow(beta, (double)(M + 1)) / (1.0 + beta);
}

// The series on [lo, 1] (Sec. 2.2's general interval): x = mid + half cos t
// turns 1 / (1 - c x) into (1 / (1 - c mid)) / (1 - chat cos t) with
// chat = c half / (1 - c mid), so its coefficients are the [-1, 1] ones of
// chat times 1 / (1 - c mid).  lo = -1 is the paper's series exactly.
IntervalMap interval_map(double c, double lo) {
    IntervalMap m;
    m.mid = 0.5 * (1.0 + lo);
    m.half = 0.5 * (1.0 - lo);
    m.chat = c * m.half / (1.0 - c * m.mid);
    m.scale = 1.0 / (1.0 - c * m.mid);
    return m;
}

void cheb_coeffs_on(double c, double lo, int M, std::vector<double> &ck) {
    if (lo == -1.0) return cheb_coeffs(c, M, ck);
    const IntervalMap m = interval_map(c, lo);
    cheb_coeffs(m.chat, M, ck);
    for (double &v : ck) v *= m.scale;
}

// (1 - c) sum_{k>M} c_k with c_k = c_0 betahat^k: (1 - c) c_0 betahat^(M+1) / (1 - betahat).
double err_bound_on(double c, double lo, int M) {
    if (lo == -1.0) return err_bound(c, M);
    const IntervalMap m = interval_map(c, lo);
    const double s = std::sqrt(1.0 - m.chat * m.chat);
    const double bh = (1.0 - s) / m.chat;
    return (1.0 - c) * (2.0 / s) * m.scale * std::pow(bh, (double)(M + 1)) / (1.0 - bh);
}

}  // namespace cpaa

extern "C" {

const char *cpaa_status_string(cpaa_status s) {
    switch (s) {
        case CPAA_OK: return "CPAA_OK";
        case CPAA_EINVAL: return "CPAA_EINVAL";
        case CPAA_ENOMEM: return "CPAA_ENOMEM";
        case CPAA_ENOTCONV: return "CPAA_ENOTCONV";
        case CPAA_ECUDA: return "CPAA_ECUDA";
        case CPAA_ETIMEOUT: return "CPAA_ETIMEOUT";
        case CPAA_EBUSY: return "CPAA_EBUSY";
        case CPAA_ECANCELLED: return "CPAA_ECANCELLED";
        case CPAA_ENOTFOUND: return "CPAA_ENOTFOUND";
    }
    return "CPAA_UNKNOWN";
}

const char *cpaa_last_error(void) { return cpaa::t_last_error.c_str(); }

void cpaa_options_init(cpaa_options *opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->precision = CPAA_F64;
    opt->normalize = 0;
    opt->fixed_rounds = 0;
    opt->max_rounds = cpaa::kDefaultMaxRounds;
    opt->lambda_lo = -1.0;
}

// Tail of the series after M rounds.  With (1 - c) scaling the error is
// (1 - c) sum_{k>M} c_k T_k(P) p; the coefficients are positive and
// (1 - c) sum_{k>M} c_k = ERR_M = 2 beta^(M+1) / (1 + beta) (Eq. 41), and
// ||T_k(P) p||_1 <= kappa, so the L1 error is at most ERR_M kappa.  Dividing
// by the sum instead (Algorithm 1) rescales by 1 / (1 - ERR_M), since every
// T_k(P) keeps e^T p = 1; that adds at most (1 + E kappa) E / (1 - E).
double cpaa_l1_bound(double c, int M, double kappa, int normalize) {
    const double E = cpaa::err_bound(c, M);
    if (normalize == 1) return E * kappa;
    return E * kappa + (1.0 + E * kappa) * E / (1.0 - E);
}

int cpaa_rounds_needed(double c, double tol, double kappa, int normalize, int max_rounds) {
    if (!(c > 0.0 && c < 1.0) || !(tol > 0.0) || max_rounds < 1) return -1;
    for (int M = 1; M <= max_rounds; ++M)
        if (cpaa_l1_bound(c, M, kappa, normalize) < tol) return M;
    return -1;
}

double cpaa_l1_bound_interval(double c, double lambda_lo, int M, double kappa, int normalize) {
    if (!(c > 0.0 && c < 1.0) || !(lambda_lo >= -1.0 && lambda_lo < 1.0) || M < 0) return NAN;
    const double E = cpaa::err_bound_on(c, lambda_lo, M);
    if (normalize == 1) return E * kappa;
    return E * kappa + (1.0 + E * kappa) * E / (1.0 - E);
}

int cpaa_rounds_needed_interval(double c, double lambda_lo, double tol, double kappa, int normalize,
                                int max_rounds) {
    if (!(c > 0.0 && c < 1.0) || !(lambda_lo >= -1.0 && lambda_lo < 1.0) || !(tol > 0.0) || max_rounds < 1)
        return -1;
    for (int M = 1; M <= max_rounds; ++M)
        if (cpaa_l1_bound_interval(c, lambda_lo, M, kappa, normalize) < tol) return M;
    return -1;
}

}  // extern "C"
