// batch.cu -- cpaa_solve_batch: B personalised vectors as tiles of W columns.
//
// The graph is read once per round for a whole tile (an SpMM: every gathered
// neighbour row brings W values), instead of once per vector.  Columns are
// sorted by the rounds their own bound asks for, so that a tile's columns
// stop close together; a column stops accumulating after its own M while the
// rest of its tile runs on.  A wider tile brings more values per gathered
// sector (the round is bound by random-gather requests), while its gathered
// array, (n + 1) W values, competes for L2; so the default width is chosen by
// measurement: the first batch of at least 16 columns on a graph times a few
// rounds at each candidate width on its own columns and keeps the fastest per
// column (cached in the graph, per precision).
//
// Each column's result is bit-identical to cpaa_solve on that column: the
// same fixed-order statistics decide its M, and the round, prep and
// finalisation kernels are the same code with the same arithmetic per column.
#include <algorithm>
#include <numeric>

#include "internal.h"

namespace cpaa {

constexpr int kTuneRounds = 3;

// Time kTuneRounds rounds for each candidate width on the batch's first
// columns; return the width with the least time per column.
static cpaa_status autotune_width(cpaa_graph *g, int prec, int B, const double *const *cols,
                                  const double *c, double *scratch_pi, cudaStream_t st, int *out) {
    float best = 0.0f;
    int best_w = 1;
    for (int W = 1; W <= kMaxWidth && W <= B; W *= 2) {
        cpaa_status s = ensure_workspace(g, prec, W, kTuneRounds);
        if (s != CPAA_OK) break;  // a width that does not fit is not a candidate
        TileJob job;
        job.width = W;
        job.precision = prec;
        job.normalize = 0;
        for (int b = 0; b < W; ++b) {
            std::vector<double> ck0;
            cheb_coeffs(c[b], 0, ck0);
            job.p[b] = cols[b];
            job.pi[b] = scratch_pi;  // results of the trial are discarded
            job.c[b] = c[b];
            job.c0half[b] = ck0[0] / 2.0;
            job.rounds[b] = kTuneRounds;
        }
        float ms = 0.0f;
        if ((s = run_tile(g, job, st, false, true)) != CPAA_OK) return s;
        if ((s = tile_rounds_ms(g, &ms)) != CPAA_OK) return s;
        const float per_col = ms / W;
        if (W == 1 || per_col < best) {
            best = per_col;
            best_w = W;
        }
    }
    *out = best_w;
    return CPAA_OK;
}

}  // namespace cpaa

using namespace cpaa;

extern "C" cpaa_status cpaa_solve_batch(cpaa_graph *g, int B, const double *P, const double *c,
                                        double tol, double *PI, const cpaa_options *opt_in,
                                        cpaa_info *info) {
    clear_error();
    cpaa_options opt;
    if (opt_in) opt = *opt_in; else cpaa_options_init(&opt);
    if (!g) return fail(CPAA_EINVAL, "graph is NULL");
    if (B < 1) return fail(CPAA_EINVAL, "B must be >= 1");
    if (!P || !PI || !c) return fail(CPAA_EINVAL, "P / PI / c is NULL");
    for (int b = 0; b < B; ++b)
        if (!(c[b] > 0.0 && c[b] < 1.0)) return fail(CPAA_EINVAL, "damping c[" + std::to_string(b) + "] must lie in (0, 1)");
    if (opt.fixed_rounds < 0) return fail(CPAA_EINVAL, "fixed_rounds < 0");
    if (opt.fixed_rounds == 0 && !(tol > 0.0)) return fail(CPAA_EINVAL, "tol must be > 0");
    if (opt.precision != CPAA_F64 && opt.precision != CPAA_F32 && opt.precision != CPAA_BF16 &&
        opt.precision != CPAA_DF64)
        return fail(CPAA_EINVAL, "unknown precision");
    if (opt.normalize != 0 && opt.normalize != 1) return fail(CPAA_EINVAL, "normalize must be 0 or 1");
    if (opt.stop_rule != CPAA_STOP_RIGOROUS && opt.stop_rule != CPAA_STOP_POSTERIORI)
        return fail(CPAA_EINVAL, "unknown stop_rule");
    const int max_rounds = opt.max_rounds > 0 ? opt.max_rounds : kDefaultMaxRounds;
    if (opt.fixed_rounds > max_rounds) return fail(CPAA_EINVAL, "fixed_rounds > max_rounds");
    int W = opt.batch_width;
    if (W != 0 && W != 1 && W != 2 && W != 4 && W != 8 && W != 16)
        return fail(CPAA_EINVAL, "batch_width must be 0 (automatic), 1, 2, 4, 8 or 16");
    const bool host_io = (opt.flags & CPAA_DEVICE_IO) == 0;
    cudaStream_t st = (cudaStream_t)opt.stream;
    const int64_t n = g->n;

    cpaa_status s;
    Workspace &w = g->ws;
    if ((s = ensure_reduction_buffers(g)) != CPAA_OK) return s;
    // device staging: host P and PI, plus 3 statistics per column
    const size_t need = sizeof(double) * ((host_io ? 2 * (size_t)n * B : 0) + 3 * (size_t)B);
    if (w.io_bytes < need) {
        dev_free(g, (void **)&w.io, w.io_bytes);
        w.io_bytes = 0;
        if ((s = dev_alloc(g, (void **)&w.io, need)) != CPAA_OK) return s;
        w.io_bytes = need;
    }
    const double *dP = P;
    double *dPI = PI;
    double *dstats = w.io;
    if (host_io) {
        dstats = w.io + 2 * (size_t)n * B;
        CPAA_CUDA(cudaMemcpyAsync(w.io, P, sizeof(double) * n * B, cudaMemcpyHostToDevice, st));
        dP = w.io;
        dPI = w.io + (size_t)n * B;
    }
    for (int b = 0; b < B; ++b) CPAA_CUDA(launch_stats(g, dP + (size_t)b * n, dstats + 3 * b, st));
    std::vector<double> hs(3 * (size_t)B);
    CPAA_CUDA(cudaMemcpyAsync(hs.data(), dstats, sizeof(double) * hs.size(), cudaMemcpyDeviceToHost, st));
    CPAA_CUDA(cudaStreamSynchronize(st));
    double lo = -1.0;
    if ((s = resolve_interval(g, opt, &lo)) != CPAA_OK) return s;
    std::vector<double> kappa(B);
    std::vector<int> M(B);
    std::vector<char> notconv(B, 0);
    for (int b = 0; b < B; ++b) {
        if ((s = check_stats(&hs[3 * b], g->nnz, &kappa[b])) != CPAA_OK)
            return fail(s, "column " + std::to_string(b) + ": " + cpaa_last_error());
        M[b] = opt.fixed_rounds;
        if (M[b] == 0) {
            M[b] = cpaa_rounds_needed_interval(c[b], lo, tol, kappa[b], opt.normalize, max_rounds);
            if (M[b] < 0) {
                M[b] = max_rounds;
                notconv[b] = 1;
            }
        }
    }
    std::vector<int> order(B);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b2) { return M[a] > M[b2]; });

    if (W == 0) {
        W = g->tuned_width[opt.precision];
        if (W == 0 || W > B) {
            const double *cols[kMaxWidth];
            double cc[kMaxWidth];
            for (int j = 0; j < kMaxWidth && j < B; ++j) {
                cols[j] = dP + (size_t)order[j] * n;
                cc[j] = c[order[j]];
            }
            if ((s = autotune_width(g, opt.precision, B, cols, cc, dPI + (size_t)order[0] * n, st, &W)) != CPAA_OK)
                return s;
            if (B >= kMaxWidth) g->tuned_width[opt.precision] = W;
        }
    }
    if ((s = ensure_workspace(g, opt.precision, W, max_rounds)) != CPAA_OK) return s;

    for (int t0 = 0; t0 < B;) {
        int tw = W;
        while (tw > 1 && tw / 2 >= B - t0) tw /= 2;  // narrower tile for the tail
        tw = std::min(tw, B - t0);
        while (tw & (tw - 1)) --tw;                  // a power of two
        TileJob job;
        job.width = tw;
        job.precision = opt.precision;
        job.normalize = opt.normalize;
        job.posteriori = opt.stop_rule == CPAA_STOP_POSTERIORI && opt.fixed_rounds == 0;
        job.frontier = (opt.flags & CPAA_SPARSE_FRONTIER) != 0;
        job.lambda_lo = lo;
        job.tol = tol;
        for (int j = 0; j < tw; ++j) {
            const int b = order[t0 + j];
            std::vector<double> ck0;
            cheb_coeffs_on(c[b], lo, 0, ck0);
            job.p[j] = dP + (size_t)b * n;
            job.pi[j] = dPI + (size_t)b * n;
            job.c[j] = c[b];
            job.c0half[j] = ck0[0] / 2.0;
            job.rounds[j] = M[b];
            job.p_l1[j] = hs[3 * b];
        }
        if ((s = run_tile(g, job, st, false, false)) != CPAA_OK) return s;
        int sr[kMaxWidth];
        bool by_post[kMaxWidth] = {};
        if (job.posteriori) {
            CPAA_CUDA(cudaMemcpyAsync(sr, w.stop_round, sizeof(int) * kMaxWidth, cudaMemcpyDeviceToHost, st));
            CPAA_CUDA(cudaStreamSynchronize(st));
            for (int j = 0; j < tw; ++j) {
                const int b = order[t0 + j];
                if (sr[j] >= 1 && sr[j] <= M[b]) {
                    M[b] = sr[j];
                    by_post[j] = true;
                    notconv[b] = 0;
                }
            }
        }
        if (info) {
            int maxM = 0;
            for (int j = 0; j < tw; ++j) maxM = std::max(maxM, job.rounds[j]);
            std::vector<double> h((size_t)(maxM + 1) * 2 * tw);
            CPAA_CUDA(cudaMemcpyAsync(h.data(), w.red, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, st));
            CPAA_CUDA(cudaMemcpyAsync(w.h_sums, w.sums, sizeof(double) * tw, cudaMemcpyDeviceToHost, st));
            CPAA_CUDA(cudaStreamSynchronize(st));
            for (int j = 0; j < tw; ++j) {
                const int b = order[t0 + j];
                cpaa_info &in = info[b];
                in.rounds = M[b];
                in.kappa = kappa[b];
                if (by_post[j]) {
                    double ml = hs[3 * b], t = 0, a = 0;
                    for (int k = 1; k <= M[b]; ++k) {
                        round_sums(tw, j, k, h, &t, &a);
                        ml = std::max(ml, a);
                    }
                    in.bound = cpaa_l1_bound_interval(c[b], lo, M[b], 2.0 * ml, opt.normalize);
                } else {
                    in.bound = cpaa_l1_bound_interval(c[b], lo, M[b], kappa[b], opt.normalize);
                }
                in.lambda_lo = lo;
                round_sums(tw, j, M[b], h, &in.mass, &in.l1);
                in.sum_pibar = w.h_sums[j];
                in.rounds_ms = 0.0;
            }
        }
        t0 += tw;
    }
    if (host_io) {
        CPAA_CUDA(cudaMemcpyAsync(PI, dPI, sizeof(double) * n * B, cudaMemcpyDeviceToHost, st));
        CPAA_CUDA(cudaStreamSynchronize(st));
    }
    for (int b = 0; b < B; ++b)
        if (notconv[b]) return fail(CPAA_ENOTCONV, "the L1 bound of some column needs more than max_rounds rounds");
    return CPAA_OK;
}
