// batch.cu -- cpaa_solve_batch.
//
// First form: the columns run one after another through the single-vector
// path, each with its own damping and its own number of rounds.
#include "internal.h"

extern "C" cpaa_status cpaa_solve_batch(cpaa_graph *g, int B, const double *P, const double *c,
                                        double tol, double *PI, const cpaa_options *opt,
                                        cpaa_info *info) {
    cpaa::clear_error();
    if (!g) return cpaa::fail(CPAA_EINVAL, "graph is NULL");
    if (B < 1) return cpaa::fail(CPAA_EINVAL, "B must be >= 1");
    if (!P || !PI || !c) return cpaa::fail(CPAA_EINVAL, "P / PI / c is NULL");
    cpaa_status worst = CPAA_OK;
    for (int b = 0; b < B; ++b) {
        cpaa_status s = cpaa_solve(g, P + (size_t)b * g->n, c[b], tol, PI + (size_t)b * g->n, opt,
                                   info ? info + b : nullptr);
        if (s == CPAA_ENOTCONV) worst = s;
        else if (s != CPAA_OK) return s;
    }
    return worst;
}
