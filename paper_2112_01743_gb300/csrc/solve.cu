// solve.cu -- cpaa_solve: one personalised PageRank vector (Algorithm 1).
//
//   prep:      y_0 = D^-1 p, rho = (c_0/2) y_0 (Algorithm 1's initial
//              accumulator, in scaled space), and in fixed order the sums
//              sum p, sum p^2/d (for kappa) and a count of invalid entries;
//   host:      kappa = sqrt(nnz) sqrt(sum p^2/d), M from the L1 bound;
//   rounds:    M launches of the step kernel (step.cu);
//   finalize:  pi = d * rho / sum(d * rho) (Algorithm 1's last line) or
//              (1 - c) d * rho (Sec. 2.1).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "internal.h"

namespace cpaa {

constexpr int kPrepBlocks = 1024;

template <class S> struct VecOf;
template <> struct VecOf<double> { using A = double; };
template <> struct VecOf<float> { using A = float; };
template <> struct VecOf<__nv_bfloat16> { using A = float; };

__device__ __forceinline__ void put(double *p, double v) { *p = v; }
__device__ __forceinline__ void put(float *p, double v) { *p = (float)v; }
__device__ __forceinline__ void put(__nv_bfloat16 *p, double v) { *p = __double2bfloat16(v); }
__device__ __forceinline__ double get(const double *p) { return *p; }
__device__ __forceinline__ double get(const float *p) { return (double)*p; }
__device__ __forceinline__ double get(const __nv_bfloat16 *p) { return (double)__bfloat162float(*p); }

// Fixed-shape CTA sum of nq values per thread into out[0..nq).
template <int NQ>
__device__ __forceinline__ void cta_sum(double (&v)[NQ], double *out) {
    __shared__ double s[NQ][kThreads];
    for (int q = 0; q < NQ; ++q) s[q][threadIdx.x] = v[q];
    __syncthreads();
    for (int o = kThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int q = 0; q < NQ; ++q) s[q][threadIdx.x] += s[q][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int q = 0; q < NQ; ++q) out[q] = s[q][0];
}

// part[b][0..5] = sum p, sum p^2/d, #invalid, sum T_0, sum |T_0|, sum d rho_0
template <class S, class R>
__global__ void __launch_bounds__(kThreads) prep_kernel(const double *__restrict__ p, int64_t n,
                                                        const double *__restrict__ deg64,
                                                        const double *__restrict__ inv64,
                                                        double c0half, S *y0, R *rho, R *comp,
                                                        double *part) {
    double v[6] = {0, 0, 0, 0, 0, 0};
    for (int64_t u = blockIdx.x * (int64_t)kThreads + threadIdx.x; u < n;
         u += (int64_t)gridDim.x * kThreads) {
        const double pu = p[u];
        const double d = deg64[u];
        if (!(pu >= 0.0) || !(pu < INFINITY)) v[2] += 1.0;  // negative, NaN or inf
        v[0] += pu;
        v[1] += pu * pu * inv64[u];
        put(y0 + u, pu * inv64[u]);
        const double yq = get(y0 + u);
        put(rho + u, c0half * yq);
        if (comp) put(comp + u, 0.0);
        const double r = get(rho + u);
        v[3] += yq * d;
        v[4] += fabs(yq * d);
        v[5] += r * d;
    }
    cta_sum<6>(v, part + 6 * blockIdx.x);
}

// One CTA: out[q] = sum over blocks of part[b][q], fixed order.
__global__ void __launch_bounds__(kThreads) prep_reduce_kernel(const double *part, int nblocks,
                                                               double *out, double *red0) {
    double v[6] = {0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblocks; b += kThreads)
        for (int q = 0; q < 6; ++q) v[q] += part[6 * b + q];
    double r[6];
    cta_sum<6>(v, r);
    if (threadIdx.x == 0) {
        out[0] = r[0];
        out[1] = r[1];
        out[2] = r[2];
        // round 0 of the per-round reductions lives in slot 0 of red0
        red0[0 * kRedSlots] = r[3];
        red0[1 * kRedSlots] = r[4];
        red0[2 * kRedSlots] = r[5];
    }
}

// Normaliser of Algorithm 1's last line, sum_u pibar[u] = sum_u d_u rho[u],
// in a fixed order: per-CTA partials over a fixed grid, then one CTA.  The
// order depends only on n, so a vector's result never depends on what else
// ran before or beside it.
template <class R>
__global__ void __launch_bounds__(kThreads) norm_partial_kernel(const R *__restrict__ rho,
                                                                const double *__restrict__ deg64,
                                                                int64_t n, double *part) {
    double v[1] = {0.0};
    for (int64_t u = blockIdx.x * (int64_t)kThreads + threadIdx.x; u < n;
         u += (int64_t)gridDim.x * kThreads)
        v[0] += deg64[u] * get(rho + u);
    cta_sum<1>(v, part + blockIdx.x);
}

__global__ void __launch_bounds__(kThreads) norm_reduce_kernel(const double *part, int nblocks,
                                                               double *out) {
    double v[1] = {0.0};
    for (int b = threadIdx.x; b < nblocks; b += kThreads) v[0] += part[b];
    cta_sum<1>(v, out);
}

// pi[u] = scale * d_u * rho[u]; scale = 1 / sum(d rho) or (1 - c).
template <class R>
__global__ void __launch_bounds__(kThreads) finalize_kernel(const R *__restrict__ rho,
                                                            const double *__restrict__ deg64,
                                                            int64_t n, const double *sum_pibar,
                                                            int normalize, double one_minus_c,
                                                            double *pi) {
    const double scale = normalize == 0 ? 1.0 / *sum_pibar : one_minus_c;
    for (int64_t u = blockIdx.x * (int64_t)kThreads + threadIdx.x; u < n;
         u += (int64_t)gridDim.x * kThreads)
        pi[u] = scale * (deg64[u] * get(rho + u));
}

static size_t store_bytes(int prec) { return prec == CPAA_F64 ? 8 : prec == CPAA_F32 ? 4 : 2; }
static size_t rho_bytes(int prec) { return prec == CPAA_F64 ? 8 : 4; }

static cpaa_status ensure_workspace(cpaa_graph *g, int prec, int max_rounds, bool host_io) {
    Workspace &w = g->ws;
    const int64_t n = g->n;
    cpaa_status st;
    if (w.precision != prec) {
        dev_free(g, &w.y0, w.vec_bytes);
        dev_free(g, &w.y1, w.vec_bytes);
        dev_free(g, &w.rho, n * 8);
        dev_free(g, &w.comp, n * 4);
        w.precision = -1;
        w.vec_bytes = store_bytes(prec) * n;
        if ((st = dev_alloc(g, &w.y0, w.vec_bytes)) != CPAA_OK) return st;
        if ((st = dev_alloc(g, &w.y1, w.vec_bytes)) != CPAA_OK) return st;
        // rho is sized for FP64 so a later precision switch can reuse it
        if ((st = dev_alloc(g, &w.rho, n * 8)) != CPAA_OK) return st;
        if ((st = dev_alloc(g, &w.comp, n * 4)) != CPAA_OK) return st;
        w.precision = prec;
    }
    if (w.red_rounds < max_rounds + 1) {
        dev_free(g, (void **)&w.red, sizeof(double) * kRedQ * kRedSlots * w.red_rounds);
        w.red_rounds = 0;
        if ((st = dev_alloc(g, (void **)&w.red, sizeof(double) * kRedQ * kRedSlots * (max_rounds + 1))) != CPAA_OK)
            return st;
        w.red_rounds = max_rounds + 1;
    }
    if (!w.prep_part) {
        if ((st = dev_alloc(g, (void **)&w.prep_part, sizeof(double) * 6 * kPrepBlocks)) != CPAA_OK) return st;
        if ((st = dev_alloc(g, (void **)&w.prep_out, sizeof(double) * 4)) != CPAA_OK) return st;
        CPAA_CUDA(cudaMallocHost((void **)&w.h_prep, sizeof(double) * 4));
    }
    if (host_io && !w.d_pi) {
        if ((st = dev_alloc(g, (void **)&w.d_pi, sizeof(double) * n)) != CPAA_OK) return st;
        if ((st = dev_alloc(g, (void **)&w.d_p, sizeof(double) * n)) != CPAA_OK) return st;
    }
    (void)rho_bytes;
    return CPAA_OK;
}

template <class S, class R>
static void launch_prep(cpaa_graph *g, const double *p, double c0half, cudaStream_t st, int blocks) {
    Workspace &w = g->ws;
    prep_kernel<S, R><<<blocks, kThreads, 0, st>>>(p, g->n, g->deg64, g->inv_deg64, c0half,
                                                   (S *)w.y0, (R *)w.rho,
                                                   std::is_same<R, float>::value ? (R *)w.comp : nullptr,
                                                   w.prep_part);
}

}  // namespace cpaa

using namespace cpaa;

extern "C" cpaa_status cpaa_solve(cpaa_graph *g, const double *p, double c, double tol, double *pi,
                                  const cpaa_options *opt_in, cpaa_info *info) {
    clear_error();
    cpaa_options opt;
    if (opt_in) opt = *opt_in; else cpaa_options_init(&opt);
    if (!g) return fail(CPAA_EINVAL, "graph is NULL");
    if (!p || !pi) return fail(CPAA_EINVAL, "p / pi is NULL");
    if (!(c > 0.0 && c < 1.0)) return fail(CPAA_EINVAL, "damping c must lie in (0, 1)");
    if (opt.fixed_rounds < 0) return fail(CPAA_EINVAL, "fixed_rounds < 0");
    if (opt.fixed_rounds == 0 && !(tol > 0.0)) return fail(CPAA_EINVAL, "tol must be > 0");
    if (opt.precision != CPAA_F64 && opt.precision != CPAA_F32 && opt.precision != CPAA_BF16)
        return fail(CPAA_EINVAL, "unknown precision");
    if (opt.normalize != 0 && opt.normalize != 1) return fail(CPAA_EINVAL, "normalize must be 0 or 1");
    const int max_rounds = opt.max_rounds > 0 ? opt.max_rounds : kDefaultMaxRounds;
    if (opt.fixed_rounds > max_rounds) return fail(CPAA_EINVAL, "fixed_rounds > max_rounds");
    const bool host_io = (opt.flags & CPAA_DEVICE_IO) == 0;
    cudaStream_t st = (cudaStream_t)opt.stream;
    const int64_t n = g->n;
    const int prec = opt.precision;

    cpaa_status s = ensure_workspace(g, prec, max_rounds, host_io);
    if (s != CPAA_OK) return s;
    Workspace &w = g->ws;
    const double *dp = p;
    double *dpi = pi;
    if (host_io) {
        CPAA_CUDA(cudaMemcpyAsync(w.d_p, p, sizeof(double) * n, cudaMemcpyHostToDevice, st));
        dp = w.d_p;
        dpi = w.d_pi;
    }

    std::vector<double> ck;
    cheb_coeffs(c, 0, ck);
    const double c0half = ck[0] / 2.0;
    const int blocks = (int)std::min<int64_t>((n + kThreads - 1) / kThreads, kPrepBlocks);
    CPAA_CUDA(cudaMemsetAsync(w.red, 0, sizeof(double) * kRedQ * kRedSlots * (max_rounds + 1), st));
    CPAA_CUDA(cudaMemsetAsync(g->long_cnt, 0, sizeof(int) * std::max(1, g->num_long), st));
    if (prec == CPAA_F64) launch_prep<double, double>(g, dp, c0half, st, blocks);
    else if (prec == CPAA_F32) launch_prep<float, float>(g, dp, c0half, st, blocks);
    else launch_prep<__nv_bfloat16, float>(g, dp, c0half, st, blocks);
    CPAA_CUDA(cudaGetLastError());
    prep_reduce_kernel<<<1, kThreads, 0, st>>>(w.prep_part, blocks, w.prep_out, w.red);
    CPAA_CUDA(cudaGetLastError());
    CPAA_CUDA(cudaMemcpyAsync(w.h_prep, w.prep_out, sizeof(double) * 3, cudaMemcpyDeviceToHost, st));
    CPAA_CUDA(cudaStreamSynchronize(st));
    const double sum_p = w.h_prep[0], q = w.h_prep[1], nbad = w.h_prep[2];
    if (nbad > 0.0) return fail(CPAA_EINVAL, "p has negative, NaN or infinite entries");
    if (!(std::fabs(sum_p - 1.0) <= 1e-9)) return fail(CPAA_EINVAL, "p must sum to 1 (|sum p - 1| <= 1e-9)");
    const double kappa = std::sqrt((double)g->nnz) * std::sqrt(q);

    cpaa_status result = CPAA_OK;
    int M = opt.fixed_rounds;
    if (M == 0) {
        M = cpaa_rounds_needed(c, tol, kappa, opt.normalize, max_rounds);
        if (M < 0) {
            M = max_rounds;
            result = CPAA_ENOTCONV;
        }
    }
    cheb_coeffs(c, M, ck);

    const bool timed = (opt.flags & CPAA_TIME_ROUNDS) != 0;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    if (timed) {
        CPAA_CUDA(cudaEventCreate(&ev[0]));
        CPAA_CUDA(cudaEventCreate(&ev[1]));
        CPAA_CUDA(cudaEventRecord(ev[0], st));
    }
    void *buf[2] = {w.y0, w.y1};
    for (int k = 1; k <= M; ++k) {
        StepLaunch sl;
        sl.g = g;
        sl.precision = prec;
        sl.y_src = buf[(k - 1) & 1];
        sl.y_io = buf[k & 1];
        sl.rho = w.rho;
        sl.comp = w.comp;
        sl.red = w.red + (size_t)k * kRedQ * kRedSlots;
        sl.ck = ck[k];
        sl.first = (k == 1);
        sl.last = (k == M);
        sl.stream = st;
        CPAA_CUDA(launch_step(sl));
    }
    if (timed) CPAA_CUDA(cudaEventRecord(ev[1], st));
    const unsigned fblocks = (unsigned)std::min<int64_t>((n + kThreads - 1) / kThreads, 4096);
    double *sum_pibar = w.prep_out + 3;
    if (prec == CPAA_F64) {
        norm_partial_kernel<double><<<blocks, kThreads, 0, st>>>((const double *)w.rho, g->deg64, n, w.prep_part);
        norm_reduce_kernel<<<1, kThreads, 0, st>>>(w.prep_part, blocks, sum_pibar);
        finalize_kernel<double><<<fblocks, kThreads, 0, st>>>((const double *)w.rho, g->deg64, n, sum_pibar,
                                                              opt.normalize, 1.0 - c, dpi);
    } else {
        norm_partial_kernel<float><<<blocks, kThreads, 0, st>>>((const float *)w.rho, g->deg64, n, w.prep_part);
        norm_reduce_kernel<<<1, kThreads, 0, st>>>(w.prep_part, blocks, sum_pibar);
        finalize_kernel<float><<<fblocks, kThreads, 0, st>>>((const float *)w.rho, g->deg64, n, sum_pibar,
                                                             opt.normalize, 1.0 - c, dpi);
    }
    CPAA_CUDA(cudaGetLastError());
    if (host_io) CPAA_CUDA(cudaMemcpyAsync(pi, dpi, sizeof(double) * n, cudaMemcpyDeviceToHost, st));

    float rounds_ms = 0.0f;
    if (timed) {
        CPAA_CUDA(cudaEventSynchronize(ev[1]));
        CPAA_CUDA(cudaEventElapsedTime(&rounds_ms, ev[0], ev[1]));
        cudaEventDestroy(ev[0]);
        cudaEventDestroy(ev[1]);
    }
    if (info || opt.history) {
        std::vector<double> h((size_t)(M + 1) * kRedQ * kRedSlots);
        CPAA_CUDA(cudaMemcpyAsync(h.data(), w.red, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, st));
        CPAA_CUDA(cudaMemcpyAsync(w.h_prep + 3, sum_pibar, sizeof(double), cudaMemcpyDeviceToHost, st));
        CPAA_CUDA(cudaStreamSynchronize(st));
        auto sum = [&](int k, int qq) {
            double a = 0;
            for (int i = 0; i < kRedSlots; ++i) a += h[((size_t)k * kRedQ + qq) * kRedSlots + i];
            return a;
        };
        if (opt.history)
            for (int k = 0; k <= M; ++k) {
                opt.history[2 * k] = sum(k, 0);
                opt.history[2 * k + 1] = sum(k, 1);
            }
        if (info) {
            info->rounds = M;
            info->kappa = kappa;
            info->bound = cpaa_l1_bound(c, M, kappa, opt.normalize);
            info->mass = sum(M, 0);
            info->l1 = sum(M, 1);
            info->sum_pibar = w.h_prep[3];
            info->rounds_ms = rounds_ms;
        }
    } else if (host_io) {
        CPAA_CUDA(cudaStreamSynchronize(st));
    }
    if (result == CPAA_ENOTCONV) fail(result, "the L1 bound needs more than max_rounds rounds");
    return result;
}
