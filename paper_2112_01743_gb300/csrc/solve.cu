// solve.cu -- the solve driver (Algorithm 1) for a tile of W vectors, and
// cpaa_solve (W = 1).  batch.cu drives tiles of W > 1 through run_tile.
//
//   stats:     per vector, in a fixed order: sum p, sum p^2/d (for kappa) and a
//              count of invalid entries;
//   host:      kappa = sqrt(nnz) sqrt(sum p^2/d); M from the L1 bound;
//   prep:      y_0 = D^-1 p, rho = (c_0/2) y_0 (Algorithm 1's initial
//              accumulator, in scaled space), comp = 0;
//   rounds:    max M launches of the round kernel (step.cu), captured once
//              as a CUDA graph per key and replayed; a vector stops
//              accumulating after its own M, or earlier under the
//              a-posteriori rule (decided on the device after each round);
//   finalize:  pi = d * rho / sum(d * rho) (Algorithm 1's last line) or
//              (1 - c) d * rho (Sec. 2.1), the sum in a fixed order.
// Every sum a vector's result depends on runs in an order fixed by the graph
// alone, and every rounding is an explicit intrinsic, so a vector gives the
// same bits alone (cpaa_solve) and in any batch.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "internal.h"

namespace cpaa {

__device__ __forceinline__ void put(double *p, double v) { *p = v; }
__device__ __forceinline__ void put(float *p, double v) { *p = __double2float_rn(v); }
__device__ __forceinline__ void put(__nv_bfloat16 *p, double v) { *p = __double2bfloat16(v); }
__device__ __forceinline__ double get(const double *p) { return *p; }
__device__ __forceinline__ double get(const float *p) { return (double)*p; }
__device__ __forceinline__ double get(const __nv_bfloat16 *p) { return (double)__bfloat162float(*p); }
__device__ __forceinline__ void put(df *p, double v) { *p = df(v); }
__device__ __forceinline__ double get(const df *p) { return __dadd_rn((double)p->hi, (double)p->lo); }

// Fixed-shape CTA sum of NQ values per thread into out[0..NQ).
template <int NQ>
__device__ __forceinline__ void cta_sum(double (&v)[NQ], double *out) {
    __shared__ double s[NQ][kThreads];
    for (int q = 0; q < NQ; ++q) s[q][threadIdx.x] = v[q];
    __syncthreads();
    for (int o = kThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int q = 0; q < NQ; ++q) s[q][threadIdx.x] = __dadd_rn(s[q][threadIdx.x], s[q][threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int q = 0; q < NQ; ++q) out[q] = s[q][0];
    __syncthreads();
}

// Per-block partial sums of one vector p (caller's order, read through perm):
// part[block][0..2] = sum p, sum p^2/d, #invalid (negative, NaN or inf).
__global__ void __launch_bounds__(kThreads) stats_kernel(const double *__restrict__ p,
                                                         const int32_t *__restrict__ perm, int64_t n,
                                                         const double *__restrict__ inv64,
                                                         double *part) {
    double v[3] = {0, 0, 0};
    for (int64_t u = blockIdx.x * (int64_t)kThreads + threadIdx.x; u < n;
         u += (int64_t)gridDim.x * kThreads) {
        const double pu = p[perm[u]];
        if (!(pu >= 0.0) || !(pu < INFINITY)) v[2] = __dadd_rn(v[2], 1.0);
        v[0] = __dadd_rn(v[0], pu);
        v[1] = __fma_rn(__dmul_rn(pu, pu), inv64[u], v[1]);
    }
    cta_sum<3>(v, part + 3 * blockIdx.x);
}

// One CTA: out[q] = sum over blocks of part[b][q], fixed order.
template <int NQ>
__global__ void __launch_bounds__(kThreads) block_sum_kernel(const double *part, int nblocks,
                                                             double *out) {
    double v[NQ];
    for (int q = 0; q < NQ; ++q) v[q] = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += kThreads)
        for (int q = 0; q < NQ; ++q) v[q] = __dadd_rn(v[q], part[NQ * b + q]);
    cta_sum<NQ>(v, out);
}

struct TileCols {
    const double *p[kMaxWidth];  // column b of the caller's input (device)
    double *pi[kMaxWidth];       // column b of the output (device)
    double c0half[kMaxWidth];
    double scale[kMaxWidth];     // (1 - c) for normalize = 1
};

// y_0 = D^-1 p, rho = (c_0/2) y_0, comp = 0 for the W columns of a tile.
// Buffers a tile's rounds expect zeroed: the per-round sums, the hub-row
// tickets and the two iterate buffers' sentinel rows (cleared by prep_kernel
// instead of four memsets).
struct TileZero {
    double *red;
    int64_t red_n;
    int *long_cnt;
    int n_cnt;
    unsigned char *sent0, *sent1;
    int sent_bytes;
};

template <class S, class R, int W>
__global__ void __launch_bounds__(kThreads) prep_kernel(const TileCols cols,
                                                        const int32_t *__restrict__ perm, int64_t n,
                                                        const double *__restrict__ inv64, S *y0,
                                                        R *rho, R *comp, const TileZero z) {
    const int64_t t0 = blockIdx.x * (int64_t)kThreads + threadIdx.x;
    const int64_t nt = (int64_t)gridDim.x * kThreads;
    for (int64_t i = t0; i < z.red_n; i += nt) z.red[i] = 0.0;
    for (int64_t i = t0; i < z.n_cnt; i += nt) z.long_cnt[i] = 0;
    for (int64_t i = t0; i < z.sent_bytes; i += nt) {
        z.sent0[i] = 0;
        z.sent1[i] = 0;
    }
    for (int64_t u = t0; u < n;
         u += (int64_t)gridDim.x * kThreads) {
        const int32_t src = perm[u];
        const double inv = inv64[u];
#pragma unroll
        for (int b = 0; b < W; ++b) {
            put(y0 + u * W + b, __dmul_rn(cols.p[b][src], inv));
            put(rho + u * W + b, __dmul_rn(cols.c0half[b], get(y0 + u * W + b)));
            if (comp) put(comp + u * W + b, 0.0);
        }
    }
}

// Per-block partials of sum_u d_u rho[u] for each column (fixed order).
template <class R, int W>
__global__ void __launch_bounds__(kThreads) norm_partial_kernel(const R *__restrict__ rho,
                                                                const double *__restrict__ deg64,
                                                                int64_t n, double *part) {
    double v[W];
#pragma unroll
    for (int b = 0; b < W; ++b) v[b] = 0.0;
    for (int64_t u = blockIdx.x * (int64_t)kThreads + threadIdx.x; u < n;
         u += (int64_t)gridDim.x * kThreads)
#pragma unroll
        for (int b = 0; b < W; ++b) v[b] = __fma_rn(deg64[u], get(rho + u * W + b), v[b]);
    cta_sum<W>(v, part + W * blockIdx.x);
}

// pi_b[perm[u]] = scale_b * d_u * rho[u][b].
template <class R, int W>
__global__ void __launch_bounds__(kThreads) finalize_kernel(const TileCols cols,
                                                            const R *__restrict__ rho,
                                                            const double *__restrict__ deg64,
                                                            const int32_t *__restrict__ perm,
                                                            int64_t n, const double *sums,
                                                            int normalize) {
    __shared__ double s_scale[W];
    if (threadIdx.x < W)
        s_scale[threadIdx.x] = normalize == 0 ? __drcp_rn(sums[threadIdx.x]) : cols.scale[threadIdx.x];
    __syncthreads();
    for (int64_t u = blockIdx.x * (int64_t)kThreads + threadIdx.x; u < n;
         u += (int64_t)gridDim.x * kThreads) {
        const int32_t dst = perm[u];
        const double d = deg64[u];
#pragma unroll
        for (int b = 0; b < W; ++b)
            cols.pi[b][dst] = __dmul_rn(s_scale[b], __dmul_rn(d, get(rho + u * W + b)));
    }
}

static size_t store_bytes(int prec) { return prec == CPAA_F64 || prec == CPAA_DF64 ? 8 : prec == CPAA_F32 ? 4 : 2; }

int stats_blocks(int64_t n) { return (int)std::min<int64_t>((n + kThreads - 1) / kThreads, kPrepBlocks); }

// The small buffers of the fixed-order reductions (needed before any stats pass).
cpaa_status ensure_reduction_buffers(cpaa_graph *g) {
    Workspace &w = g->ws;
    cpaa_status st;
    if (!w.part) {
        if ((st = dev_alloc(g, (void **)&w.part, sizeof(double) * kMaxWidth * kPrepBlocks * 3)) != CPAA_OK) return st;
    }
    if (!w.sums) {
        if ((st = dev_alloc(g, (void **)&w.sums, sizeof(double) * 4 * kMaxWidth)) != CPAA_OK) return st;
    }
    if (!w.h_sums) CPAA_CUDA(cudaMallocHost((void **)&w.h_sums, sizeof(double) * 4 * kMaxWidth));
    return CPAA_OK;
}

static cpaa_status ensure_workspace_buffers(cpaa_graph *g, int prec, int width, int max_rounds);

// Sizes the workspace; captured round graphs refer to its buffers, so they
// are dropped when any buffer moves.
cpaa_status ensure_workspace(cpaa_graph *g, int prec, int width, int max_rounds) {
    Workspace &w = g->ws;
    const void *before[] = {w.y0, w.y1, w.rho, w.comp, w.red, w.long_part, w.ipart, w.ipart2, w.maxl1};
    const cpaa_status st = ensure_workspace_buffers(g, prec, width, max_rounds);
    const void *after[] = {w.y0, w.y1, w.rho, w.comp, w.red, w.long_part, w.ipart, w.ipart2, w.maxl1};
    if (std::memcmp(before, after, sizeof before) != 0) {
        for (auto &rg : w.round_graphs) cudaGraphExecDestroy(rg.exec);
        w.round_graphs.clear();
    }
    return st;
}

static cpaa_status ensure_workspace_buffers(cpaa_graph *g, int prec, int width, int max_rounds) {
    Workspace &w = g->ws;
    const int64_t n = g->n;
    cpaa_status st;
    const size_t vb = store_bytes(prec) * (size_t)(n + 1) * width;
    const size_t rb = 8 * (size_t)n * width;  // sized for FP64 so precisions can share it
    if (w.vec_bytes < vb) {
        dev_free(g, &w.y0, w.vec_bytes);
        dev_free(g, &w.y1, w.vec_bytes);
        w.vec_bytes = 0;
        if ((st = dev_alloc(g, &w.y0, vb)) != CPAA_OK) return st;
        if ((st = dev_alloc(g, &w.y1, vb)) != CPAA_OK) return st;
        w.vec_bytes = vb;
    }
    if (w.rho_bytes < rb) {
        dev_free(g, &w.rho, w.rho_bytes);
        dev_free(g, &w.comp, w.rho_bytes);
        w.rho_bytes = 0;
        if ((st = dev_alloc(g, &w.rho, rb)) != CPAA_OK) return st;
        if ((st = dev_alloc(g, &w.comp, rb)) != CPAA_OK) return st;
        w.rho_bytes = rb;
    }
    const size_t red = sizeof(double) * 2 * (size_t)width * (max_rounds + 1);
    if (w.red_bytes < red) {
        dev_free(g, (void **)&w.red, w.red_bytes);
        w.red_bytes = 0;
        if ((st = dev_alloc(g, (void **)&w.red, red)) != CPAA_OK) return st;
        w.red_bytes = red;
    }
    const size_t ip = sizeof(double) * 2 * (size_t)width * ((size_t)g->n_hub + g->num_chunks);
    if (w.ipart_bytes < ip) {
        dev_free(g, (void **)&w.ipart, w.ipart_bytes);
        w.ipart_bytes = 0;
        if ((st = dev_alloc(g, (void **)&w.ipart, ip)) != CPAA_OK) return st;
        w.ipart_bytes = ip;
    }
    if (!w.ipart2) {
        if ((st = dev_alloc(g, (void **)&w.ipart2, sizeof(double) * 2 * kMaxWidth * kSumBlocks)) != CPAA_OK)
            return st;
        if ((st = dev_alloc(g, &w.ivtab, sizeof(double) * (size_t)g->tab_n)) != CPAA_OK) return st;
        if ((st = dev_alloc(g, (void **)&w.maxl1, sizeof(double) * kMaxWidth)) != CPAA_OK) return st;
        if ((st = dev_alloc(g, (void **)&w.stop, sizeof(unsigned))) != CPAA_OK) return st;
        if ((st = dev_alloc(g, (void **)&w.stop_round, sizeof(int) * kMaxWidth)) != CPAA_OK) return st;
    }
    const size_t lp = sizeof(double) * std::max(1, g->num_hub_tiles) * (size_t)width;
    if (w.long_part_bytes < lp) {
        dev_free(g, &w.long_part, w.long_part_bytes);
        w.long_part_bytes = 0;
        if ((st = dev_alloc(g, &w.long_part, lp)) != CPAA_OK) return st;
        w.long_part_bytes = lp;
    }
    return ensure_reduction_buffers(g);
}

// sum p, sum p^2/d and #invalid of one device vector into out[0..2] (device),
// in the same order for every caller.
cudaError_t launch_stats(cpaa_graph *g, const double *p, double *out, cudaStream_t st) {
    if (!g->ws.part) return cudaErrorInvalidValue;  // ensure_reduction_buffers first
    const int blocks = stats_blocks(g->n);
    stats_kernel<<<blocks, kThreads, 0, st>>>(p, g->perm, g->n, g->inv_deg64, g->ws.part);
    block_sum_kernel<3><<<1, kThreads, 0, st>>>(g->ws.part, blocks, out);
    return cudaGetLastError();
}

cpaa_status check_stats(const double *s, int64_t nnz, double *kappa) {
    if (s[2] > 0.0) return fail(CPAA_EINVAL, "p has negative, NaN or infinite entries");
    if (!(std::fabs(s[0] - 1.0) <= 1e-9)) return fail(CPAA_EINVAL, "p must sum to 1 (|sum p - 1| <= 1e-9)");
    *kappa = std::sqrt((double)nnz) * std::sqrt(s[1]);
    return CPAA_OK;
}

template <class S, class R, int W>
static cudaError_t tile_kernels(cpaa_graph *g, const TileJob &job, cudaStream_t st, int phase,
                                const void *final_src) {
    Workspace &w = g->ws;
    const int64_t n = g->n;
    TileCols cols;
    for (int b = 0; b < kMaxWidth; ++b) {
        const int bb = b < job.width ? b : 0;
        cols.p[b] = job.p[bb];
        cols.pi[b] = job.pi[bb];
        cols.c0half[b] = job.c0half[bb];
        // normalize = 1: (1 - c) pibar for CPAA (Sec. 2.1); the power iterate
        // x_T is already the estimate
        cols.scale[b] = job.power ? 1.0 : 1.0 - job.c[bb];
    }
    const unsigned grid = (unsigned)std::min<int64_t>((n + kThreads - 1) / kThreads, 8192);
    if (phase == 0) {
        int maxM = 0;
        for (int b = 0; b < job.width; ++b) maxM = std::max(maxM, job.rounds[b]);
        TileZero z;
        z.red = w.red;
        z.red_n = 2 * (int64_t)W * (maxM + 1);
        z.long_cnt = g->long_cnt;
        z.n_cnt = std::max(1, g->n_hub);
        z.sent_bytes = (int)(sizeof(S) * W);
        z.sent0 = (unsigned char *)w.y0 + (size_t)z.sent_bytes * n;
        z.sent1 = (unsigned char *)w.y1 + (size_t)z.sent_bytes * n;
        prep_kernel<S, R, W><<<grid, kThreads, 0, st>>>(cols, g->perm, n, g->inv_deg64, (S *)w.y0,
                                                        (R *)w.rho,
                                                        std::is_same<R, float>::value ? (R *)w.comp : nullptr, z);
        if (job.lambda_lo > -1.0 && !job.power)
            launch_ivtab(g, job.precision, 1.0 / interval_map(0.5, job.lambda_lo).half, w.ivtab, st);
    } else {
        // the accumulator, or (power method) the last iterate, which has the
        // same element type on the FP64 and FP32 paths
        const R *src = (const R *)(final_src ? final_src : w.rho);
        const int blocks = stats_blocks(n);
        norm_partial_kernel<R, W><<<blocks, kThreads, 0, st>>>(src, g->deg64, n, w.part);
        block_sum_kernel<W><<<1, kThreads, 0, st>>>(w.part, blocks, w.sums);
        finalize_kernel<R, W><<<grid, kThreads, 0, st>>>(cols, src, g->deg64, g->perm, n, w.sums,
                                                         job.normalize);
    }
    return cudaGetLastError();
}

template <class S, class R>
static cudaError_t tile_kernels_w(cpaa_graph *g, const TileJob &job, cudaStream_t st, int phase,
                                  const void *final_src) {
    switch (job.width) {
        case 1: return tile_kernels<S, R, 1>(g, job, st, phase, final_src);
        case 2: return tile_kernels<S, R, 2>(g, job, st, phase, final_src);
        case 4: return tile_kernels<S, R, 4>(g, job, st, phase, final_src);
        case 8: return tile_kernels<S, R, 8>(g, job, st, phase, final_src);
        case 16: return tile_kernels<S, R, 16>(g, job, st, phase, final_src);
    }
    return cudaErrorInvalidValue;
}

static cudaError_t tile_phase(cpaa_graph *g, const TileJob &job, cudaStream_t st, int phase,
                              const void *final_src = nullptr) {
    switch (job.precision) {
        case CPAA_F64: return tile_kernels_w<double, double>(g, job, st, phase, final_src);
        case CPAA_F32: return tile_kernels_w<float, float>(g, job, st, phase, final_src);
        case CPAA_BF16: return tile_kernels_w<__nv_bfloat16, float>(g, job, st, phase, final_src);
        case CPAA_DF64: return tile_kernels_w<df, df>(g, job, st, phase, final_src);
    }
    return cudaErrorInvalidValue;
}

// Deferred accumulation (StepLaunch::pend, defer): a column leaves the term
// of an odd round k for round k + 1 unless k is its last, so the accumulator
// is read and written in every other round.  k and rounds[b] are the rounds
// of the columns; ck[b][j] their coefficients.
void defer_terms(int k, const int *rounds, int W, const std::vector<std::vector<double>> &ck, StepLaunch &sl) {
    sl.pend = sl.defer = 0;
    for (int b = 0; b < W; ++b) {
        if (k > rounds[b]) continue;
        if ((k & 1) && k < rounds[b]) sl.defer |= 1u << b;
        if (!(k & 1) && k >= 2) {
            sl.pend |= 1u << b;
            sl.ck_prev[b] = ck[b][k - 1];
        }
    }
}

// The M round launches of a tile on stream st.
static cudaError_t launch_rounds(cpaa_graph *g, const TileJob &job, bool history_all_rounds, int maxM,
                                 cudaStream_t st) {
    Workspace &w = g->ws;
    const int W = job.width;
    std::vector<std::vector<double>> ck(W);
    for (int b = 0; b < W; ++b) cheb_coeffs_on(job.c[b], job.lambda_lo, job.rounds[b], ck[b]);
    const bool interval = job.lambda_lo > -1.0 && !job.power;
    const IntervalMap im = interval_map(0.5, job.lambda_lo);  // mid and half depend on the interval alone
    void *buf[2] = {w.y0, w.y1};
    for (int k = 1; k <= maxM; ++k) {
        StepLaunch sl;
        sl.g = g;
        sl.precision = job.precision;
        sl.width = W;
        sl.y_src = buf[(k - 1) & 1];
        sl.y_io = buf[k & 1];
        sl.rho = w.rho;
        sl.comp = w.comp;
        sl.long_part = w.long_part;
        sl.ipart = w.ipart;
        sl.ipart2 = w.ipart2;
        sl.red = w.red + (size_t)k * 2 * W;
        sl.active = 0;
        sl.reduce = 0;
        for (int b = 0; b < kMaxWidth; ++b) sl.ck[b] = 0.0;
        for (int b = 0; b < W; ++b) {
            if (k <= job.rounds[b]) {
                sl.active |= 1u << b;
                sl.ck[b] = job.power ? job.c[b] : ck[b][k];
            }
            if (k == job.rounds[b] || (history_all_rounds && k <= job.rounds[b])) sl.reduce |= 1u << b;
        }
        // every column's last round is known here
        if (!job.power && !job.posteriori && defer_supported(job.precision, W))
            defer_terms(k, job.rounds, W, ck, sl);
        if (job.posteriori) {
            // every round takes its sums; columns still within their
            // rigorous M test the a-posteriori rule after it
            sl.stop = w.stop;
            sl.sa.decide = sl.active;
            for (int b = 0; b < W; ++b) {
                sl.sa.k[b] = k;
                sl.sa.err[b] = err_bound_on(job.c[b], job.lambda_lo, k);
                sl.sa.tol[b] = job.tol;
            }
            sl.sa.normalize = job.normalize;
            sl.sa.maxl1 = w.maxl1;
            sl.sa.stop = w.stop;
            sl.sa.stop_round = w.stop_round;
            sl.reduce |= sl.active;
        }
        sl.first = (k == 1) ? (1u << W) - 1u : 0u;
        sl.power = job.power;
        if (interval) {
            sl.interval = 1;
            sl.ia = 1.0 / im.half;
            sl.mb = -2.0 * im.mid / im.half;
            sl.ivtab = w.ivtab;
        }
        sl.long_cnt = nullptr;
        sl.stream = st;
        if (job.frontier && k <= kFrontierRounds) {
            // grow the ball by one hop, then a round over the items it covers
            const cudaError_t fe = frontier_expand(g, w.fr, k, st);
            if (fe != cudaSuccess) return fe;
            frontier_launch(g, w.fr, k, sl);
        }
        const cudaError_t e = launch_step(sl);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

constexpr size_t kMaxRoundGraphs = 8;

// The round sequence of a tile as an instantiated CUDA graph: found in the
// graph's cache, or captured on the private stream and added to it.  The key
// holds everything the launches read (buffers, widths, coefficients' inputs,
// masks), so a replay issues exactly the launches launch_rounds would.
static cpaa_status round_graph(cpaa_graph *g, const TileJob &job, bool history_all_rounds, int maxM,
                               cudaGraphExec_t *out) {
    Workspace &w = g->ws;
    uint64_t tolb, lob;
    std::memcpy(&tolb, &job.tol, sizeof tolb);
    std::memcpy(&lob, &job.lambda_lo, sizeof lob);
    std::vector<uint64_t> key = {(uint64_t)job.precision, (uint64_t)job.width, (uint64_t)job.power,
                                 (uint64_t)job.frontier, (uint64_t)(uintptr_t)w.fr.cur, lob,
                                 (uint64_t)history_all_rounds, (uint64_t)maxM, (uint64_t)job.posteriori,
                                 job.posteriori ? tolb : 0, (uint64_t)job.normalize,
                                 (uint64_t)(uintptr_t)w.y0, (uint64_t)(uintptr_t)w.y1,
                                 (uint64_t)(uintptr_t)w.rho, (uint64_t)(uintptr_t)w.comp,
                                 (uint64_t)(uintptr_t)w.long_part, (uint64_t)(uintptr_t)w.red,
                                 (uint64_t)(uintptr_t)w.ipart, (uint64_t)(uintptr_t)w.maxl1,
                                 (uint64_t)(uintptr_t)w.ivtab};
    for (int b = 0; b < job.width; ++b) {
        uint64_t cb;
        std::memcpy(&cb, &job.c[b], sizeof cb);
        key.push_back(cb);
        key.push_back((uint64_t)job.rounds[b]);
    }
    for (auto &rg : w.round_graphs)
        if (rg.key == key) {
            *out = rg.exec;
            return CPAA_OK;
        }
    if (!w.capture) CPAA_CUDA(cudaStreamCreateWithFlags(&w.capture, cudaStreamNonBlocking));
    prepare_step(job.precision, job.width, job.lambda_lo > -1.0);
    CPAA_CUDA(cudaStreamBeginCapture(w.capture, cudaStreamCaptureModeThreadLocal));
    const cudaError_t le = launch_rounds(g, job, history_all_rounds, maxM, w.capture);
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(w.capture, &graph);
    if (le != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return cuda_fail(le, "round launch during capture");
    }
    CPAA_CUDA(ce);
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    CPAA_CUDA(ie);
    if (w.round_graphs.size() >= kMaxRoundGraphs) {
        cudaGraphExecDestroy(w.round_graphs.front().exec);
        w.round_graphs.erase(w.round_graphs.begin());
    }
    w.round_graphs.push_back({std::move(key), exec});
    *out = exec;
    return CPAA_OK;
}

// Prep, the rounds and the finalisation of one tile (workspace must be sized).
cpaa_status run_tile(cpaa_graph *g, const TileJob &job, cudaStream_t st, bool history_all_rounds,
                     bool time_rounds) {
    Workspace &w = g->ws;
    const int W = job.width;
    int maxM = 0;
    for (int b = 0; b < W; ++b) maxM = std::max(maxM, job.rounds[b]);
    if (job.posteriori) {
        // the running max of ||T_j p||_1 starts at j = 0 (||p||_1); no column
        // has stopped
        CPAA_CUDA(cudaMemcpyAsync(w.maxl1, job.p_l1, sizeof(double) * W, cudaMemcpyHostToDevice, st));
        CPAA_CUDA(cudaMemsetAsync(w.stop, 0, sizeof(unsigned), st));
        CPAA_CUDA(cudaMemsetAsync(w.stop_round, 0xff, sizeof(int) * kMaxWidth, st));
        // the copy reads the caller's job, which ends with this call
        CPAA_CUDA(cudaStreamSynchronize(st));
    }
    if (job.frontier) {
        cpaa_status fs = ensure_frontier(g, w.fr, g);
        if (fs != CPAA_OK) return fs;
        CPAA_CUDA(frontier_reset(w.fr, st));
        // items the early rounds skip keep a zero partial-sum slot
        CPAA_CUDA(cudaMemsetAsync(w.ipart, 0, sizeof(double) * 2 * (size_t)W * ((size_t)g->n_hub + g->num_chunks),
                                  st));
    }
    // prep also zeroes the sums, the tickets and the sentinel rows n
    CPAA_CUDA(tile_phase(g, job, st, 0));
    // the ball starts at the rows where some column of y_0 = D^-1 p is nonzero
    if (job.frontier) CPAA_CUDA(frontier_mark_nonzero(g, w.fr, job.precision, W, w.y0, w.y1, st));

    cudaGraphExec_t exec = nullptr;
    if (maxM > 0) {
        cpaa_status s = round_graph(g, job, history_all_rounds, maxM, &exec);
        if (s != CPAA_OK) return s;
    }
    if (time_rounds) {
        if (!w.tev[0]) {
            CPAA_CUDA(cudaEventCreate(&w.tev[0]));
            CPAA_CUDA(cudaEventCreate(&w.tev[1]));
        }
        CPAA_CUDA(cudaEventRecord(w.tev[0], st));
    }
    if (exec) CPAA_CUDA(cudaGraphLaunch(exec, st));
    if (time_rounds) CPAA_CUDA(cudaEventRecord(w.tev[1], st));
    void *buf[2] = {w.y0, w.y1};
    CPAA_CUDA(tile_phase(g, job, st, 1, job.power ? buf[maxM & 1] : nullptr));
    return CPAA_OK;
}

// Device time of the last run_tile's rounds (run with time_rounds); waits
// for them.
cpaa_status tile_rounds_ms(cpaa_graph *g, float *ms) {
    Workspace &w = g->ws;
    if (!w.tev[0]) return fail(CPAA_EINVAL, "no timed rounds");
    CPAA_CUDA(cudaEventSynchronize(w.tev[1]));
    CPAA_CUDA(cudaEventElapsedTime(ms, w.tev[0], w.tev[1]));
    return CPAA_OK;
}

// Sums of column b (of a tile of `width`) in round k from the host copy h of
// the reduction slots.
void round_sums(int width, int b, int k, const std::vector<double> &h, double *sumT, double *sumA) {
    *sumT = h[((size_t)k * 2 + 0) * width + b];
    *sumA = h[((size_t)k * 2 + 1) * width + b];
}

}  // namespace cpaa

using namespace cpaa;

// Rounds of the power method for an L1 bound: ||x_T - pi*||_1 <= c^T ||p - pi*||_1
// <= 2 c^T (cP has L1 norm c), so the smallest T with 2 c^T < tol.
static int power_rounds(double c, double tol, int max_rounds) {
    double b = 2.0;
    for (int T = 1; T <= max_rounds; ++T) {
        b *= c;
        if (b < tol) return T;
    }
    return -1;
}

namespace cpaa {

// The interval [lo, 1] a solve's series runs on: -1 unless CPAA_INTERVAL
// (the caller's lambda_lo) or CPAA_CERTIFY_INTERVAL (the graph's own bound)
// raise it.
cpaa_status resolve_interval(const cpaa_graph *g, const cpaa_options &opt, double *lo) {
    *lo = -1.0;
    if (opt.flags & CPAA_INTERVAL) {
        if (!(opt.lambda_lo >= -1.0 && opt.lambda_lo < 1.0)) return fail(CPAA_EINVAL, "lambda_lo must lie in [-1, 1)");
        *lo = opt.lambda_lo;
    }
    if (opt.flags & CPAA_CERTIFY_INTERVAL) *lo = std::max(*lo, graph_lambda_lo(g));
    return CPAA_OK;
}

}  // namespace cpaa

static cpaa_status solve_one(cpaa_graph *g, const double *p, double c, double tol, double *pi,
                             const cpaa_options *opt_in, cpaa_info *info, int power) {
    clear_error();
    cpaa_options opt;
    if (opt_in) opt = *opt_in; else cpaa_options_init(&opt);
    if (!g) return fail(CPAA_EINVAL, "graph is NULL");
    if (!p || !pi) return fail(CPAA_EINVAL, "p / pi is NULL");
    if (!(c > 0.0 && c < 1.0)) return fail(CPAA_EINVAL, "damping c must lie in (0, 1)");
    if (opt.fixed_rounds < 0) return fail(CPAA_EINVAL, "fixed_rounds < 0");
    if (opt.fixed_rounds == 0 && !(tol > 0.0)) return fail(CPAA_EINVAL, "tol must be > 0");
    if (opt.precision != CPAA_F64 && opt.precision != CPAA_F32 && opt.precision != CPAA_BF16 &&
        opt.precision != CPAA_DF64)
        return fail(CPAA_EINVAL, "unknown precision");
    if (power && opt.precision == CPAA_BF16)
        return fail(CPAA_EINVAL, "the power method runs in FP64, FP32 or DF64");
    if (opt.normalize != 0 && opt.normalize != 1) return fail(CPAA_EINVAL, "normalize must be 0 or 1");
    if (opt.stop_rule != CPAA_STOP_RIGOROUS && opt.stop_rule != CPAA_STOP_POSTERIORI)
        return fail(CPAA_EINVAL, "unknown stop_rule");
    if (power && opt.stop_rule != CPAA_STOP_RIGOROUS)
        return fail(CPAA_EINVAL, "the power method has its own stopping rule (2 c^T < tol)");
    const int max_rounds = opt.max_rounds > 0 ? opt.max_rounds : kDefaultMaxRounds;
    if (opt.fixed_rounds > max_rounds) return fail(CPAA_EINVAL, "fixed_rounds > max_rounds");
    double lo = -1.0;
    {
        cpaa_status ls = resolve_interval(g, opt, &lo);
        if (ls != CPAA_OK) return ls;
    }
    if (power) lo = -1.0;  // the power method is not a Chebyshev series
    const bool host_io = (opt.flags & CPAA_DEVICE_IO) == 0;
    cudaStream_t st = (cudaStream_t)opt.stream;
    const int64_t n = g->n;

    cpaa_status s = ensure_workspace(g, opt.precision, 1, max_rounds);
    if (s != CPAA_OK) return s;
    Workspace &w = g->ws;
    if (host_io && w.io_bytes < 2 * sizeof(double) * (size_t)n) {
        dev_free(g, (void **)&w.io, w.io_bytes);
        w.io_bytes = 0;
        if ((s = dev_alloc(g, (void **)&w.io, 2 * sizeof(double) * n)) != CPAA_OK) return s;
        w.io_bytes = 2 * sizeof(double) * n;
    }
    const double *dp = p;
    double *dpi = pi;
    if (host_io) {
        CPAA_CUDA(cudaMemcpyAsync(w.io, p, sizeof(double) * n, cudaMemcpyHostToDevice, st));
        dp = w.io;
        dpi = w.io + n;
    }
    CPAA_CUDA(launch_stats(g, dp, w.sums, st));
    CPAA_CUDA(cudaMemcpyAsync(w.h_sums, w.sums, sizeof(double) * 3, cudaMemcpyDeviceToHost, st));
    CPAA_CUDA(cudaStreamSynchronize(st));
    double kappa = 0;
    if ((s = check_stats(w.h_sums, g->nnz, &kappa)) != CPAA_OK) return s;
    const double sum_p = w.h_sums[0];

    cpaa_status result = CPAA_OK;
    int M = opt.fixed_rounds;
    if (M == 0) {
        M = power ? power_rounds(c, tol, max_rounds)
                  : cpaa_rounds_needed_interval(c, lo, tol, kappa, opt.normalize, max_rounds);
        if (M < 0) {
            M = max_rounds;
            result = CPAA_ENOTCONV;
        }
    }
    std::vector<double> ck0;
    cheb_coeffs_on(c, lo, 0, ck0);
    TileJob job;
    job.lambda_lo = lo;
    job.width = 1;
    job.precision = opt.precision;
    job.normalize = opt.normalize;
    job.p[0] = dp;
    job.pi[0] = dpi;
    job.c[0] = c;
    job.c0half[0] = power ? 1.0 - c : ck0[0] / 2.0;
    job.rounds[0] = M;
    job.power = power;
    job.frontier = !power && (opt.flags & CPAA_SPARSE_FRONTIER) != 0;
    // the a-posteriori rule may stop the rounds before the rigorous M
    job.posteriori = opt.stop_rule == CPAA_STOP_POSTERIORI && opt.fixed_rounds == 0 && M > 0;
    job.tol = tol;
    job.p_l1[0] = sum_p;
    float rounds_ms = 0.0f;
    // per-round sums every round only when the caller asked for the history;
    // otherwise just the last round's (for info)
    const bool time_rounds = (opt.flags & CPAA_TIME_ROUNDS) != 0;
    if ((s = run_tile(g, job, st, opt.history != nullptr, time_rounds)) != CPAA_OK) return s;
    if (host_io) CPAA_CUDA(cudaMemcpyAsync(pi, dpi, sizeof(double) * n, cudaMemcpyDeviceToHost, st));

    bool by_posteriori = false;
    if (job.posteriori) {
        int sr = -1;
        CPAA_CUDA(cudaMemcpyAsync(&sr, w.stop_round, sizeof(int), cudaMemcpyDeviceToHost, st));
        CPAA_CUDA(cudaStreamSynchronize(st));
        if (sr >= 1 && sr <= M) {
            M = sr;
            by_posteriori = true;
            result = CPAA_OK;  // the estimate passed within max_rounds
        }
    }
    if (info || opt.history) {
        std::vector<double> h((size_t)(M + 1) * 2);
        CPAA_CUDA(cudaMemcpyAsync(h.data(), w.red, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, st));
        CPAA_CUDA(cudaMemcpyAsync(w.h_sums + 3, w.sums, sizeof(double), cudaMemcpyDeviceToHost, st));
        CPAA_CUDA(cudaStreamSynchronize(st));
        // round 0 is T_0 = p >= 0: sum T_0 = sum |T_0| = sum p (from the stats)
        if (opt.history) {
            opt.history[0] = opt.history[1] = sum_p;
            for (int k = 1; k <= M; ++k) round_sums(1, 0, k, h, &opt.history[2 * k], &opt.history[2 * k + 1]);
        }
        if (info) {
            info->rounds = M;
            info->kappa = kappa;
            if (power) {
                info->bound = 2.0 * std::pow(c, (double)M);
            } else if (by_posteriori) {
                double ml = sum_p, t = 0, a = 0;
                for (int k = 1; k <= M; ++k) {
                    round_sums(1, 0, k, h, &t, &a);
                    ml = std::max(ml, a);
                }
                info->bound = cpaa_l1_bound_interval(c, lo, M, 2.0 * ml, opt.normalize);
            } else {
                info->bound = cpaa_l1_bound_interval(c, lo, M, kappa, opt.normalize);
            }
            info->lambda_lo = lo;
            if (M == 0) {
                info->mass = info->l1 = sum_p;
            } else {
                round_sums(1, 0, M, h, &info->mass, &info->l1);
            }
            info->sum_pibar = w.h_sums[3];
            // the stream has been synchronised: the round events are complete
            if (time_rounds && (s = tile_rounds_ms(g, &rounds_ms)) != CPAA_OK) return s;
            info->rounds_ms = rounds_ms;
        }
    } else if (host_io) {
        CPAA_CUDA(cudaStreamSynchronize(st));
    }
    if (result == CPAA_ENOTCONV) fail(result, "the L1 bound needs more than max_rounds rounds");
    return result;
}

extern "C" cpaa_status cpaa_solve(cpaa_graph *g, const double *p, double c, double tol, double *pi,
                                  const cpaa_options *opt, cpaa_info *info) {
    return solve_one(g, p, c, tol, pi, opt, info, 0);
}

extern "C" cpaa_status cpaa_power_solve(cpaa_graph *g, const double *p, double c, double tol, double *pi,
                                        const cpaa_options *opt, cpaa_info *info) {
    return solve_one(g, p, c, tol, pi, opt, info, 1);
}
