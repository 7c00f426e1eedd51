// noalloc.cu -- cpaa_solve_fixed_noalloc: a solve that allocates no memory.
//
// Some callers cannot allocate device memory themselves: a host application
// whose allocator owns the whole device (a framework's caching allocator or a
// fixed arena that forbids third-party cudaMalloc), a process held to a strict
// memory budget, or a latency-critical loop that cannot afford the device-wide
// synchronisation cudaMalloc/cudaFree can cause.  This entry point serves them:
// the caller passes the graph, p and pi in device memory, and every
// intermediate vector lives in one file-scope device array of fixed size,
// kNoAllocScratchBytes (32 MiB), that the library reserves on each GPU that
// loads it and keeps until the process exits.
//
// Set-up: a call on a device whose scratch address is not yet known (with
// that device current) looks it up with cudaGetSymbolAddress and caches it
// for that device; only a successful lookup is cached, so a lookup that
// failed (for instance for lack of memory to load the module) is tried again
// by the next call.  Every call reads back an error counter and waits for its
// stream, so no call may be made on a stream that is being captured.  Every
// later call reuses the same array, which keeps the previous call's contents.
// Every value a call reads from the array is written earlier in the same
// call, except the error counter, which is cleared at the start.  Calls whose
// work overlaps on the GPU (two streams, or two host threads) race on the
// array: serialise them.
//
// The kernels are a plain FP64 variant of the round kernel in step.cu: one
// warp per row, lanes striding over the row's entries, a fixed shuffle tree
// for the sum, and the same recurrence and accumulation in the scaled space
// y = D^-1 T.
#include <mutex>

#include "internal.h"

namespace cpaa {
namespace noalloc {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;
constexpr int kMaxDevices = 64;
constexpr int kThreadsNA = 256;
constexpr int kPartBlocks = 1024;
constexpr size_t kAlign = 256;

static __device__ __align__(256) unsigned char g_scratch[kNoAllocScratchBytes];

static void *g_scratch_ptr[kMaxDevices];  // cached device address, NULL until a lookup succeeds
static std::mutex g_setup_mu;

static size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Layout: y0[n] y1[n] rho[n] (FP64), part[kPartBlocks], sum, error counter.
struct Layout {
    size_t y0, y1, rho, part, sum, err, total;
};

static Layout layout(int64_t n) {
    Layout L;
    const size_t v = align_up(sizeof(double) * (size_t)n);
    L.y0 = 0;
    L.y1 = L.y0 + v;
    L.rho = L.y1 + v;
    L.part = L.rho + v;
    L.sum = L.part + align_up(sizeof(double) * kPartBlocks);
    L.err = L.sum + kAlign;
    L.total = L.err + kAlign;
    return L;
}

__device__ __forceinline__ int deg_of(const int32_t *rp, int64_t u) { return rp[u + 1] - rp[u]; }

// y_0 = D^-1 p, rho = (c_0/2) y_0; counts rows of degree 0.
__global__ void __launch_bounds__(kThreadsNA) na_prep(const int32_t *__restrict__ rp,
                                                      const double *__restrict__ p, int64_t n,
                                                      double c0half, double *y0, double *rho,
                                                      unsigned long long *err) {
    for (int64_t u = blockIdx.x * (int64_t)kThreadsNA + threadIdx.x; u < n;
         u += (int64_t)gridDim.x * kThreadsNA) {
        const int d = deg_of(rp, u);
        if (d <= 0) {
            atomicAdd(err, 1ull);
            y0[u] = 0.0;
            rho[u] = 0.0;
            continue;
        }
        const double y = p[u] / (double)d;
        y0[u] = y;
        rho[u] = c0half * y;
    }
}

// One round, one warp per row: y_io[u] <- (2/d) sum y_src[j] - y_io[u]
// (k >= 2) or (1/d) sum y_src[j] (k = 1); rho[u] += c_k y_io[u].  Entry
// ranges are clamped to [0, nnz) and columns outside [0, n) are skipped; both
// are counted as errors, so a malformed CSR never reads out of bounds.
__global__ void __launch_bounds__(kThreadsNA) na_round(const int32_t *__restrict__ rp,
                                                       const int32_t *__restrict__ ci, int64_t n,
                                                       int64_t nnz,
                                                       const double *__restrict__ y_src,
                                                       double *y_io, double *rho, double ck,
                                                       int first, unsigned long long *err) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)kThreadsNA + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * kThreadsNA) >> 5;
    for (int64_t u = warp; u < n; u += nwarps) {
        const int r0 = rp[u], r1 = rp[u + 1];
        const int e0 = max(r0, 0), e1 = (int)min((int64_t)r1, nnz);
        double s = 0.0;
        int bad = (lane == 0 && (e0 != r0 || e1 != r1)) ? 1 : 0;
        for (int e = e0 + lane; e < e1; e += 32) {
            const int j = ci[e];
            if (j < 0 || j >= n) { ++bad; continue; }
            s += __ldg(y_src + j);
        }
        for (int o = 16; o > 0; o >>= 1) {
            s += __shfl_xor_sync(0xffffffffu, s, o);
            bad += __shfl_xor_sync(0xffffffffu, bad, o);
        }
        if (lane == 0) {
            if (bad) atomicAdd(err, (unsigned long long)bad);
            const int d = e1 - e0;
            if (d > 0) {
                const double y = first ? s / (double)d : 2.0 * s / (double)d - y_io[u];
                y_io[u] = y;
                rho[u] = rho[u] + ck * y;
            }
        }
    }
}

// Column range check on its own, for a call with no rounds (na_round checks
// the columns it gathers in every round).
__global__ void __launch_bounds__(kThreadsNA) na_check_cols(const int32_t *__restrict__ ci, int64_t n,
                                                            int64_t nnz, unsigned long long *err) {
    unsigned long long bad = 0;
    for (int64_t e = blockIdx.x * (int64_t)kThreadsNA + threadIdx.x; e < nnz;
         e += (int64_t)gridDim.x * kThreadsNA) {
        const int32_t j = ci[e];
        if (j < 0 || j >= n) ++bad;
    }
    if (bad) atomicAdd(err, bad);
}

// Fixed-order sum of d_u rho[u]: per-CTA partials over a fixed grid.
__global__ void __launch_bounds__(kThreadsNA) na_norm_part(const int32_t *__restrict__ rp,
                                                           const double *__restrict__ rho,
                                                           int64_t n, double *part) {
    __shared__ double s[kThreadsNA];
    double v = 0.0;
    for (int64_t u = blockIdx.x * (int64_t)kThreadsNA + threadIdx.x; u < n;
         u += (int64_t)gridDim.x * kThreadsNA)
        v += (double)deg_of(rp, u) * rho[u];
    s[threadIdx.x] = v;
    __syncthreads();
    for (int o = kThreadsNA / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

__global__ void __launch_bounds__(kThreadsNA) na_norm_sum(const double *part, int nblocks,
                                                          double *sum) {
    __shared__ double s[kThreadsNA];
    double v = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += kThreadsNA) v += part[b];
    s[threadIdx.x] = v;
    __syncthreads();
    for (int o = kThreadsNA / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *sum = s[0];
}

__global__ void __launch_bounds__(kThreadsNA) na_finalize(const int32_t *__restrict__ rp,
                                                          const double *__restrict__ rho,
                                                          int64_t n, const double *sum,
                                                          int normalize, double one_minus_c,
                                                          double *pi) {
    const double scale = normalize == 0 ? 1.0 / *sum : one_minus_c;
    for (int64_t u = blockIdx.x * (int64_t)kThreadsNA + threadIdx.x; u < n;
         u += (int64_t)gridDim.x * kThreadsNA)
        pi[u] = scale * ((double)deg_of(rp, u) * rho[u]);
}

// Per-device address of g_scratch, looked up with that device current.  A
// successful lookup is kept for the life of the process; a failed one is not,
// so the next call tries again.
static cudaError_t scratch_for_current_device(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_ptr[dev]) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_scratch);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            return e;
        }
        g_scratch_ptr[dev] = ptr;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace noalloc
}  // namespace cpaa

using namespace cpaa;
using namespace cpaa::noalloc;

extern "C" cpaa_status cpaa_solve_fixed_noalloc(int64_t n, int64_t nnz, const int32_t *row_ptr,
                                                const int32_t *col_idx, const double *p, double c,
                                                int rounds, int normalize, double *pi,
                                                void *stream) {
    clear_error();
    if (n < 1 || n > CPAA_NOALLOC_MAX_N)
        return fail(CPAA_EINVAL, "n must lie in [1, CPAA_NOALLOC_MAX_N = " +
                                     std::to_string(CPAA_NOALLOC_MAX_N) +
                                     "]: the no-allocation scratch array is fixed at 32 MiB");
    if (nnz < 1 || nnz >= (int64_t(1) << 31)) return fail(CPAA_EINVAL, "nnz out of range [1, 2^31)");
    if (!row_ptr || !col_idx || !p || !pi) return fail(CPAA_EINVAL, "NULL pointer argument");
    if (!(c > 0.0 && c < 1.0)) return fail(CPAA_EINVAL, "damping c must lie in (0, 1)");
    if (rounds < 0 || rounds > kDefaultMaxRounds) return fail(CPAA_EINVAL, "rounds out of range [0, 2000]");
    if (normalize != 0 && normalize != 1) return fail(CPAA_EINVAL, "normalize must be 0 or 1");
    const Layout L = layout(n);
    if (L.total > kNoAllocScratchBytes) return fail(CPAA_EINVAL, "graph too large for the scratch array");

    void *base = nullptr;
    cudaError_t e = scratch_for_current_device(&base);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-allocation scratch)");
    unsigned char *b = static_cast<unsigned char *>(base);
    double *y[2] = {reinterpret_cast<double *>(b + L.y0), reinterpret_cast<double *>(b + L.y1)};
    double *rho = reinterpret_cast<double *>(b + L.rho);
    double *part = reinterpret_cast<double *>(b + L.part);
    double *sum = reinterpret_cast<double *>(b + L.sum);
    unsigned long long *err = reinterpret_cast<unsigned long long *>(b + L.err);
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    std::vector<double> ck;
    cheb_coeffs(c, rounds, ck);
    const unsigned grid = (unsigned)std::min<int64_t>((n + kThreadsNA - 1) / kThreadsNA, 4096);
    const unsigned rgrid = (unsigned)std::min<int64_t>((n * 32 + kThreadsNA - 1) / kThreadsNA, 8192);
    const unsigned pgrid = (unsigned)std::min<int64_t>((n + kThreadsNA - 1) / kThreadsNA, kPartBlocks);
    CPAA_CUDA(cudaMemsetAsync(err, 0, sizeof(unsigned long long), st));
    na_prep<<<grid, kThreadsNA, 0, st>>>(row_ptr, p, n, ck[0] / 2.0, y[0], rho, err);
    CPAA_CUDA(cudaGetLastError());
    if (rounds == 0) {
        na_check_cols<<<grid, kThreadsNA, 0, st>>>(col_idx, n, nnz, err);
        CPAA_CUDA(cudaGetLastError());
    }
    for (int k = 1; k <= rounds; ++k) {
        na_round<<<rgrid, kThreadsNA, 0, st>>>(row_ptr, col_idx, n, nnz, y[(k - 1) & 1], y[k & 1], rho,
                                               ck[k], k == 1, err);
        CPAA_CUDA(cudaGetLastError());
    }
    na_norm_part<<<pgrid, kThreadsNA, 0, st>>>(row_ptr, rho, n, part);
    na_norm_sum<<<1, kThreadsNA, 0, st>>>(part, pgrid, sum);
    na_finalize<<<grid, kThreadsNA, 0, st>>>(row_ptr, rho, n, sum, normalize, 1.0 - c, pi);
    CPAA_CUDA(cudaGetLastError());
    unsigned long long herr = 0;
    CPAA_CUDA(cudaMemcpyAsync(&herr, err, sizeof(herr), cudaMemcpyDeviceToHost, st));
    CPAA_CUDA(cudaStreamSynchronize(st));
    if (herr) return fail(CPAA_EINVAL, std::to_string(herr) +
                                           " invalid CSR entr(ies): a column outside [0, n) or a row of degree 0");
    return CPAA_OK;
}
