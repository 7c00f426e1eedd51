// graph.cu -- graph upload, degree vectors, row tiling and validation.
//
// The graph is the undirected G of Sec. 2.1 held as symmetric CSR.  Its
// degrees d_u = row_ptr[u+1] - row_ptr[u] give P = A D^-1; the step kernels
// work in the scaled space y = D^-1 T (see step.cu), so the graph also keeps
// d and 1/d in FP64 and FP32.
#include <algorithm>
#include <cstring>

#include "internal.h"

namespace cpaa {

__global__ void degree_kernel(const int32_t *__restrict__ row_ptr, int64_t n, double *deg64,
                              double *inv64, float *deg32, float *inv32) {
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n;
         u += (int64_t)gridDim.x * blockDim.x) {
        const int d = row_ptr[u + 1] - row_ptr[u];
        const double dd = (double)d;
        deg64[u] = dd;
        inv64[u] = 1.0 / dd;
        deg32[u] = (float)d;
        inv32[u] = 1.0f / (float)d;
    }
}

// Row of entry e (row_ptr[row] <= e < row_ptr[row+1]); rows are non-empty.
__device__ __forceinline__ int64_t row_of(const int32_t *row_ptr, int64_t n, int64_t e) {
    int64_t lo = 0, hi = n - 1;
    while (lo < hi) {
        int64_t mid = (lo + hi + 1) >> 1;
        if (row_ptr[mid] <= e) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// bad[0]: column out of range, bad[1]: row not strictly ascending,
// bad[2]: entry (u, v) without its mirror (v, u).
__global__ void validate_kernel(const int32_t *__restrict__ row_ptr,
                                const int32_t *__restrict__ col_idx, int64_t n, int64_t nnz,
                                unsigned long long *bad) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t u = row_of(row_ptr, n, e);
        const int32_t v = col_idx[e];
        if (v < 0 || v >= n) { atomicAdd(&bad[0], 1ull); continue; }
        if (e > row_ptr[u] && col_idx[e - 1] >= v) atomicAdd(&bad[1], 1ull);
        // binary search for u in row v (rows assumed ascending; a disorder is
        // reported above and may also show up here)
        int32_t lo = row_ptr[v], hi = row_ptr[v + 1] - 1;
        bool found = false;
        while (lo <= hi) {
            const int32_t mid = lo + ((hi - lo) >> 1);
            const int32_t w = col_idx[mid];
            if (w == u) { found = true; break; }
            if (w < u) lo = mid + 1; else hi = mid - 1;
        }
        if (!found) atomicAdd(&bad[2], 1ull);
    }
}

static void release(cpaa_graph *g) {
    if (!g) return;
    Workspace &w = g->ws;
    cudaFree(w.y0); cudaFree(w.y1); cudaFree(w.rho); cudaFree(w.comp); cudaFree(w.red);
    cudaFree(w.prep_part); cudaFree(w.prep_out); cudaFree(w.d_pi); cudaFree(w.d_p);
    if (w.h_prep) cudaFreeHost(w.h_prep);
    cudaFree(g->row_ptr); cudaFree(g->col_idx); cudaFree(g->deg64); cudaFree(g->inv_deg64);
    cudaFree(g->deg32); cudaFree(g->inv_deg32); cudaFree(g->tiles); cudaFree(g->long_part);
    cudaFree(g->long_cnt);
    delete g;
}

// Greedy tiling over the host copy of row_ptr (see internal.h for the
// encoding).  One pass, O(n).
static void build_tiles(const int32_t *rp, int64_t n, std::vector<int4> &chunks,
                        std::vector<int4> &blocks, int &num_long, int &total_chunks) {
    num_long = 0;
    total_chunks = 0;
    int64_t r = 0;
    while (r < n) {
        const int64_t d = (int64_t)rp[r + 1] - rp[r];
        if (d + 1 > kTileItems) {
            const int nch = (int)((d + kTileItems - 1) / kTileItems);
            for (int j = 0; j < nch; ++j)
                chunks.push_back(make_int4((int)r, j, total_chunks, num_long + 1));
            total_chunks += nch;
            ++num_long;
            ++r;
            continue;
        }
        const int64_t r0 = r;
        int64_t items = 0;
        while (r < n) {
            const int64_t dr = (int64_t)rp[r + 1] - rp[r];
            if (dr + 1 > kTileItems || items + dr + 1 > kTileItems) break;
            items += dr + 1;
            ++r;
        }
        blocks.push_back(make_int4((int)r0, (int)r, 0, 0));
    }
}

}  // namespace cpaa

using namespace cpaa;

extern "C" cpaa_status cpaa_graph_create(int64_t n, int64_t nnz, const int32_t *row_ptr,
                                         const int32_t *col_idx, unsigned flags,
                                         cpaa_graph **out) {
    clear_error();
    if (!out) return fail(CPAA_EINVAL, "out is NULL");
    *out = nullptr;
    if (n < 1 || n >= (int64_t(1) << 31)) return fail(CPAA_EINVAL, "n out of range [1, 2^31)");
    if (nnz < 1 || nnz >= (int64_t(1) << 31)) return fail(CPAA_EINVAL, "nnz out of range [1, 2^31)");
    if (!row_ptr || !col_idx) return fail(CPAA_EINVAL, "row_ptr / col_idx is NULL");
    const bool dev_in = (flags & CPAA_GRAPH_DEVICE_INPUT) != 0;

    // Host copy of row_ptr: needed for the tiling in any case.
    std::vector<int32_t> hrp((size_t)n + 1);
    if (dev_in) {
        CPAA_CUDA(cudaMemcpy(hrp.data(), row_ptr, sizeof(int32_t) * (n + 1), cudaMemcpyDeviceToHost));
    } else {
        std::memcpy(hrp.data(), row_ptr, sizeof(int32_t) * (n + 1));
    }
    if (hrp[0] != 0) return fail(CPAA_EINVAL, "row_ptr[0] != 0");
    if ((int64_t)hrp[n] != nnz) return fail(CPAA_EINVAL, "row_ptr[n] != nnz");
    for (int64_t u = 0; u < n; ++u) {
        if (hrp[u + 1] < hrp[u]) return fail(CPAA_EINVAL, "row_ptr decreases at row " + std::to_string(u));
        if (hrp[u + 1] == hrp[u])
            return fail(CPAA_EINVAL, "vertex " + std::to_string(u) + " has degree 0 (Sec. 2.1 needs d_i > 0)");
    }

    cpaa_graph *g = new cpaa_graph();
    g->n = n;
    g->nnz = nnz;
    cudaGetDevice(&g->device);
    cpaa_status st;
#define ALLOC(ptr, bytes)                                                      \
    do {                                                                       \
        st = dev_alloc(g, (void **)&(ptr), (bytes));                           \
        if (st != CPAA_OK) { release(g); return st; }                          \
    } while (0)
#define CK(call)                                                               \
    do {                                                                       \
        cudaError_t e_ = (call);                                               \
        if (e_ != cudaSuccess) { st = cuda_fail(e_, #call); release(g); return st; } \
    } while (0)

    ALLOC(g->row_ptr, sizeof(int32_t) * (n + 1));
    ALLOC(g->col_idx, sizeof(int32_t) * (nnz + 4));
    const cudaMemcpyKind kind = dev_in ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CK(cudaMemcpy(g->row_ptr, row_ptr, sizeof(int32_t) * (n + 1), kind));
    CK(cudaMemcpy(g->col_idx, col_idx, sizeof(int32_t) * nnz, kind));
    CK(cudaMemset(g->col_idx + nnz, 0, sizeof(int32_t) * 4));

    if (flags & CPAA_GRAPH_VALIDATE) {
        unsigned long long *bad = nullptr;
        ALLOC(bad, 3 * sizeof(unsigned long long));
        CK(cudaMemset(bad, 0, 3 * sizeof(unsigned long long)));
        validate_kernel<<<1024, 256>>>(g->row_ptr, g->col_idx, n, nnz, bad);
        CK(cudaGetLastError());
        unsigned long long hb[3];
        CK(cudaMemcpy(hb, bad, sizeof(hb), cudaMemcpyDeviceToHost));
        dev_free(g, (void **)&bad, 3 * sizeof(unsigned long long));
        if (hb[0] || hb[1] || hb[2]) {
            std::string m = "invalid CSR: " + std::to_string(hb[0]) + " column(s) out of range, " +
                            std::to_string(hb[1]) + " unsorted/duplicate entr(ies), " +
                            std::to_string(hb[2]) + " entr(ies) without a mirror (graph not undirected)";
            release(g);
            return fail(CPAA_EINVAL, m);
        }
    }

    ALLOC(g->deg64, sizeof(double) * n);
    ALLOC(g->inv_deg64, sizeof(double) * n);
    ALLOC(g->deg32, sizeof(float) * n);
    ALLOC(g->inv_deg32, sizeof(float) * n);
    degree_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256>>>(
        g->row_ptr, n, g->deg64, g->inv_deg64, g->deg32, g->inv_deg32);
    CK(cudaGetLastError());

    std::vector<int4> chunks, blocks;
    build_tiles(hrp.data(), n, chunks, blocks, g->num_long, g->total_chunks);
    g->num_chunk_tiles = (int)chunks.size();
    g->num_tiles = (int)(chunks.size() + blocks.size());
    chunks.insert(chunks.end(), blocks.begin(), blocks.end());
    ALLOC(g->tiles, sizeof(int4) * chunks.size());
    CK(cudaMemcpy(g->tiles, chunks.data(), sizeof(int4) * chunks.size(), cudaMemcpyHostToDevice));
    ALLOC(g->long_part, sizeof(double) * std::max(1, g->total_chunks));
    ALLOC(g->long_cnt, sizeof(int) * std::max(1, g->num_long));
    CK(cudaMemset(g->long_cnt, 0, sizeof(int) * std::max(1, g->num_long)));
    CK(cudaDeviceSynchronize());
#undef ALLOC
#undef CK
    *out = g;
    return CPAA_OK;
}

extern "C" cpaa_status cpaa_graph_destroy(cpaa_graph *g) {
    clear_error();
    if (!g) return CPAA_OK;
    cudaDeviceSynchronize();
    release(g);
    return CPAA_OK;
}

extern "C" cpaa_status cpaa_graph_info(const cpaa_graph *g, int64_t *n, int64_t *nnz,
                                       int64_t *device_bytes, int64_t *num_tiles) {
    clear_error();
    if (!g) return fail(CPAA_EINVAL, "graph is NULL");
    if (n) *n = g->n;
    if (nnz) *nnz = g->nnz;
    if (device_bytes) *device_bytes = g->device_bytes;
    if (num_tiles) *num_tiles = g->num_tiles;
    return CPAA_OK;
}
