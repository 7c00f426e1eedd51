// graph.cu -- graph upload, validation, relabelling and the SELL-C-sigma /
// hub layout the round kernel walks (see internal.h).
//
// The graph is the undirected G of Sec. 2.1 held as symmetric CSR.  Its
// degrees d_u = row_ptr[u+1] - row_ptr[u] give P = A D^-1; the round kernels
// work in the scaled space y = D^-1 T (see step.cu), so the graph also keeps
// d, 1/d and 2/d in FP64 and FP32 (and d, 2/d as double-floats), in the new
// vertex order.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <numeric>
#include <thread>

#include <cub/device/device_segmented_sort.cuh>

#include "internal.h"

namespace cpaa {

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

// Per-vertex arrays in the new order, and the inverse permutation.
__global__ void vertex_arrays_kernel(const int32_t *__restrict__ row_ptr,
                                     const int32_t *__restrict__ perm, int64_t n, double *deg64,
                                     double *inv64, double *inv2_64, float *deg32, float *inv32,
                                     float *inv2_32, df *deg_df, df *inv_df, df *inv2_df, uint16_t *deg16,
                                     int32_t *inv_perm) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int32_t u = perm[r];
        const int d = row_ptr[u + 1] - row_ptr[u];
        deg64[r] = (double)d;
        inv64[r] = 1.0 / (double)d;
        inv2_64[r] = 2.0 / (double)d;
        deg32[r] = (float)d;
        inv32[r] = 1.0f / (float)d;
        inv2_32[r] = 2.0f / (float)d;
        deg_df[r] = df((double)d);
        inv_df[r] = df(1.0 / (double)d);
        inv2_df[r] = df(2.0 / (double)d);
        deg16[r] = (uint16_t)min(d, 65535);
        inv_perm[u] = (int32_t)r;
    }
}

// Column ids in the new vertex order (in place; col_idx is the library's own
// device copy).  Every column is range-checked here, whatever the caller's
// flags: an id outside [0, n) is counted in *bad and replaced by 0, so it is
// never used as an index (the caller then rejects the graph).
__global__ void relabel_kernel(int32_t *col, const int32_t *__restrict__ inv_perm, int64_t n, int64_t nnz,
                               unsigned long long *bad) {
    unsigned long long nbad = 0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = col[e];
        if (v < 0 || v >= n) {
            ++nbad;
            col[e] = 0;
        } else {
            col[e] = inv_perm[v];
        }
    }
    if (nbad) atomicAdd(bad, nbad);
}

// One warp per SELL chunk: lane l writes entry i of row n_hub + 32c + l at
// chunk_off[c] + 128 (i / 4) + 4 l + i % 4 (each lane's entries in groups of
// four, one 16-byte load); padding gets the sentinel n.  rcol holds the
// relabelled graph's CSR rows (new ids, ascending) at the caller's row offsets,
// so a row's first entries are its hub and heavy neighbours: the 32 lanes of a
// chunk gather those together, from the few cache lines that hold them.
__global__ void build_sell_kernel(const int32_t *__restrict__ row_ptr,
                                  const int32_t *__restrict__ rcol,
                                  const int32_t *__restrict__ perm, int64_t n, int n_hub,
                                  int num_chunks, const int64_t *__restrict__ chunk_off,
                                  const int32_t *__restrict__ chunk_len, int32_t *sell,
                                  unsigned long long *loops) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long nloop = 0;
    for (int64_t c = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; c < num_chunks;
         c += nwarps) {
        const int64_t r = n_hub + c * kChunkRows + lane;
        int e0 = 0, d = 0;
        if (r < n) {
            const int32_t u = perm[r];
            e0 = row_ptr[u];
            d = row_ptr[u + 1] - e0;
        }
        const int64_t off = chunk_off[c];
        const int len = chunk_len[c];
        bool loop = false;
        for (int i = 0; i < len; ++i) {
            const int32_t v = (i < d) ? rcol[e0 + i] : (int32_t)n;
            loop |= (i < d && v == r);
            sell[off + (int64_t)(i / kSellVec) * (kChunkRows * kSellVec) + lane * kSellVec + i % kSellVec] = v;
        }
        nloop += loop ? 1 : 0;
    }
    if (nloop) atomicAdd(loops, nloop);  // rows with a self-loop
}

// One CTA per hub row: a copy of its relabelled, sorted entries.
__global__ void build_hub_kernel(const int32_t *__restrict__ row_ptr,
                                 const int32_t *__restrict__ rcol,
                                 const int32_t *__restrict__ perm,
                                 const int32_t *__restrict__ hub_row_ptr, int n_hub,
                                 int32_t *hub_col, unsigned long long *loops) {
    for (int h = blockIdx.x; h < n_hub; h += gridDim.x) {
        const int32_t u = perm[h];
        const int e0 = row_ptr[u], d = row_ptr[u + 1] - e0;
        const int o = hub_row_ptr[h];
        for (int i = threadIdx.x; i < d; i += blockDim.x) {
            const int32_t v = rcol[e0 + i];
            hub_col[o + i] = v;
            if (v == h) atomicAdd(loops, 1ull);  // the row's self-loop (a row holds each id once)
        }
    }
}

static void release(cpaa_graph *g) {
    if (!g) return;
    Workspace &w = g->ws;
    cudaFree(w.y0); cudaFree(w.y1); cudaFree(w.rho); cudaFree(w.comp); cudaFree(w.red);
    cudaFree(w.long_part); cudaFree(w.part); cudaFree(w.sums); cudaFree(w.io);
    cudaFree(w.ipart); cudaFree(w.ipart2); cudaFree(w.maxl1); cudaFree(w.stop); cudaFree(w.stop_round);
    if (w.h_sums) cudaFreeHost(w.h_sums);
    for (auto &rg : w.round_graphs) cudaGraphExecDestroy(rg.exec);
    if (w.capture) cudaStreamDestroy(w.capture);
    if (w.tev[0]) cudaEventDestroy(w.tev[0]);
    if (w.tev[1]) cudaEventDestroy(w.tev[1]);
    cudaFree(w.fr.cur); cudaFree(w.fr.ring); cudaFree(w.fr.add); cudaFree(w.fr.full);
    cudaFree(g->perm); cudaFree(g->hub_row_ptr); cudaFree(g->hub_col); cudaFree(g->hub_tiles);
    cudaFree(g->long_cnt); cudaFree(g->sell_col); cudaFree(g->chunk_off);
    cudaFree(g->chunk_len); cudaFree(g->chunk_order); cudaFree(g->chunk_desc); cudaFree(g->deg64); cudaFree(g->inv_deg64);
    cudaFree(g->deg32); cudaFree(g->inv_deg32); cudaFree(g->inv2_deg64); cudaFree(g->inv2_deg32);
    cudaFree(g->deg_df); cudaFree(g->inv_deg_df); cudaFree(g->inv2_deg_df);
    cudaFree(g->tab64); cudaFree(g->tab32); cudaFree(g->tab_df); cudaFree(g->deg16); cudaFree(w.ivtab);
    delete g;
}

// Host side of the relabelling: hub rows by decreasing degree, then windows
// of lp.sort_window rows sorted by decreasing degree (stable).
struct HostLayout {
    std::vector<int32_t> perm;
    int n_hub = 0;
    std::vector<int32_t> hub_row_ptr;
    std::vector<int64_t> chunk_off;
    std::vector<int32_t> chunk_len;
    std::vector<int32_t> chunk_order;
    std::vector<int4> chunk_desc;
    std::vector<int4> hub_tiles;
    int64_t sell_entries = 0;
};

static int hub_degree(int64_t nnz) {
    return (int)std::min<int64_t>(kHubDegree, std::max<int64_t>(kMinHubDegree, nnz / 4096));
}

static int hub_tile_entries(int hub_deg) { return std::min(kMaxHubTile, std::max(kMinHubTile, 2 * hub_deg)); }

// The default layout of a graph with nnz entries.
static LayoutParams default_layout(int64_t nnz) {
    LayoutParams lp;
    lp.hub_degree = hub_degree(nnz);
    lp.hub_tile = hub_tile_entries(lp.hub_degree);
    lp.long_chunk = nnz < (int64_t(1) << 22) ? kSmallLongChunk : kLongChunk;
    lp.sort_window = kSortWindow;
    return lp;
}

// Caller's parameters with every 0 replaced by its default; out-of-range values are EINVAL.
static cpaa_status resolve_layout(const cpaa_layout_params *in, int64_t nnz, LayoutParams *out) {
    LayoutParams lp = default_layout(nnz);
    if (in) {
        if (in->hub_degree < 0 || (in->hub_degree > 0 && in->hub_degree < 32))
            return fail(CPAA_EINVAL, "layout hub_degree must be 0 (default) or >= 32");
        if (in->hub_tile < 0 || (in->hub_tile > 0 && (in->hub_tile < 256 || in->hub_tile > (1 << 20) ||
                                                     in->hub_tile % 4 != 0)))
            return fail(CPAA_EINVAL, "layout hub_tile must be 0 (default) or a multiple of 4 in [256, 2^20]");
        if (in->long_chunk < 0) return fail(CPAA_EINVAL, "layout long_chunk must be >= 0");
        if (in->sort_window < 0 ||
            (in->sort_window > 0 && (in->sort_window % kChunkRows != 0 || in->sort_window > (1 << 20))))
            return fail(CPAA_EINVAL, "layout sort_window must be 0 (default) or a multiple of 32 up to 2^20");
        if (in->hub_degree > 0) {
            lp.hub_degree = in->hub_degree;
            lp.hub_tile = hub_tile_entries(lp.hub_degree);
        }
        if (in->hub_tile > 0) lp.hub_tile = in->hub_tile;
        if (in->long_chunk > 0) lp.long_chunk = in->long_chunk;
        if (in->sort_window > 0) lp.sort_window = in->sort_window;
    }
    *out = lp;
    return CPAA_OK;
}

static void host_layout(const int32_t *rp, int64_t n, const LayoutParams &lp, HostLayout &L) {
    const int hub_deg = lp.hub_degree, tile = lp.hub_tile, window = lp.sort_window;
    auto deg = [&](int32_t u) { return rp[u + 1] - rp[u]; };
    // heavy rows (degree at least kHeavyFactor times the mean, and at least kHeavyMin) follow the
    // hubs as one block sorted by degree: in an undirected graph a vertex is
    // gathered once per edge, so these are the hottest gather targets, and
    // placing them together keeps their iterate values in few cache lines
    // whatever order the caller's ids have
    const int64_t nnz = rp[n];
    const int heavy = (int)std::max<int64_t>(kHeavyMin, kHeavyFactor * nnz / std::max<int64_t>(1, n));
    std::vector<int32_t> hubs, heavy_rows, rest;
    rest.reserve((size_t)n);
    for (int64_t u = 0; u < n; ++u) {
        const int d = deg((int32_t)u);
        (d > hub_deg ? hubs : d >= heavy ? heavy_rows : rest).push_back((int32_t)u);
    }
    std::stable_sort(hubs.begin(), hubs.end(), [&](int32_t a, int32_t b) { return deg(a) > deg(b); });
    std::stable_sort(heavy_rows.begin(), heavy_rows.end(), [&](int32_t a, int32_t b) { return deg(a) > deg(b); });
    // the heavy block leads the SELL part; the window sort below keeps it first
    // (its rows are the longest of any window they share with light rows)
    rest.insert(rest.begin(), heavy_rows.begin(), heavy_rows.end());
    const int64_t nrest = (int64_t)rest.size();
    const int64_t nwin = (nrest + window - 1) / window;
    const int nth = (int)std::max<int64_t>(1, std::min<int64_t>(16, nwin / 64));
    std::vector<std::thread> th;
    for (int t = 0; t < nth; ++t)
        th.emplace_back([&, t]() {
            for (int64_t w = t; w < nwin; w += nth) {
                auto b = rest.begin() + w * window;
                auto e = rest.begin() + std::min<int64_t>(nrest, (w + 1) * window);
                std::stable_sort(b, e, [&](int32_t a, int32_t c) { return deg(a) > deg(c); });
            }
        });
    for (auto &x : th) x.join();
    L.n_hub = (int)hubs.size();
    L.perm = hubs;
    L.perm.insert(L.perm.end(), rest.begin(), rest.end());
    L.hub_row_ptr.assign((size_t)L.n_hub + 1, 0);
    int slot = 0;
    for (int h = 0; h < L.n_hub; ++h) {
        const int d = deg(hubs[h]);
        L.hub_row_ptr[h + 1] = L.hub_row_ptr[h] + d;
        const int nt = (d + tile - 1) / tile;
        for (int j = 0; j < nt; ++j) L.hub_tiles.push_back(make_int4(h, j, slot, h + 1));
        slot += nt;
    }
    const int64_t nch = (nrest + kChunkRows - 1) / kChunkRows;
    L.chunk_off.resize((size_t)nch);
    L.chunk_len.resize((size_t)nch);
    int64_t off = 0;
    for (int64_t c = 0; c < nch; ++c) {
        // the longest row, rounded up to whole groups of kSellVec entries
        const int len = (deg(rest[(size_t)(c * kChunkRows)]) + kSellVec - 1) / kSellVec * kSellVec;
        L.chunk_off[c] = off;
        L.chunk_len[c] = len;
        off += (int64_t)len * kChunkRows;
    }
    L.sell_entries = off;
    L.chunk_order.resize((size_t)nch);
    std::iota(L.chunk_order.begin(), L.chunk_order.end(), 0);
    std::stable_sort(L.chunk_order.begin(), L.chunk_order.end(),
                     [&](int32_t a, int32_t b) { return L.chunk_len[a] > L.chunk_len[b]; });
    // one 16-byte descriptor per chunk in processing order: the round kernel
    // finds a chunk's row, offset, stored length and longest row (the entries
    // it gathers per lane; the stored groups past it are never read) with a
    // single load
    L.chunk_desc.resize((size_t)nch);
    for (int64_t i = 0; i < nch; ++i) {
        const int32_t c = L.chunk_order[(size_t)i];
        L.chunk_desc[(size_t)i] = make_int4(c, (int)(L.chunk_off[c] / (kChunkRows * kSellVec)), L.chunk_len[c],
                                            deg(rest[(size_t)c * kChunkRows]));
    }
}

// The graph for a checked host copy hrp of row_ptr and resolved parameters.
static cpaa_status build_graph(int64_t n, int64_t nnz, const int32_t *row_ptr, const int32_t *col_idx,
                               unsigned flags, const std::vector<int32_t> &hrp, const LayoutParams &lp,
                               cpaa_graph **out) {
    const bool dev_in = (flags & CPAA_GRAPH_DEVICE_INPUT) != 0;
    cpaa_graph *g = new cpaa_graph();
    g->n = n;
    g->nnz = nnz;
    cudaGetDevice(&g->device);
    cpaa_status st;
    int32_t *d_rp = nullptr, *d_ci = nullptr, *d_inv = nullptr, *d_rs = nullptr;
    unsigned long long *d_bad = nullptr;  // [0..2] validate_kernel, [3] relabel_kernel
    unsigned long long *d_loops = nullptr;  // rows with a self-loop
    void *d_tmp = nullptr;
    size_t rp_bytes = sizeof(int32_t) * (n + 1), ci_bytes = sizeof(int32_t) * nnz, tmp_bytes = 0;
#define ALLOC(ptr, bytes)                                                      \
    do {                                                                       \
        st = dev_alloc(g, (void **)&(ptr), (bytes));                           \
        if (st != CPAA_OK) goto fail_out;                                      \
    } while (0)
#define CK(call)                                                               \
    do {                                                                       \
        cudaError_t e_ = (call);                                               \
        if (e_ != cudaSuccess) { st = cuda_fail(e_, #call); goto fail_out; }   \
    } while (0)
    {
        // original CSR on the device (a temporary copy)
        const cudaMemcpyKind kind = dev_in ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        ALLOC(d_rp, rp_bytes);
        ALLOC(d_ci, ci_bytes);
        CK(cudaMemcpy(d_rp, row_ptr, rp_bytes, kind));
        CK(cudaMemcpy(d_ci, col_idx, ci_bytes, kind));

        // order and symmetry (and column range) unless the caller vouches for
        // the CSR; the column range alone is checked again by relabel_kernel
        ALLOC(d_bad, 4 * sizeof(unsigned long long));
        CK(cudaMemset(d_bad, 0, 4 * sizeof(unsigned long long)));
        if (!(flags & CPAA_GRAPH_TRUSTED)) {
            validate_kernel<<<1024, 256>>>(d_rp, d_ci, n, nnz, d_bad);
            CK(cudaGetLastError());
            unsigned long long hb[3];
            CK(cudaMemcpy(hb, d_bad, sizeof(hb), cudaMemcpyDeviceToHost));
            if (hb[0] || hb[1] || hb[2]) {
                st = fail(CPAA_EINVAL, "invalid CSR: " + std::to_string(hb[0]) + " column(s) out of range, " +
                                           std::to_string(hb[1]) + " unsorted/duplicate entr(ies), " +
                                           std::to_string(hb[2]) +
                                           " entr(ies) without a mirror (graph not undirected)");
                goto fail_out;
            }
        }

        HostLayout L;
        g->lp = lp;
        g->hub_degree = lp.hub_degree;
        g->hub_tile = lp.hub_tile;
        host_layout(hrp.data(), n, lp, L);
        g->n_hub = L.n_hub;
        g->hub_nnz = L.hub_row_ptr.back();
        g->num_hub_tiles = (int)L.hub_tiles.size();
        g->num_chunks = (int)L.chunk_off.size();
        g->num_long_chunks = 0;
        while (g->num_long_chunks < g->num_chunks &&
               L.chunk_len[L.chunk_order[g->num_long_chunks]] > std::min(lp.long_chunk, kMaxShortRow))
            ++g->num_long_chunks;
        g->sell_entries = L.sell_entries;

        ALLOC(g->perm, sizeof(int32_t) * n);
        ALLOC(d_inv, sizeof(int32_t) * n);
        CK(cudaMemcpy(g->perm, L.perm.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice));
        ALLOC(g->deg64, sizeof(double) * n);
        ALLOC(g->inv_deg64, sizeof(double) * n);
        ALLOC(g->deg32, sizeof(float) * n);
        ALLOC(g->inv_deg32, sizeof(float) * n);
        ALLOC(g->inv2_deg64, sizeof(double) * n);
        ALLOC(g->inv2_deg32, sizeof(float) * n);
        ALLOC(g->deg_df, sizeof(df) * n);
        ALLOC(g->inv_deg_df, sizeof(df) * n);
        ALLOC(g->inv2_deg_df, sizeof(df) * n);
        ALLOC(g->deg16, sizeof(uint16_t) * n);
        vertex_arrays_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 8192), 256>>>(
            d_rp, g->perm, n, g->deg64, g->inv_deg64, g->inv2_deg64, g->deg32, g->inv_deg32, g->inv2_deg32,
            g->deg_df, g->inv_deg_df, g->inv2_deg_df, g->deg16, d_inv);
        CK(cudaGetLastError());
        {
            // the same factors by degree for the short chunks' rows, by the
            // same expressions (IEEE division and conversions give the same
            // bits on host and device)
            int dmax = 0;
            for (int64_t u = 0; u < n; ++u) dmax = std::max(dmax, hrp[u + 1] - hrp[u]);
            g->dmax = dmax;
            const int T = std::min(std::min(dmax, lp.hub_degree), std::min(lp.long_chunk, kMaxShortRow)) + 1;
            std::vector<double> t64(3 * (size_t)T, 0.0);
            std::vector<float> t32(3 * (size_t)T, 0.0f);
            std::vector<df> tdf(3 * (size_t)T, df(0.0));
            for (int d = 1; d < T; ++d) {
                t64[d] = (double)d;
                t64[T + d] = 1.0 / (double)d;
                t64[2 * T + d] = 2.0 / (double)d;
                t32[d] = (float)d;
                t32[T + d] = 1.0f / (float)d;
                t32[2 * T + d] = 2.0f / (float)d;
                tdf[d] = df((double)d);
                tdf[T + d] = df(1.0 / (double)d);
                tdf[2 * T + d] = df(2.0 / (double)d);
            }
            ALLOC(g->tab64, sizeof(double) * 3 * T);
            ALLOC(g->tab32, sizeof(float) * 3 * T);
            ALLOC(g->tab_df, sizeof(df) * 3 * T);
            CK(cudaMemcpy(g->tab64, t64.data(), sizeof(double) * 3 * T, cudaMemcpyHostToDevice));
            CK(cudaMemcpy(g->tab32, t32.data(), sizeof(float) * 3 * T, cudaMemcpyHostToDevice));
            CK(cudaMemcpy(g->tab_df, tdf.data(), sizeof(df) * 3 * T, cudaMemcpyHostToDevice));
            g->tab_n = T;
        }

        // the relabelled graph's CSR: every caller row's entries in new ids,
        // sorted ascending (the order in which the round adds them)
        relabel_kernel<<<(unsigned)std::min<int64_t>((nnz + 255) / 256, 16384), 256>>>(d_ci, d_inv, n, nnz,
                                                                                      d_bad + 3);
        CK(cudaGetLastError());
        {
            unsigned long long nbad = 0;
            CK(cudaMemcpy(&nbad, d_bad + 3, sizeof(nbad), cudaMemcpyDeviceToHost));
            if (nbad) {
                st = fail(CPAA_EINVAL, "invalid CSR: " + std::to_string(nbad) + " column(s) out of range [0, n)");
                goto fail_out;
            }
        }
        dev_free(g, (void **)&d_bad, 4 * sizeof(unsigned long long));
        CK(cub::DeviceSegmentedSort::SortKeys(nullptr, tmp_bytes, d_ci, d_rs, nnz, n, d_rp, d_rp + 1));
        ALLOC(d_tmp, std::max<size_t>(tmp_bytes, 16));
        ALLOC(d_rs, ci_bytes);
        CK(cub::DeviceSegmentedSort::SortKeys(d_tmp, tmp_bytes, d_ci, d_rs, nnz, n, d_rp, d_rp + 1));
        dev_free(g, &d_tmp, std::max<size_t>(tmp_bytes, 16));
        dev_free(g, (void **)&d_ci, ci_bytes);
        d_ci = d_rs;
        d_rs = nullptr;

        ALLOC(d_loops, sizeof(unsigned long long));
        CK(cudaMemset(d_loops, 0, sizeof(unsigned long long)));
        ALLOC(g->hub_row_ptr, sizeof(int32_t) * (L.n_hub + 1));
        CK(cudaMemcpy(g->hub_row_ptr, L.hub_row_ptr.data(), sizeof(int32_t) * (L.n_hub + 1),
                      cudaMemcpyHostToDevice));
        ALLOC(g->hub_col, sizeof(int32_t) * (g->hub_nnz + 4));
        CK(cudaMemset(g->hub_col, 0, sizeof(int32_t) * (g->hub_nnz + 4)));
        if (L.n_hub > 0) {
            build_hub_kernel<<<std::min(L.n_hub, 4096), 256>>>(d_rp, d_ci, g->perm, g->hub_row_ptr, L.n_hub,
                                                                g->hub_col, d_loops);
            CK(cudaGetLastError());
        }
        ALLOC(g->hub_tiles, sizeof(int4) * std::max<size_t>(1, L.hub_tiles.size()));
        if (!L.hub_tiles.empty())
            CK(cudaMemcpy(g->hub_tiles, L.hub_tiles.data(), sizeof(int4) * L.hub_tiles.size(),
                          cudaMemcpyHostToDevice));
        ALLOC(g->long_cnt, sizeof(int) * std::max(1, g->n_hub));
        CK(cudaMemset(g->long_cnt, 0, sizeof(int) * std::max(1, g->n_hub)));

        const int nch = std::max(1, g->num_chunks);
        ALLOC(g->chunk_off, sizeof(int64_t) * nch);
        ALLOC(g->chunk_len, sizeof(int32_t) * nch);
        ALLOC(g->chunk_order, sizeof(int32_t) * nch);
        ALLOC(g->chunk_desc, sizeof(int4) * nch);
        ALLOC(g->sell_col, sizeof(int32_t) * std::max<int64_t>(4, g->sell_entries));
        if (g->num_chunks > 0) {
            CK(cudaMemcpy(g->chunk_off, L.chunk_off.data(), sizeof(int64_t) * g->num_chunks, cudaMemcpyHostToDevice));
            CK(cudaMemcpy(g->chunk_len, L.chunk_len.data(), sizeof(int32_t) * g->num_chunks, cudaMemcpyHostToDevice));
            CK(cudaMemcpy(g->chunk_order, L.chunk_order.data(), sizeof(int32_t) * g->num_chunks,
                          cudaMemcpyHostToDevice));
            CK(cudaMemcpy(g->chunk_desc, L.chunk_desc.data(), sizeof(int4) * g->num_chunks,
                          cudaMemcpyHostToDevice));
            build_sell_kernel<<<(unsigned)std::min<int64_t>(((int64_t)g->num_chunks * 32 + 255) / 256, 16384), 256>>>(
                d_rp, d_ci, g->perm, n, L.n_hub, g->num_chunks, g->chunk_off, g->chunk_len, g->sell_col, d_loops);
            CK(cudaGetLastError());
        }
        CK(cudaDeviceSynchronize());
        {
            unsigned long long nl = 0;
            CK(cudaMemcpy(&nl, d_loops, sizeof(nl), cudaMemcpyDeviceToHost));
            g->loops_all = (int64_t)nl == n;
        }
        dev_free(g, (void **)&d_loops, sizeof(unsigned long long));
        dev_free(g, (void **)&d_inv, sizeof(int32_t) * n);
        dev_free(g, (void **)&d_ci, ci_bytes);
        dev_free(g, (void **)&d_rp, rp_bytes);
        *out = g;
        return CPAA_OK;
    }
fail_out:
    if (d_bad) dev_free(g, (void **)&d_bad, 4 * sizeof(unsigned long long));
    if (d_loops) dev_free(g, (void **)&d_loops, sizeof(unsigned long long));
    if (d_tmp) dev_free(g, &d_tmp, std::max<size_t>(tmp_bytes, 16));
    if (d_rs) dev_free(g, (void **)&d_rs, ci_bytes);
    if (d_inv) dev_free(g, (void **)&d_inv, sizeof(int32_t) * n);
    if (d_ci) dev_free(g, (void **)&d_ci, ci_bytes);
    if (d_rp) dev_free(g, (void **)&d_rp, rp_bytes);
    release(g);
    return st;
#undef ALLOC
#undef CK
}

// ---------------------------------------------------------------------------
// Autotuning of the layout parameters (CPAA_GRAPH_AUTOTUNE).
//
// Coordinate search from the starting parameters: the sort window, then the
// hub threshold, the hub tile and the long-chunk threshold, each over a few
// candidates around the current best; every candidate layout is built and
// kTuneLayoutRounds single-vector rounds of uniform p are timed on it (CUDA
// events, the second of two runs).  Candidates that give the same layout as
// one already timed (same hub rows, hub tiles, long chunks and window) are
// not timed again.  The pick is cached for the process, keyed by device,
// size, a log2 histogram of the degrees, the timing precision and the start.
constexpr int kTuneLayoutRounds = 4;

struct TuneKey {
    int device, precision;
    int64_t n, nnz;
    std::vector<int64_t> hist;
    LayoutParams start;
    bool operator==(const TuneKey &o) const {
        return device == o.device && precision == o.precision && n == o.n && nnz == o.nnz && hist == o.hist &&
               start.hub_degree == o.start.hub_degree && start.hub_tile == o.start.hub_tile &&
               start.long_chunk == o.start.long_chunk && start.sort_window == o.start.sort_window;
    }
};
static std::mutex g_tune_mu;
static std::vector<std::pair<TuneKey, std::pair<LayoutParams, int>>> g_tune_cache;

// Device time per round of kTuneLayoutRounds rounds on graph g (uniform p).
static cpaa_status time_layout(cpaa_graph *g, int prec, const double *d_p, double *d_pi, float *ms_per_round) {
    cpaa_status s = ensure_workspace(g, prec, 1, kTuneLayoutRounds);
    if (s != CPAA_OK) return s;
    TileJob job;
    job.width = 1;
    job.precision = prec;
    job.p[0] = d_p;
    job.pi[0] = d_pi;
    job.c[0] = 0.85;
    std::vector<double> ck;
    cheb_coeffs(0.85, 0, ck);
    job.c0half[0] = ck[0] / 2.0;
    job.rounds[0] = kTuneLayoutRounds;
    float ms = 0.0f;
    for (int rep = 0; rep < 2; ++rep) {  // the first run also captures the round graph
        if ((s = run_tile(g, job, nullptr, false, true)) != CPAA_OK) return s;
        if ((s = tile_rounds_ms(g, &ms)) != CPAA_OK) return s;
    }
    CPAA_CUDA(cudaDeviceSynchronize());
    *ms_per_round = ms / kTuneLayoutRounds;
    return CPAA_OK;
}

static cpaa_status autotune_graph(int64_t n, int64_t nnz, const int32_t *row_ptr, const int32_t *col_idx,
                                  unsigned flags, const std::vector<int32_t> &hrp, const LayoutParams &start,
                                  int prec, cpaa_graph **out) {
    TuneKey key;
    cudaGetDevice(&key.device);
    key.precision = prec;
    key.n = n;
    key.nnz = nnz;
    key.hist.assign(32, 0);
    int maxdeg = 0;
    for (int64_t u = 0; u < n; ++u) {
        const int d = hrp[u + 1] - hrp[u];
        maxdeg = std::max(maxdeg, d);
        int b = 0;
        while ((2 << b) <= d && b < 31) ++b;
        ++key.hist[b];
    }
    key.start = start;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        for (auto &e : g_tune_cache)
            if (e.first == key) {
                cpaa_status s = build_graph(n, nnz, row_ptr, col_idx, flags, hrp, e.second.first, out);
                if (s == CPAA_OK) {
                    (*out)->tuned = 1;
                    (*out)->tune_candidates = e.second.second;
                }
                return s;
            }
    }
    // uniform p and a scratch output for the timed rounds
    double *d_p = nullptr, *d_pi = nullptr;
    CPAA_CUDA(cudaMalloc(&d_p, sizeof(double) * n));
    if (cudaMalloc(&d_pi, sizeof(double) * n) != cudaSuccess) {
        cudaFree(d_p);
        return fail(CPAA_ENOMEM, "autotune: no room for its test vectors");
    }
    {
        std::vector<double> hp((size_t)n, 1.0 / (double)n);
        cudaMemcpy(d_p, hp.data(), sizeof(double) * n, cudaMemcpyHostToDevice);
    }
    struct Timed {
        LayoutParams lp;
        int64_t sig[4];
        float ms;
    };
    std::vector<Timed> timed;
    cpaa_graph *best = nullptr;
    float best_ms = 0.0f;
    LayoutParams best_lp = start;
    cpaa_status st = CPAA_OK;
    unsigned cand_flags = flags | CPAA_GRAPH_TRUSTED;  // checked once, by the first build
    auto eval = [&](const LayoutParams &lp) -> cpaa_status {
        cpaa_graph *g = nullptr;
        cpaa_status s = build_graph(n, nnz, row_ptr, col_idx, timed.empty() && !best ? flags : cand_flags, hrp,
                                    lp, &g);
        if (s != CPAA_OK) return s;
        const int64_t sig[4] = {g->n_hub, g->num_hub_tiles, g->num_long_chunks, lp.sort_window};
        float ms = -1.0f;
        for (auto &t : timed)
            if (std::equal(sig, sig + 4, t.sig)) ms = t.ms;
        const bool fresh = ms < 0.0f;
        if (fresh) {
            s = time_layout(g, prec, d_p, d_pi, &ms);
            if (s != CPAA_OK) {
                release(g);
                return s;
            }
            Timed t;
            t.lp = lp;
            std::copy(sig, sig + 4, t.sig);
            t.ms = ms;
            timed.push_back(t);
        }
        if (!best || ms < best_ms) {
            if (best) release(best);
            best = g;
            best_ms = ms;
            best_lp = lp;
        } else {
            release(g);
        }
        return CPAA_OK;
    };
    st = eval(start);
    // the sort window
    for (int w : {64, 256, 1024, 4096})
        if (st == CPAA_OK && w != best_lp.sort_window) {
            LayoutParams lp = best_lp;
            lp.sort_window = w;
            st = eval(lp);
        }
    // the hub threshold (only thresholds some row exceeds make hub rows)
    const LayoutParams after_window = best_lp;
    for (int f : {-2, -1, 1})
        if (st == CPAA_OK) {
            LayoutParams lp = after_window;
            lp.hub_degree = f < 0 ? after_window.hub_degree >> (-f) : after_window.hub_degree << f;
            if (lp.hub_degree < 32 || lp.hub_degree >= maxdeg) continue;
            lp.hub_tile = std::min(16384, std::max(512, 2 * lp.hub_degree));
            st = eval(lp);
        }
    // the hub tile (only with hub rows)
    const LayoutParams after_hub = best_lp;
    if (best && best->n_hub > 0)
        for (int f : {-1, 1})
            if (st == CPAA_OK) {
                LayoutParams lp = after_hub;
                lp.hub_tile = f < 0 ? after_hub.hub_tile / 2 : after_hub.hub_tile * 2;
                if (lp.hub_tile < 256 || lp.hub_tile > 32768) continue;
                st = eval(lp);
            }
    // the long-chunk threshold
    const LayoutParams after_tile = best_lp;
    for (int lc : {8, 16, 32, 64})
        if (st == CPAA_OK && lc != after_tile.long_chunk && lc < std::min(maxdeg, after_tile.hub_degree)) {
            LayoutParams lp = after_tile;
            lp.long_chunk = lc;
            st = eval(lp);
        }
    cudaFree(d_p);
    cudaFree(d_pi);
    if (st != CPAA_OK) {
        if (best) release(best);
        return st;
    }
    best->tuned = 1;
    best->tune_candidates = (int)timed.size();
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache.push_back({key, {best_lp, (int)timed.size()}});
    }
    *out = best;
    return CPAA_OK;
}

}  // namespace cpaa

using namespace cpaa;

extern "C" cpaa_status cpaa_graph_create_ex(int64_t n, int64_t nnz, const int32_t *row_ptr,
                                            const int32_t *col_idx, unsigned flags,
                                            const cpaa_layout_params *params, cpaa_graph **out) {
    clear_error();
    if (!out) return fail(CPAA_EINVAL, "out is NULL");
    *out = nullptr;
    if (n < 1 || n >= (int64_t(1) << 31) - 1) return fail(CPAA_EINVAL, "n out of range [1, 2^31 - 1)");
    if (nnz < 1 || nnz >= (int64_t(1) << 31)) return fail(CPAA_EINVAL, "nnz out of range [1, 2^31)");
    if (!row_ptr || !col_idx) return fail(CPAA_EINVAL, "row_ptr / col_idx is NULL");
    const bool dev_in = (flags & CPAA_GRAPH_DEVICE_INPUT) != 0;
    LayoutParams lp;
    cpaa_status s = resolve_layout(params, nnz, &lp);
    if (s != CPAA_OK) return s;
    int tune_prec = params ? params->tune_precision : CPAA_F64;
    if (tune_prec != CPAA_F64 && tune_prec != CPAA_F32 && tune_prec != CPAA_BF16 && tune_prec != CPAA_DF64)
        return fail(CPAA_EINVAL, "layout tune_precision is not a cpaa_precision");

    // Host copy of row_ptr: the layout is planned on the host.
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
    if (flags & CPAA_GRAPH_AUTOTUNE) return autotune_graph(n, nnz, row_ptr, col_idx, flags, hrp, lp, tune_prec, out);
    return build_graph(n, nnz, row_ptr, col_idx, flags, hrp, lp, out);
}

extern "C" cpaa_status cpaa_graph_create(int64_t n, int64_t nnz, const int32_t *row_ptr,
                                         const int32_t *col_idx, unsigned flags, cpaa_graph **out) {
    return cpaa_graph_create_ex(n, nnz, row_ptr, col_idx, flags, nullptr, out);
}

extern "C" cpaa_status cpaa_graph_destroy(cpaa_graph *g) {
    clear_error();
    if (!g) return CPAA_OK;
    cudaDeviceSynchronize();
    release(g);
    return CPAA_OK;
}

extern "C" cpaa_status cpaa_graph_layout(const cpaa_graph *g, cpaa_layout *out) {
    clear_error();
    if (!g || !out) return fail(CPAA_EINVAL, "graph or out is NULL");
    out->hub_rows = g->n_hub;
    out->hub_entries = g->hub_nnz;
    out->hub_tiles = g->num_hub_tiles;
    out->chunks = g->num_chunks;
    out->long_chunks = g->num_long_chunks;
    out->sell_entries = g->sell_entries;
    out->hub_degree = g->hub_degree;
    out->hub_tile = g->hub_tile;
    out->long_chunk = g->lp.long_chunk;
    out->sort_window = g->lp.sort_window;
    out->tuned = g->tuned;
    out->tune_candidates = g->tune_candidates;
    return CPAA_OK;
}

namespace cpaa {
// Every vertex with a self-loop makes D' + A' (the loop-free degree and
// adjacency matrices) positive semidefinite, so A + D >= 2I and
// D^-1/2 A D^-1/2 + I >= 2 D^-1 >= (2 / d_max) I.
double graph_lambda_lo(const cpaa_graph *g) {
    return g->loops_all && g->dmax > 0 ? -1.0 + 2.0 / (double)g->dmax : -1.0;
}
}  // namespace cpaa

extern "C" cpaa_status cpaa_graph_spectrum_bound(const cpaa_graph *g, double *lambda_lo) {
    clear_error();
    if (!g || !lambda_lo) return fail(CPAA_EINVAL, "graph or lambda_lo is NULL");
    *lambda_lo = graph_lambda_lo(g);
    return CPAA_OK;
}

extern "C" cpaa_status cpaa_graph_info(const cpaa_graph *g, int64_t *n, int64_t *nnz,
                                       int64_t *device_bytes, int64_t *num_tiles) {
    clear_error();
    if (!g) return fail(CPAA_EINVAL, "graph is NULL");
    if (n) *n = g->n;
    if (nnz) *nnz = g->nnz;
    if (device_bytes) *device_bytes = g->device_bytes;
    if (num_tiles) *num_tiles = (int64_t)g->num_hub_tiles + g->num_chunks;
    return CPAA_OK;
}
