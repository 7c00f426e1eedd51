// frontier.cu -- sparse-frontier early rounds (CPAA_SPARSE_FRONTIER).
//
// A personalised vector p with a few seeds makes T_0 p = p zero outside the
// seeds, and T_{k+1} p = 2 P T_k p - T_{k-1} p (Sec. 4.1) is zero outside the
// closed neighbourhood of the support of T_k p: after k rounds the iterates
// live on the k-hop ball of the seeds.  A full round over every row computes
// exact zeros outside it (0 + ... + 0, times 2/d, minus 0), so a round may
// skip every work item (hub tile, SELL chunk) none of whose rows is in the
// ball and still leave every value bit-identical.
//
// The ball is kept as bitmaps over the rows (internal.h, Frontier): `cur`
// holds every row that may be nonzero, `ring` the rows added last time, `add`
// the neighbours marked by the current expansion.  Before each early round
//   frontier_mark_kernel    marks the neighbours of the ring rows in add;
//   frontier_update_kernel  cur |= add, ring = the new rows, add = 0, and
//                           counts the stored entries of the items cur covers;
// then the round kernel (step.cu) skips the items with no bit in cur, unless
// the covered entries passed nnz / kFrontierLimitDiv, from which round on
// (sticky flag) every round runs over every item and the two kernels above
// return at once.  Rows only ever join the ball, so an item's partial-sum
// slot is either written in a round or still zero from the reset.
#include <algorithm>

#include "device_common.cuh"

namespace cpaa {

constexpr int kFrThreads = 256;

struct FrontierArgs {
    unsigned *cur, *ring, *add;
    int *full;
    unsigned long long *entries;
    int64_t words;
    int hub_words;
    int64_t n;
    int n_hub;
    int num_hub_tiles, hub_tile, num_chunks;
    const int4 *hub_tiles;
    const int32_t *hub_row_ptr, *hub_col;
    const int32_t *sell_col;
    const int64_t *chunk_off;
    const int32_t *chunk_len;
    const float *deg32;
};

// Word and bit of row r in the frontier bitmaps.
__device__ __forceinline__ void fr_pos(const FrontierArgs &a, int64_t r, int64_t &w, unsigned &bit) {
    if (r < a.n_hub) {
        w = r >> 5;
        bit = 1u << (r & 31);
    } else {
        const int64_t q = r - a.n_hub;
        w = a.hub_words + (q >> 5);
        bit = 1u << (q & 31);
    }
}

__device__ __forceinline__ void fr_mark(const FrontierArgs &a, int32_t j) {
    if (j < 0 || j >= a.n) return;  // the padding sentinel n
    int64_t w;
    unsigned bit;
    fr_pos(a, j, w, bit);
    if (!(a.cur[w] & bit) && !(a.add[w] & bit)) atomicOr(a.add + w, bit);
}

// Neighbours of the ring rows into add: hub rows one CTA per hub tile, SELL
// rows one warp per chunk word, the warp's lanes over each marked row's
// entries in turn.
__global__ void __launch_bounds__(kFrThreads) frontier_mark_kernel(const FrontierArgs a) {
    if (*a.full) return;
    for (int t = blockIdx.x; t < a.num_hub_tiles; t += gridDim.x) {
        const int4 ti = a.hub_tiles[t];
        const int h = ti.x;
        if (!(a.ring[h >> 5] >> (h & 31) & 1u)) continue;  // the same for the whole CTA
        const int e0 = a.hub_row_ptr[h], e1 = a.hub_row_ptr[h + 1];
        const int c0 = e0 + ti.y * a.hub_tile, c1 = min(c0 + a.hub_tile, e1);
        for (int e = c0 + (int)threadIdx.x; e < c1; e += kFrThreads) fr_mark(a, a.hub_col[e]);
    }
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * kFrThreads) >> 5;
    for (int64_t c = ((int64_t)blockIdx.x * kFrThreads + threadIdx.x) >> 5; c < a.num_chunks; c += nwarps) {
        unsigned w = a.ring[a.hub_words + c];
        if (w == 0) continue;
        const int32_t *col = a.sell_col + a.chunk_off[c];
        while (w) {
            const int l = __ffs(w) - 1;
            w &= w - 1;
            const int64_t r = a.n_hub + c * kChunkRows + l;
            const int d = (int)a.deg32[r];
            for (int i = lane; i < d; i += 32) fr_mark(a, col[(int64_t)(i >> 2) * (kChunkRows * kSellVec) + 4 * l + (i & 3)]);
        }
    }
}

// cur |= add, ring = add & ~cur, add = 0, and the stored entries of the items
// cur now covers into entries[parity] (entries[parity ^ 1] is cleared for the
// next update).
__global__ void __launch_bounds__(kFrThreads) frontier_update_kernel(const FrontierArgs a, int parity) {
    if (*a.full) return;
    unsigned long long ent = 0;
    for (int64_t w = blockIdx.x * (int64_t)kFrThreads + threadIdx.x; w < a.words;
         w += (int64_t)gridDim.x * kFrThreads) {
        const unsigned c = a.cur[w], ad = a.add[w];
        a.ring[w] = ad & ~c;
        const unsigned nw = c | ad;
        if (ad) {
            a.cur[w] = nw;
            a.add[w] = 0;
        }
        if (!nw) continue;
        if (w < a.hub_words) {
            unsigned m = nw;
            while (m) {
                const int h = (int)(w << 5) + __ffs(m) - 1;
                m &= m - 1;
                if (h < a.n_hub) ent += (unsigned long long)(a.hub_row_ptr[h + 1] - a.hub_row_ptr[h]);
            }
        } else {
            ent += (unsigned long long)a.chunk_len[w - a.hub_words] * kChunkRows;
        }
    }
    for (int o = 16; o > 0; o >>= 1) ent += __shfl_xor_sync(0xffffffffu, ent, o);
    if ((threadIdx.x & 31) == 0 && ent) atomicAdd(a.entries + parity, ent);
    if (blockIdx.x == 0 && threadIdx.x == 0) a.entries[parity ^ 1] = 0;
}

// Whether a stored value is anything but +0 (a -0 counts as nonzero: rows
// outside the ball must hold exactly the +0 a full round would give them).
__device__ __forceinline__ bool not_pos_zero(double v) { return __double_as_longlong(v) != 0; }
__device__ __forceinline__ bool not_pos_zero(float v) { return __float_as_uint(v) != 0u; }
__device__ __forceinline__ bool not_pos_zero(__nv_bfloat16 v) { return __bfloat16_as_ushort(v) != 0; }
__device__ __forceinline__ bool not_pos_zero(df v) { return not_pos_zero(v.hi) || not_pos_zero(v.lo); }

// Rows where any of the W columns of y0 is not +0 join cur and ring.
template <class S, int W>
__global__ void __launch_bounds__(kFrThreads) frontier_nonzero_kernel(const FrontierArgs a, const S *__restrict__ y0) {
    for (int64_t r = blockIdx.x * (int64_t)kFrThreads + threadIdx.x; r < a.n;
         r += (int64_t)gridDim.x * kFrThreads) {
        bool nz = false;
#pragma unroll
        for (int b = 0; b < W; ++b) nz |= not_pos_zero(y0[r * W + b]);
        if (nz) {
            int64_t w;
            unsigned bit;
            fr_pos(a, r, w, bit);
            atomicOr(a.cur + w, bit);
            atomicOr(a.ring + w, bit);
        }
    }
}

struct FrontierRows {
    int count;
    int32_t r[kMaxFrontierSeeds];
};

__global__ void frontier_rows_kernel(const FrontierArgs a, const FrontierRows rows) {
    const int i = threadIdx.x;
    if (i < rows.count) {
        int64_t w;
        unsigned bit;
        fr_pos(a, rows.r[i], w, bit);
        atomicOr(a.cur + w, bit);
        atomicOr(a.ring + w, bit);
    }
}

static FrontierArgs args_of(const cpaa_graph *g, const Frontier &f) {
    FrontierArgs a;
    a.cur = f.cur;
    a.ring = f.ring;
    a.add = f.add;
    a.full = f.full;
    a.entries = f.entries;
    a.words = f.words;
    a.hub_words = f.hub_words;
    a.n = g->n;
    a.n_hub = g->n_hub;
    a.num_hub_tiles = g->num_hub_tiles;
    a.hub_tile = g->hub_tile;
    a.num_chunks = g->num_chunks;
    a.hub_tiles = g->hub_tiles;
    a.hub_row_ptr = g->hub_row_ptr;
    a.hub_col = g->hub_col;
    a.sell_col = g->sell_col;
    a.chunk_off = g->chunk_off;
    a.chunk_len = g->chunk_len;
    a.deg32 = g->deg32;
    return a;
}

static int fr_blocks(int64_t units) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((units + kFrThreads - 1) / kFrThreads, 2048));
}

size_t frontier_bytes(const cpaa_graph *g) {
    const int64_t words = (int64_t)((g->n_hub + 31) / 32) + g->num_chunks;
    return 3 * sizeof(unsigned) * (size_t)std::max<int64_t>(1, words) + 64;
}

cpaa_status ensure_frontier(const cpaa_graph *g, Frontier &f, cpaa_graph *track) {
    if (f.cur) return CPAA_OK;
    f.hub_words = (g->n_hub + 31) / 32;
    f.words = (int64_t)f.hub_words + g->num_chunks;
    const size_t wb = sizeof(unsigned) * (size_t)std::max<int64_t>(1, f.words);
    cpaa_status s;
    if ((s = dev_alloc(track, (void **)&f.cur, wb)) != CPAA_OK) return s;
    if ((s = dev_alloc(track, (void **)&f.ring, wb)) != CPAA_OK) return s;
    if ((s = dev_alloc(track, (void **)&f.add, wb)) != CPAA_OK) return s;
    if ((s = dev_alloc(track, (void **)&f.full, 64)) != CPAA_OK) return s;
    f.entries = reinterpret_cast<unsigned long long *>(reinterpret_cast<char *>(f.full) + 16);
    return CPAA_OK;
}

void free_frontier(cpaa_graph *track, Frontier &f) {
    const size_t wb = sizeof(unsigned) * (size_t)std::max<int64_t>(1, f.words);
    dev_free(track, (void **)&f.cur, wb);
    dev_free(track, (void **)&f.ring, wb);
    dev_free(track, (void **)&f.add, wb);
    dev_free(track, (void **)&f.full, 64);
    f.entries = nullptr;
}

cudaError_t frontier_reset(const Frontier &f, cudaStream_t st) {
    const size_t wb = sizeof(unsigned) * (size_t)std::max<int64_t>(1, f.words);
    cudaError_t e;
    if ((e = cudaMemsetAsync(f.cur, 0, wb, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(f.ring, 0, wb, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(f.add, 0, wb, st)) != cudaSuccess) return e;
    return cudaMemsetAsync(f.full, 0, 64, st);
}

// y1, the other iterate buffer, is cleared to +0: early rounds leave the rows
// outside the ball untouched, and later rounds gather them.
template <class S>
static cudaError_t nonzero_w(const FrontierArgs &a, int width, const void *y0, void *y1, cudaStream_t st) {
    const cudaError_t e = cudaMemsetAsync(y1, 0, sizeof(S) * (size_t)(a.n + 1) * width, st);
    if (e != cudaSuccess) return e;
    const int nb = fr_blocks(a.n);
    switch (width) {
        case 1: frontier_nonzero_kernel<S, 1><<<nb, kFrThreads, 0, st>>>(a, (const S *)y0); break;
        case 2: frontier_nonzero_kernel<S, 2><<<nb, kFrThreads, 0, st>>>(a, (const S *)y0); break;
        case 4: frontier_nonzero_kernel<S, 4><<<nb, kFrThreads, 0, st>>>(a, (const S *)y0); break;
        case 8: frontier_nonzero_kernel<S, 8><<<nb, kFrThreads, 0, st>>>(a, (const S *)y0); break;
        case 16: frontier_nonzero_kernel<S, 16><<<nb, kFrThreads, 0, st>>>(a, (const S *)y0); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t frontier_mark_nonzero(const cpaa_graph *g, const Frontier &f, int precision, int width,
                                  const void *y0, void *y1, cudaStream_t st) {
    const FrontierArgs a = args_of(g, f);
    switch (precision) {
        case CPAA_F64: return nonzero_w<double>(a, width, y0, y1, st);
        case CPAA_F32: return nonzero_w<float>(a, width, y0, y1, st);
        case CPAA_BF16: return nonzero_w<__nv_bfloat16>(a, width, y0, y1, st);
        case CPAA_DF64: return nonzero_w<df>(a, width, y0, y1, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t frontier_mark_rows(const cpaa_graph *g, const Frontier &f, int count, const int32_t *rows,
                               cudaStream_t st) {
    if (count < 0 || count > kMaxFrontierSeeds) return cudaErrorInvalidValue;
    FrontierRows fr;
    fr.count = count;
    for (int i = 0; i < count; ++i) fr.r[i] = rows[i];
    frontier_rows_kernel<<<1, kMaxFrontierSeeds, 0, st>>>(args_of(g, f), fr);
    return cudaGetLastError();
}

cudaError_t frontier_expand(const cpaa_graph *g, const Frontier &f, int parity, cudaStream_t st) {
    const FrontierArgs a = args_of(g, f);
    const int mb = (int)std::max<int64_t>(
        1, std::min<int64_t>(2048, std::max<int64_t>(g->num_hub_tiles, (int64_t)g->num_chunks * 32 / kFrThreads)));
    frontier_mark_kernel<<<mb, kFrThreads, 0, st>>>(a);
    frontier_update_kernel<<<fr_blocks(f.words), kFrThreads, 0, st>>>(a, parity & 1);
    return cudaGetLastError();
}

void frontier_launch(const cpaa_graph *g, const Frontier &f, int parity, StepLaunch &sl) {
    sl.front = f.cur;
    sl.front_full = f.full;
    sl.front_entries = f.entries + (parity & 1);
    sl.front_limit = (unsigned long long)(g->nnz / kFrontierLimitDiv);
    sl.front_hub_words = f.hub_words;
}

}  // namespace cpaa
