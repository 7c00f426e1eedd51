// step.cu -- one round of the Chebyshev recurrence, fused with the
// accumulation and the per-round reductions (Algorithm 1, Sec. 4.1).
//
// Scaled space.  The kernels keep y_k = D^-1 T_k p instead of T_k p.  Then
//     (P T_k)[u] = sum_{j in N(u)} T_k[j] / d_j = sum_{j in N(u)} y_k[j],
// so the gather is a plain sum of neighbour values with no degree lookup, and
//     y_1[u]     = (1/d_u) sum_{j in N(u)} y_0[j]                  (k = 1)
//     y_{k+1}[u] = (2/d_u) sum_{j in N(u)} y_k[j] - y_{k-1}[u]     (k >= 1)
// which is T_{k+1} = 2 P T_k - T_{k-1} (Chebyshev property (3), Sec. 2.2)
// divided by d_u.  The accumulator is rho = D^-1 pibar, rho += c_k y_k, and
// the finalisation multiplies by d_u again.  y_{k+1} overwrites y_{k-1} in
// place: row u is the only reader of y_{k-1}[u].
//
// Per-round reductions (the mass view of Sec. 4.1): sum_u T_k[u] and
// sum_u |T_k[u]|.  Each CTA adds its values into one of kRedSlots FP64 slots
// (diagnostics only: the slot atomics are not ordered).
//
// Work split.  See internal.h: block tiles of whole rows, walked by a merge
// path inside the CTA (every thread gets kItemsPerThread consecutive items of
// the rows+entries sequence), and chunk tiles of long rows combined by the
// CTA holding the last ticket.  Each sum runs in a fixed order, so results
// are the same from run to run.
#include "internal.h"

namespace cpaa {

template <int P> struct Prec;
template <> struct Prec<CPAA_F64> {
    using S = double;  // storage of y
    using A = double;  // arithmetic
    using R = double;  // accumulator rho
    static constexpr bool kKahan = false;
};
template <> struct Prec<CPAA_F32> {
    using S = float;
    using A = float;
    using R = float;
    static constexpr bool kKahan = true;
};
template <> struct Prec<CPAA_BF16> {
    using S = __nv_bfloat16;
    using A = float;
    using R = float;
    static constexpr bool kKahan = true;
};

__device__ __forceinline__ double load_y(const double *p) { return __ldg(p); }
__device__ __forceinline__ float load_y(const float *p) { return __ldg(p); }
__device__ __forceinline__ float load_y(const __nv_bfloat16 *p) { return __bfloat162float(__ldg(p)); }

__device__ __forceinline__ double to_acc(double v) { return v; }
__device__ __forceinline__ float to_acc(float v) { return v; }
__device__ __forceinline__ float to_acc(__nv_bfloat16 v) { return __bfloat162float(v); }

template <class S> __device__ __forceinline__ S to_store(double v);
template <> __device__ __forceinline__ double to_store<double>(double v) { return v; }
template <class S> __device__ __forceinline__ S to_store_f(float v);
template <> __device__ __forceinline__ float to_store_f<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 to_store_f<__nv_bfloat16>(float v) {
    return __float2bfloat16_rn(v);
}
__device__ __forceinline__ void store_y(double *p, double v) { *p = v; }
__device__ __forceinline__ void store_y(float *p, float v) { *p = v; }
__device__ __forceinline__ void store_y(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }

// Streaming 16-byte load of four column indices (read once per round).
__device__ __forceinline__ int4 load_cols(const int32_t *p) { return __ldcs(reinterpret_cast<const int4 *>(p)); }

template <int P>
struct StepParams {
    using S = typename Prec<P>::S;
    using A = typename Prec<P>::A;
    using R = typename Prec<P>::R;
    const int4 *tiles;
    const int32_t *row_ptr;
    const int32_t *col_idx;
    const A *deg;
    const A *inv_deg;
    const S *y_src;
    S *y_io;
    R *rho;
    R *comp;
    A *long_part;
    int *long_cnt;
    double *red;
    A ck;
    int first;
    int last;
};

// Row epilogue: recurrence, accumulation, and this row's reduction terms.
template <int P>
__device__ __forceinline__ void row_update(const StepParams<P> &p, int u, typename Prec<P>::A s,
                                           typename Prec<P>::A &sT, typename Prec<P>::A &sA,
                                           double &sR) {
    using A = typename Prec<P>::A;
    using R = typename Prec<P>::R;
    const A inv = p.inv_deg[u];
    A y;
    if (p.first) y = s * inv;
    else y = (s + s) * inv - to_acc(p.y_io[u]);
    store_y(p.y_io + u, y);
    const A yq = to_acc(p.y_io[u]);  // the value later rounds will read
    R r = p.rho[u];
    if constexpr (Prec<P>::kKahan) {
        R cmp = p.comp[u];
        const R t1 = p.ck * yq - cmp;
        const R t = r + t1;
        cmp = (t - r) - t1;
        r = t;
        p.comp[u] = cmp;
    } else {
        r = r + p.ck * yq;
    }
    p.rho[u] = r;
    const A d = p.deg[u];
    const A T = yq * d;
    sT += T;
    sA += (T < A(0) ? -T : T);
    if (p.last) sR += (double)r * (double)d;
}

// Reduce three per-thread values over the CTA and add them to this round's
// slots.  Deterministic within the CTA; the slot atomics are not ordered.
__device__ __forceinline__ void cta_reduce_add(double a, double b, double c, double *red) {
    __shared__ double s_red[kThreads / 32][3];
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { s_red[w][0] = a; s_red[w][1] = b; s_red[w][2] = c; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = 0, y = 0, z = 0;
        for (int i = 0; i < kThreads / 32; ++i) { x += s_red[i][0]; y += s_red[i][1]; z += s_red[i][2]; }
        const int slot = blockIdx.x % kRedSlots;
        atomicAdd(red + 0 * kRedSlots + slot, x);
        atomicAdd(red + 1 * kRedSlots + slot, y);
        atomicAdd(red + 2 * kRedSlots + slot, z);
    }
}

template <int P>
__global__ void __launch_bounds__(kThreads) cheb_step_kernel(const StepParams<P> p) {
    using A = typename Prec<P>::A;
    __shared__ int s_end[kMaxTileRows + 1];      // row ends, relative to the tile's first entry
    __shared__ A s_val[kTileItems];              // gathered y values of the tile's entries
    __shared__ A s_sum[kMaxTileRows + 1];        // row sums
    __shared__ int s_crow[kThreads];             // carry row of each thread
    __shared__ A s_cval[kThreads];               // carry partial of each thread
    __shared__ int s_last;

    const int tid = threadIdx.x;
    const int4 t = p.tiles[blockIdx.x];
    A sT = 0, sA = 0;
    double sR = 0;

    if (t.w > 0) {
        // ---- chunk of a long row ------------------------------------------
        const int u = t.x, j = t.y, slot = t.z, lid = t.w - 1;
        const int e0 = p.row_ptr[u], e1 = p.row_ptr[u + 1];
        const int nch = (e1 - e0 + kTileItems - 1) / kTileItems;
        const int c0 = e0 + j * kTileItems;
        const int c1 = min(c0 + kTileItems, e1);
        const int a0 = c0 & ~3;
        const int nvec = (c1 - a0 + 3) >> 2;
        A acc = 0;
        for (int v = tid; v < nvec; v += kThreads) {
            const int e = a0 + 4 * v;
            const int4 q = load_cols(p.col_idx + e);
            if (e >= c0 && e < c1) acc += load_y(p.y_src + q.x);
            if (e + 1 >= c0 && e + 1 < c1) acc += load_y(p.y_src + q.y);
            if (e + 2 >= c0 && e + 2 < c1) acc += load_y(p.y_src + q.z);
            if (e + 3 >= c0 && e + 3 < c1) acc += load_y(p.y_src + q.w);
        }
        // fixed-shape CTA sum
        s_cval[tid] = acc;
        __syncthreads();
        for (int o = kThreads / 2; o > 0; o >>= 1) {
            if (tid < o) s_cval[tid] = s_cval[tid] + s_cval[tid + o];
            __syncthreads();
        }
        if (tid == 0) {
            p.long_part[slot + j] = s_cval[0];
            __threadfence();
            const int ticket = atomicAdd(p.long_cnt + lid, 1);
            s_last = (ticket == nch - 1);
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            // every chunk partial is visible: add them in chunk order, in a
            // fixed shape (thread i takes chunks i, i+256, ...)
            A part = 0;
            for (int c = tid; c < nch; c += kThreads) part += __ldcg(p.long_part + slot + c);
            __syncthreads();
            s_cval[tid] = part;
            __syncthreads();
            for (int o = kThreads / 2; o > 0; o >>= 1) {
                if (tid < o) s_cval[tid] = s_cval[tid] + s_cval[tid + o];
                __syncthreads();
            }
            if (tid == 0) {
                row_update<P>(p, u, s_cval[0], sT, sA, sR);
                p.long_cnt[lid] = 0;  // ready for the next round
            }
            cta_reduce_add((double)sT, (double)sA, sR, p.red);
        }
        return;
    }

    // ---- block tile of whole rows -------------------------------------------
    const int r0 = t.x, r1 = t.y;
    const int nrows = r1 - r0;
    const int e0 = p.row_ptr[r0], e1 = p.row_ptr[r1];
    const int nnz = e1 - e0;
    for (int i = tid; i < nrows; i += kThreads) s_end[i] = p.row_ptr[r0 + 1 + i] - e0;
    {
        const int a0 = e0 & ~3;
        const int nvec = (e1 - a0 + 3) >> 2;
#pragma unroll 2
        for (int v = tid; v < nvec; v += kThreads) {
            const int e = a0 + 4 * v;
            const int4 q = load_cols(p.col_idx + e);
            const int k = e - e0;
            if (k >= 0 && k < nnz) s_val[k] = load_y(p.y_src + q.x);
            if (k + 1 >= 0 && k + 1 < nnz) s_val[k + 1] = load_y(p.y_src + q.y);
            if (k + 2 >= 0 && k + 2 < nnz) s_val[k + 2] = load_y(p.y_src + q.z);
            if (k + 3 >= 0 && k + 3 < nnz) s_val[k + 3] = load_y(p.y_src + q.w);
        }
    }
    __syncthreads();

    // merge path over (row ends, entries): thread tid owns diagonals [d0, d1)
    const int items = nrows + nnz;
    const int d0 = min(tid * kItemsPerThread, items);
    const int d1 = min(d0 + kItemsPerThread, items);
    int lo = max(d0 - nnz, 0), hi = min(d0, nrows);
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (s_end[mid] <= d0 - mid - 1) lo = mid + 1; else hi = mid;
    }
    int row = lo, k = d0 - lo;
    int first_emit = -1;
    A acc = 0;
    for (int d = d0; d < d1; ++d) {
        if (k < s_end[row]) {
            acc += s_val[k];
            ++k;
        } else {
            s_sum[row] = acc;
            if (first_emit < 0) first_emit = row;
            acc = 0;
            ++row;
        }
    }
    s_crow[tid] = (d0 < d1) ? row : -1;
    s_cval[tid] = acc;
    __syncthreads();
    if (first_emit >= 0) {
        // the row this thread closed first may have started in earlier threads
        int j = tid - 1;
        while (j >= 0 && s_crow[j] == first_emit) --j;
        A pre = 0;
        for (int i = j + 1; i < tid; ++i) pre += s_cval[i];
        s_sum[first_emit] = pre + s_sum[first_emit];
    }
    __syncthreads();
    for (int i = tid; i < nrows; i += kThreads) row_update<P>(p, r0 + i, s_sum[i], sT, sA, sR);
    cta_reduce_add((double)sT, (double)sA, sR, p.red);
}

template <int P>
static cudaError_t launch_typed(const StepLaunch &s) {
    using A = typename Prec<P>::A;
    using S = typename Prec<P>::S;
    using R = typename Prec<P>::R;
    const cpaa_graph *g = s.g;
    StepParams<P> p;
    p.tiles = g->tiles;
    p.row_ptr = g->row_ptr;
    p.col_idx = g->col_idx;
    if constexpr (P == CPAA_F64) {
        p.deg = g->deg64;
        p.inv_deg = g->inv_deg64;
    } else {
        p.deg = g->deg32;
        p.inv_deg = g->inv_deg32;
    }
    p.y_src = static_cast<const S *>(s.y_src);
    p.y_io = static_cast<S *>(s.y_io);
    p.rho = static_cast<R *>(s.rho);
    p.comp = static_cast<R *>(s.comp);
    p.long_part = reinterpret_cast<A *>(g->long_part);
    p.long_cnt = g->long_cnt;
    p.red = s.red;
    p.ck = (A)s.ck;
    p.first = s.first;
    p.last = s.last;
    cheb_step_kernel<P><<<g->num_tiles, kThreads, 0, s.stream>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_step(const StepLaunch &s) {
    switch (s.precision) {
        case CPAA_F64: return launch_typed<CPAA_F64>(s);
        case CPAA_F32: return launch_typed<CPAA_F32>(s);
        case CPAA_BF16: return launch_typed<CPAA_BF16>(s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace cpaa
