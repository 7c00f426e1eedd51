// step_impl.cuh -- one round of the Chebyshev recurrence for a tile of W vectors,
// fused with the accumulation and the per-round reductions (Algorithm 1,
// Sec. 4.1).  W = 1 is the single-vector solve; W > 1 is the batched form
// (an SpMM: each gathered neighbour row brings W values at once).  Both use
// this one kernel, so a vector's result does not depend on how it was batched.
//
// Scaled space.  The kernels keep y_k = D^-1 T_k p instead of T_k p.  Then
//     (P T_k)[u] = sum_{j in N(u)} T_k[j] / d_j = sum_{j in N(u)} y_k[j],
// so the gather is a plain sum of neighbour values with no degree lookup, and
//     y_1[u]     = (1/d_u) sum_{j in N(u)} y_0[j]                  (k = 1)
//     y_{k+1}[u] = (2/d_u) sum_{j in N(u)} y_k[j] - y_{k-1}[u]     (k >= 1)
// which is T_{k+1} = 2 P T_k - T_{k-1} (Chebyshev property (3), Sec. 2.2)
// divided by d_u; the kernel reads 2/d_u and makes the update one fused
// multiply-add.  The accumulator is rho = D^-1 pibar, rho += c_k y_k, and the
// finalisation multiplies by d_u again.  y_{k+1} overwrites y_{k-1} in place:
// row u is the only reader of y_{k-1}[u].
//
// Layout: vector b of a tile is column b of a row-major [(n+1) x W] array
// (row n is the padding sentinel, kept at zero).  Column b accumulates while
// bit b of `active` is set and bit b of *stop is clear.
//
// Per-round sums (the mass view of Sec. 4.1: sum_u T_k[u] and sum_u |T_k[u]|)
// are taken in rounds whose `reduce` mask is not zero.  Every work item (a hub
// row, a SELL chunk) writes its own partial sums to a slot of its own (a
// chunk's 32 rows by a fixed shuffle tree), and two small kernels add the
// slots in a fixed order; so the sums, and the stopping decision taken from
// them, are the same bits for a vector alone and in any tile.
//
// Work split (internal.h): a persistent grid.  CTAs first take the hub tiles
// (one tile of a hub row each) and the long SELL chunks (above the long-chunk
// threshold, split over the CTA's warps) round-robin; then every warp takes
// short SELL chunks, one lane per row, round-robin from the longest-first
// order (chunk descriptors are stored in that order).  Every sum runs in a
// fixed order (a lane adds its row's entries in CSR order, slices are added
// in warp order; hub tiles use shuffle trees over thread-strided sums and the
// tiles are added in tile order), so a result never depends on scheduling.
//
// Number formats (device_common.cuh): FP64, FP32 and BF16 iterates, and
// double-float pairs of FP32 (DF64) whose arithmetic runs on the FP32 pipes.
#pragma once

#include <algorithm>
#include <cstring>

#include "device_common.cuh"

namespace cpaa {

template <int P, int W>
struct StepParams {
    using S = typename Prec<P>::S;
    using A = typename Prec<P>::A;
    using R = typename Prec<P>::R;
    // hub rows
    const int4 *hub_tiles;
    int num_hub_tiles;
    int hub_tile;  // entries per hub tile
    const int32_t *hub_row_ptr;
    const int32_t *hub_col;
    A *long_part;  // [num_hub_tiles][W]
    int *long_cnt;
    // SELL chunks
    const int32_t *sell_col;
    const int4 *chunk_desc;  // {chunk, offset / 128, stored length, longest row}, longest first
    int num_chunks;
    int num_long_chunks;  // chunk_desc[0, num_long_chunks) take one CTA each
    int n_hub;
    int64_t n;
    // vectors (new order)
    const A *deg;
    const A *inv_deg;  // 2 / d for Chebyshev rounds, 1 / d for power-method rounds
    // the same by degree for the rows of short chunks, which read their
    // degree as a 2-byte word: tab_inv[d] is inv_deg's value (ia 2 / d for the
    // interval series), tab_deg[d] = d
    const uint16_t *deg16;
    const A *tab_inv;
    const A *tab_deg;
    const S *y_src;  // [(n+1) x W]
    S *y_io;         // [(n+1) x W]
    R *rho;          // [n x W]
    R *comp;         // [n x W]
    double *ipart;   // item partial sums [(n_hub + num_chunks)][2][W] (reducing rounds)
    const unsigned *stop;  // columns stopped by the a-posteriori rule, or NULL
    A ck[W];
    A ck_prev[W];     // coefficient of a term left from the last round
    unsigned pend;    // columns adding last round's term c_{k-1} y_{k-1} now (read back from y_src)
    unsigned defer;   // columns whose term this round is added in the next one
    unsigned active;
    unsigned reduce;
    unsigned first;  // columns in their first round (y_1 = D^-1 P y_0... scaled: s / d)
    int power;       // 1: power-method round y' = c s / d + q, ck[b] = c, q held in rho
    int interval;    // 1: the series on [lambda_lo, 1] (interval_iterate), with
    A ia, mb;        //    ia = 1 / half and mb = -2 mid / half
    // sparse frontier (frontier.cu), or front == NULL: items with no row in
    // front are skipped, unless *front_full or the covered entries exceed
    // front_limit (then this and every later round take every item)
    const unsigned *front;
    int *front_full;
    const unsigned long long *front_entries;
    unsigned long long front_limit;
    int front_hub_words;
};

// Whether an item holds a row of the frontier: a hub tile's row, a chunk's rows.
__device__ __forceinline__ bool hub_in_front(const unsigned *fr, int h) { return fr[h >> 5] >> (h & 31) & 1u; }
__device__ __forceinline__ bool chunk_in_front(const unsigned *fr, int hub_words, int c) {
    return fr[hub_words + c] != 0u;
}

// W consecutive values of one row, with the widest loads the row size allows.
template <class T, int W>
__device__ __forceinline__ void load_row(const T *p, T (&v)[W], bool stream) {
    constexpr int B = W * (int)sizeof(T);
    if constexpr (B % 16 == 0) {
        uint4 raw[B / 16];
#pragma unroll
        for (int i = 0; i < B / 16; ++i)
            raw[i] = stream ? __ldcs(reinterpret_cast<const uint4 *>(p) + i)
                            : __ldg(reinterpret_cast<const uint4 *>(p) + i);
        memcpy(v, raw, B);
    } else if constexpr (B % 8 == 0) {
        uint2 raw[B / 8];
#pragma unroll
        for (int i = 0; i < B / 8; ++i)
            raw[i] = stream ? __ldcs(reinterpret_cast<const uint2 *>(p) + i)
                            : __ldg(reinterpret_cast<const uint2 *>(p) + i);
        memcpy(v, raw, B);
    } else if constexpr (B % 4 == 0) {
        unsigned raw[B / 4];
#pragma unroll
        for (int i = 0; i < B / 4; ++i)
            raw[i] = stream ? __ldcs(reinterpret_cast<const unsigned *>(p) + i)
                            : __ldg(reinterpret_cast<const unsigned *>(p) + i);
        memcpy(v, raw, B);
    } else {
        unsigned short raw = __ldg(reinterpret_cast<const unsigned short *>(p));
        memcpy(v, &raw, B);
    }
}

template <class T, int W>
__device__ __forceinline__ void store_row(T *p, const T (&v)[W], bool stream) {
    constexpr int B = W * (int)sizeof(T);
    if constexpr (B % 16 == 0) {
        uint4 raw[B / 16];
        memcpy(raw, v, B);
#pragma unroll
        for (int i = 0; i < B / 16; ++i) {
            if (stream) __stcs(reinterpret_cast<uint4 *>(p) + i, raw[i]);
            else reinterpret_cast<uint4 *>(p)[i] = raw[i];
        }
    } else if constexpr (B % 8 == 0) {
        uint2 raw[B / 8];
        memcpy(raw, v, B);
#pragma unroll
        for (int i = 0; i < B / 8; ++i) {
            if (stream) __stcs(reinterpret_cast<uint2 *>(p) + i, raw[i]);
            else reinterpret_cast<uint2 *>(p)[i] = raw[i];
        }
    } else if constexpr (B % 4 == 0) {
        unsigned raw[B / 4];
        memcpy(raw, v, B);
#pragma unroll
        for (int i = 0; i < B / 4; ++i) {
            if (stream) __stcs(reinterpret_cast<unsigned *>(p) + i, raw[i]);
            else reinterpret_cast<unsigned *>(p)[i] = raw[i];
        }
    } else {
        unsigned short raw;
        memcpy(&raw, v, B);
        *reinterpret_cast<unsigned short *>(p) = raw;
    }
}

// Warp shuffle and L2-coherent load of an arithmetic value (a double-float
// moves as its two halves).
__device__ __forceinline__ float shfl_xor(float v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ double shfl_xor(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ df shfl_xor(df v, int o) {
    return df(__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o));
}
__device__ __forceinline__ float ld_cg(const float *p) { return __ldcg(p); }
__device__ __forceinline__ double ld_cg(const double *p) { return __ldcg(p); }
__device__ __forceinline__ df ld_cg(const df *p) {
    const float2 v = __ldcg(reinterpret_cast<const float2 *>(p));
    return df(v.x, v.y);
}

// Gathered neighbour row j: W values in arithmetic precision.
template <int P, int W>
__device__ __forceinline__ void gather_row(const typename Prec<P>::S *y, int j,
                                           typename Prec<P>::A (&x)[W]) {
    using S = typename Prec<P>::S;
    S v[W];
    load_row<S, W>(y + (int64_t)j * W, v, false);
#pragma unroll
    for (int b = 0; b < W; ++b) x[b] = to_acc(v[b]);
}

// A row's own operands: the iterate it overwrites, its current one (read
// when a deferred term is added or by the interval series), the accumulator
// and its compensation.
template <int P, int W>
struct RowOps {
    typename Prec<P>::A y_old[W];
    typename Prec<P>::A yp[W];
    typename Prec<P>::R rr[W];
    typename Prec<P>::R cmp[W];
};

// Whether a round kernel form takes deferred terms (defer_supported on the
// host gives the same answer): the single-vector FP32, BF16 and DF64 forms.
// Elsewhere the pending term's read and add cost more registers than its
// bytes save (measured: the FP64 single vector 32 -> 40, FP32 tiles of two
// 32 -> 40, FP64 tiles of 16 156 -> 251).
template <int P, int W, bool I>
__device__ __forceinline__ constexpr bool deferred_form() {
    return W == 1 && P != CPAA_F64;
}

// Whether this round reads and writes the accumulator: a term is added now
// (one left from the last round, or this round's own), or rho holds the power
// method's q.  The same for every thread of the launch.
template <int P, int W, bool I>
__device__ __forceinline__ bool rho_touched(const StepParams<P, W> &p) {
    if constexpr (!deferred_form<P, W, I>()) return p.power || p.active != 0u;
    else return p.power || (p.pend | (p.active & ~p.defer)) != 0u;
}

// The row's stored y_{k-1} into o.yp.
template <int P, int W>
__device__ __forceinline__ void load_yp(const StepParams<P, W> &p, int64_t r, RowOps<P, W> &o) {
    typename Prec<P>::S v[W];
    load_row<typename Prec<P>::S, W>(p.y_src + r * W, v, false);
#pragma unroll
    for (int b = 0; b < W; ++b) o.yp[b] = to_acc(v[b]);
}

template <int P, int W, bool I>
__device__ __forceinline__ void load_ops(const StepParams<P, W> &p, int64_t r, RowOps<P, W> &o) {
    using S = typename Prec<P>::S;
    using A = typename Prec<P>::A;
    using R = typename Prec<P>::R;
    if (p.first == (W == 32 ? 0xffffffffu : ((1u << W) - 1u))) {
#pragma unroll
        for (int b = 0; b < W; ++b) o.y_old[b] = A(0);
    } else {  // columns in their first round ignore the value read here
        S v[W];
        load_row<S, W>(p.y_io + r * W, v, true);
#pragma unroll
        for (int b = 0; b < W; ++b) o.y_old[b] = to_acc(v[b]);
    }
    // y_{k-1}: narrow tiles fetch their operands before the gather, so they
    // read it in the epilogue (registers) and only bring it to L1 here
    if (I || (deferred_form<P, W, I>() && p.pend)) {
        if constexpr (W <= 4) asm volatile("prefetch.global.L1 [%0];" ::"l"(p.y_src + r * W));
        else load_yp<P, W>(p, r, o);
    }
    if (rho_touched<P, W, I>(p)) {
        load_row<R, W>(p.rho + r * W, o.rr, true);
        if constexpr (Prec<P>::kKahan) load_row<R, W>(p.comp + r * W, o.cmp, true);
        else {
#pragma unroll
            for (int b = 0; b < W; ++b) o.cmp[b] = R(0);
        }
    } else {  // nothing is added to rho this round
#pragma unroll
        for (int b = 0; b < W; ++b) o.rr[b] = o.cmp[b] = R(0);
    }
}

// The row's factor for the recurrence: inv_deg's value, times ia for the
// interval series (the table path has it scaled already).
template <int P, int W, bool I>
__device__ __forceinline__ typename Prec<P>::A row_factor(const StepParams<P, W> &p, typename Prec<P>::A inv) {
    if constexpr (I) return mul_rn(p.ia, inv);
    else return inv;
}

// Row epilogue: new iterates and accumulation; yv receives the new iterates
// (as stored) for the round's sums.  inv is the row's factor (row_factor).
// A term left from the last round is added first, from the stored y_{k-1}
// (which is the value that round accumulated would have used), so rho takes
// the same operations in the same order as without deferral.
template <int P, int W, bool I>
__device__ __forceinline__ void row_finish(const StepParams<P, W> &p, int64_t r,
                                           const typename Prec<P>::A (&s)[W],
                                           typename Prec<P>::A inv, RowOps<P, W> &o,
                                           typename Prec<P>::A (&yv)[W], unsigned active) {
    using S = typename Prec<P>::S;
    using A = typename Prec<P>::A;
    using R = typename Prec<P>::R;
    S ys[W];
    if (p.power) {
        // power method (x' = c P x + (1 - c) p, scaled by D^-1): q = (1 - c) p / d
#pragma unroll
        for (int b = 0; b < W; ++b) {
            const A y = power_iterate<P>(s[b], inv, p.ck[b], o.rr[b]);
            store_y(&ys[b], y);
            yv[b] = y;
        }
        store_row<S, W>(p.y_io + r * W, ys, false);
        return;
    }
    // o.yp: the row's own y_{k-1} as stored (a pending term's value, the
    // interval series' y_cur; the plain form reads it here, only in rounds
    // that add a pending term, to keep its registers)
    constexpr bool kDefer = deferred_form<P, W, I>();
    if constexpr (W <= 4) {
        if (I || (kDefer && p.pend)) load_yp<P, W>(p, r, o);
    }
    const unsigned pend = kDefer ? p.pend : 0u;
    const unsigned now = kDefer ? (active & ~p.defer) : active;
    auto column = [&](int b, unsigned first) {
        if (pend >> b & 1u) accumulate<P>(o.rr[b], o.cmp[b], p.ck_prev[b], o.yp[b]);
        A y;
        if constexpr (I) y = interval_iterate<P>(s[b], inv, o.yp[b], o.y_old[b], first, p.mb);
        else y = new_iterate<P>(s[b], inv, o.y_old[b], first);
        store_y(&ys[b], y);
        if (now >> b & 1u) accumulate<P>(o.rr[b], o.cmp[b], p.ck[b], y);
        yv[b] = y;
    };
    // every round but a column's first takes the plain update: a branch on the
    // launch's mask, so that the first round's form is not evaluated (and
    // selected away) on every row of every round.  On GB300's FP64 pipe that
    // evaluation was two multiplies a row and column: the branch took the FP64
    // lattice round from 0.270 to 0.211 ms, and an FP64 batch of 8 on the
    // lattice from 92.3 to 79.7 ms.  FP32 and BF16 tiles keep one loop (the
    // branch would cost them registers), and so does DF64, whose products run
    // on the FP32 pipes (2% slower with it).
    if ((W == 1 && P != CPAA_DF64 && p.first == 0u) || (W > 1 && P == CPAA_F64 && p.first == 0u)) {
#pragma unroll
        for (int b = 0; b < W; ++b) column(b, 0u);
    } else {
#pragma unroll
        for (int b = 0; b < W; ++b) column(b, (p.first >> b) & 1u);
    }
    store_row<S, W>(p.y_io + r * W, ys, false);
    if (rho_touched<P, W, I>(p)) {
        store_row<R, W>(p.rho + r * W, o.rr, true);
        if constexpr (Prec<P>::kKahan) store_row<R, W>(p.comp + r * W, o.cmp, true);
    }
}

// A row's terms of the round's sums: T = d y and |T| (only in rounds that take
// sums; the others skip this arithmetic, which matters on GB300's slow FP64
// pipe).
template <class A, int W>
__device__ __forceinline__ void row_terms(const A (&yv)[W], A d, A (&tT)[W], A (&tA)[W]) {
#pragma unroll
    for (int b = 0; b < W; ++b) {
        const A T = yv[b] * d;
        tT[b] = T;
        tA[b] = (T < A(0) ? -T : T);
    }
}

// A chunk's partial sums: the 32 rows' T and |T| added by a fixed shuffle
// tree, written by lane 0 to item slot `item` (all W columns).
template <class A, int W>
__device__ __forceinline__ void warp_item_sums(A (&tT)[W], A (&tA)[W], double *ipart, int64_t item) {
#pragma unroll
    for (int b = 0; b < W; ++b)
        for (int o = 16; o > 0; o >>= 1) {
            tT[b] += shfl_xor(tT[b], o);
            tA[b] += shfl_xor(tA[b], o);
        }
    if ((threadIdx.x & 31) == 0) {
        double *d = ipart + item * 2 * W;
#pragma unroll
        for (int b = 0; b < W; ++b) {
            d[b] = to_double(tT[b]);
            d[W + b] = to_double(tA[b]);
        }
    }
}

// Fixed-shape sum over the CTA of one value per thread and column: a shuffle
// tree in each warp, then thread 0 adds the kWarps warp sums in warp order.
// Returns the total in thread 0 (other threads: unspecified).
template <class A, int W>
__device__ __forceinline__ void cta_sum_w(A (&v)[W], A (&s_w)[kWarps][W]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int b = 0; b < W; ++b)
        for (int o = 16; o > 0; o >>= 1) v[b] += shfl_xor(v[b], o);
    if (lane == 0)
#pragma unroll
        for (int b = 0; b < W; ++b) s_w[warp][b] = v[b];
    __syncthreads();
    if (threadIdx.x == 0)
#pragma unroll
        for (int b = 0; b < W; ++b) {
            A t = s_w[0][b];
            for (int q = 1; q < kWarps; ++q) t += s_w[q][b];
            v[b] = t;
        }
}

// One hub tile (p.hub_tile entries of a hub row) by one CTA.  The CTA
// that takes the row's last ticket adds the tile partials in tile order and
// writes the row (an atomic ticket: no CTA waits for another).
template <int P, int W, bool I>
__device__ __forceinline__ void hub_tile(const StepParams<P, W> &p, int4 t, unsigned active) {
    using A = typename Prec<P>::A;
    __shared__ A s_w[kWarps][W];
    __shared__ int s_last;
    const int tid = threadIdx.x;
    const int h = t.x, j = t.y, slot = t.z, hub = t.w - 1;
    const int e0 = p.hub_row_ptr[h], e1 = p.hub_row_ptr[h + 1];
    const int nt = (e1 - e0 + p.hub_tile - 1) / p.hub_tile;
    const int c0 = e0 + j * p.hub_tile;
    const int c1 = min(c0 + p.hub_tile, e1);
    const int a0 = c0 & ~3;
    const int nvec = (c1 - a0 + 3) >> 2;
    A acc[W];
#pragma unroll
    for (int b = 0; b < W; ++b) acc[b] = A(0);
#pragma unroll 2
    for (int v = tid; v < nvec; v += kThreads) {
        const int e = a0 + 4 * v;
        const int4 q = ld_stream4(p.hub_col + e);
        A x0[W], x1[W], x2[W], x3[W];
        // entries outside [c0, c1) gather the sentinel row n, which holds zeros
        gather_row<P, W>(p.y_src, (e >= c0 && e < c1) ? q.x : (int)p.n, x0);
        gather_row<P, W>(p.y_src, (e + 1 >= c0 && e + 1 < c1) ? q.y : (int)p.n, x1);
        gather_row<P, W>(p.y_src, (e + 2 >= c0 && e + 2 < c1) ? q.z : (int)p.n, x2);
        gather_row<P, W>(p.y_src, (e + 3 >= c0 && e + 3 < c1) ? q.w : (int)p.n, x3);
#pragma unroll
        for (int b = 0; b < W; ++b) acc[b] += ((x0[b] + x1[b]) + (x2[b] + x3[b]));
    }
    cta_sum_w<A, W>(acc, s_w);
    if (tid == 0) {
#pragma unroll
        for (int b = 0; b < W; ++b) p.long_part[(int64_t)(slot + j) * W + b] = acc[b];
        __threadfence();
        const int ticket = atomicAdd(p.long_cnt + hub, 1);
        s_last = (ticket == nt - 1);
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        // every tile partial is visible: add them in tile order, fixed shape
        A part[W];
#pragma unroll
        for (int b = 0; b < W; ++b) part[b] = A(0);
        for (int c = tid; c < nt; c += kThreads)
#pragma unroll
            for (int b = 0; b < W; ++b) part[b] += ld_cg(p.long_part + (int64_t)(slot + c) * W + b);
        __syncthreads();  // s_w is free again
        cta_sum_w<A, W>(part, s_w);
        if (tid == 0) {
            RowOps<P, W> o;
            load_ops<P, W, I>(p, h, o);
            A yv[W], tT[W], tA[W];
            row_finish<P, W, I>(p, h, part, row_factor<P, W, I>(p, p.inv_deg[h]), o, yv, active);
            if (p.reduce) {
                row_terms<A, W>(yv, p.deg[h], tT, tA);
                double *d = p.ipart + (int64_t)h * 2 * W;
#pragma unroll
                for (int b = 0; b < W; ++b) {
                    d[b] = to_double(tT[b]);
                    d[W + b] = to_double(tA[b]);
                }
            }
            p.long_cnt[hub] = 0;  // ready for the next round
        }
    }
    __syncthreads();  // s_w and s_last are reused by the CTA's next item
}

// Groups of kSellVec entries a lane gathers at once in a short chunk (single
// vector); wider tiles bring W values per gathered row and take fewer groups.
#ifndef CPAA_SELL_GROUPS
#define CPAA_SELL_GROUPS 2
#endif
template <int W> struct Unroll {
    static constexpr int value = W >= 4 ? 1 : (CPAA_SELL_GROUPS / W > 0 ? CPAA_SELL_GROUPS / W : 1);
};

// U full groups of a lane's SELL entries starting at group q, in CSR order.
template <int P, int W, int U>
__device__ __forceinline__ void sum_groups(const StepParams<P, W> &p, const int32_t *col, int q,
                                           typename Prec<P>::A (&acc)[W]) {
    using A = typename Prec<P>::A;
    constexpr int G = kChunkRows * kSellVec;
    int4 jj[U];
#pragma unroll
    for (int k = 0; k < U; ++k) jj[k] = ld_stream4(col + (int64_t)(q + k) * G);
    A x[U][4][W];
#pragma unroll
    for (int k = 0; k < U; ++k) {
        gather_row<P, W>(p.y_src, jj[k].x, x[k][0]);
        gather_row<P, W>(p.y_src, jj[k].y, x[k][1]);
        gather_row<P, W>(p.y_src, jj[k].z, x[k][2]);
        gather_row<P, W>(p.y_src, jj[k].w, x[k][3]);
    }
#pragma unroll
    for (int k = 0; k < U; ++k)
#pragma unroll
        for (int e = 0; e < 4; ++e)
#pragma unroll
            for (int b = 0; b < W; ++b) acc[b] += x[k][e][b];
}

// Sum of the lane's row entries in SELL groups [q0, q1) plus the first `tail`
// (0..4) entries of group q1.  `col` points at the chunk's lane group (chunk
// start + kSellVec * lane).  The tail and every bound are the same for the 32
// lanes (the chunk's longest row sets them), so every branch here is
// warp-uniform; a chunk is trimmed to its longest row's length, so groups
// past it are never loaded and no sentinel is added there.  Order: the tail's
// entries first (the sum starts from its first entry, while no other value is
// live), then the full groups in CSR order.
#ifndef CPAA_SELL_TAIL
#define CPAA_SELL_TAIL 1
#endif
template <int P, int W>
__device__ __forceinline__ void chunk_sum(const StepParams<P, W> &p, const int32_t *col, int q0, int q1, int tail,
                                          typename Prec<P>::A (&acc)[W]) {
    using A = typename Prec<P>::A;
    constexpr int U = Unroll<W>::value;  // groups of four entries in flight per lane
    constexpr int G = kChunkRows * kSellVec;
    if (tail) {
        // all four loads at once (slots past the longest row hold the zero
        // sentinel), so their latencies overlap; only the additions depend on
        // the tail's length
        const int4 j = ld_stream4(col + (int64_t)q1 * G);
        A x1[W], x2[W], x3[W];
        gather_row<P, W>(p.y_src, j.x, acc);
        gather_row<P, W>(p.y_src, j.y, x1);
        gather_row<P, W>(p.y_src, j.z, x2);
        gather_row<P, W>(p.y_src, j.w, x3);
        if (tail > 1)
#pragma unroll
            for (int b = 0; b < W; ++b) acc[b] += x1[b];
        if (tail > 2)
#pragma unroll
            for (int b = 0; b < W; ++b) acc[b] += x2[b];
        if (tail > 3)
#pragma unroll
            for (int b = 0; b < W; ++b) acc[b] += x3[b];
    } else {
#pragma unroll
        for (int b = 0; b < W; ++b) acc[b] = A(0);
    }
    int q = q0;
    if constexpr (W >= 8) {
        // wide rows: one gathered row in registers at a time
        for (; q < q1; ++q) {
            const int4 j = ld_stream4(col + (int64_t)q * G);
            const int jj[4] = {j.x, j.y, j.z, j.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                A x[W];
                gather_row<P, W>(p.y_src, jj[e], x);
#pragma unroll
                for (int b = 0; b < W; ++b) acc[b] += x[b];
            }
        }
    } else {
        for (; q + U <= q1; q += U) sum_groups<P, W, U>(p, col, q, acc);
        for (; q < q1; ++q) sum_groups<P, W, 1>(p, col, q, acc);
    }
}

// Full groups and tail (the last group, 1..kSellVec entries: its first
// entry starts the sum) of a chunk whose longest row has `exact` >= 1 entries.
// Only FP64 takes the tail: there every addition costs a slot of GB300's slow
// FP64 pipe (the lattice round keeps it 70% busy), while the other formats,
// bound by memory, lose more to the tail's branches than they save
// (measured: FP64 lattice round 0.328 -> 0.286 ms; FP32 0.138 -> 0.142 ms).
template <int P>
__device__ __forceinline__ void chunk_extent(int exact, int &groups, int &tail) {
    if (CPAA_SELL_TAIL && P == CPAA_F64) {
        groups = (exact - 1) / kSellVec;
        tail = exact - kSellVec * groups;
    } else {
        groups = (exact + kSellVec - 1) / kSellVec;
        tail = 0;
    }
}

// A long chunk by one CTA: warp w sums slice w of the entries of all 32
// rows; the slices are added in warp order and warp 0 finishes the rows.
template <int P, int W, bool I>
__device__ __forceinline__ void long_chunk(const StepParams<P, W> &p, int4 dsc, unsigned active) {
    using A = typename Prec<P>::A;
    __shared__ A s_part[kWarps][W][kChunkRows];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c = dsc.x;
    const int64_t off = (int64_t)dsc.y * (kChunkRows * kSellVec);
    int groups, tail;
    chunk_extent<P>(dsc.w, groups, tail);
    // slices of whole kSellVec groups; the last slice takes the tail
    const int per = (groups + (tail ? 1 : 0) + kWarps - 1) / kWarps;
    const int q0 = min(groups, warp * per), q1 = min(groups, q0 + per);
    const int t = (warp * per <= groups && groups < (warp + 1) * per) ? tail : 0;  // the tail's slice
    A acc[W];
    chunk_sum<P, W>(p, p.sell_col + off + kSellVec * lane, q0, q1, t, acc);
#pragma unroll
    for (int b = 0; b < W; ++b) s_part[warp][b][lane] = acc[b];
    __syncthreads();
    if (warp == 0) {
        const int64_t r = p.n_hub + (int64_t)c * kChunkRows + lane;
        A s[W];
#pragma unroll
        for (int b = 0; b < W; ++b) {
            s[b] = s_part[0][b][lane];
            for (int q = 1; q < kWarps; ++q) s[b] += s_part[q][b][lane];
        }
        A yv[W];
#pragma unroll
        for (int b = 0; b < W; ++b) yv[b] = A(0);
        if (r < p.n) {
            RowOps<P, W> o;
            load_ops<P, W, I>(p, r, o);
            row_finish<P, W, I>(p, r, s, row_factor<P, W, I>(p, ld_once(p.inv_deg + r)), o, yv, active);
        }
        if (p.reduce) {
            A tT[W], tA[W];
            row_terms<A, W>(yv, r < p.n ? ld_once(p.deg + r) : A(0), tT, tA);
            warp_item_sums<A, W>(tT, tA, p.ipart, p.n_hub + c);
        }
    }
    __syncthreads();  // s_part is reused by the CTA's next item
}

// A short SELL chunk by one warp: lane l sums row n_hub + 32 c + l and
// finishes it; the chunk's partial sums go to its item slot in rounds that
// take sums.
template <int P, int W, bool I>
__device__ __forceinline__ void short_chunk(const StepParams<P, W> &p, int4 dsc, unsigned active) {
    using A = typename Prec<P>::A;
    const int lane = threadIdx.x & 31;
    const int c = dsc.x;
    const int64_t off = (int64_t)dsc.y * (kChunkRows * kSellVec);
    int groups, tail;
    chunk_extent<P>(dsc.w, groups, tail);
    const int64_t r = p.n_hub + (int64_t)c * kChunkRows + lane;
    const bool live = r < p.n;
    // for narrow tiles the row's own operands are fetched before the gather
    // so that their latency overlaps it
    constexpr bool kEarly = W <= 4;
    // the row's factors by its degree: a 2-byte word and the degree tables
    // (cached), fetched before the gather like the other operands
    A inv = A(0), d = A(0);
    RowOps<P, W> o;
    if (live) {
        const int dg = ld_once(p.deg16 + r);
        inv = ld_ro(p.tab_inv + dg);
        if (p.reduce) d = ld_ro(p.tab_deg + dg);  // only the round's sums need d
        if constexpr (kEarly) load_ops<P, W, I>(p, r, o);
    }
    A acc[W];
    chunk_sum<P, W>(p, p.sell_col + off + kSellVec * lane, 0, groups, tail, acc);
    A yv[W];
#pragma unroll
    for (int b = 0; b < W; ++b) yv[b] = A(0);
    if (live) {
        if constexpr (!kEarly) load_ops<P, W, I>(p, r, o);
        row_finish<P, W, I>(p, r, acc, inv, o, yv, active);
    }
    if (p.reduce) {
        A tT[W], tA[W];
        row_terms<A, W>(yv, d, tT, tA);
        warp_item_sums<A, W>(tT, tA, p.ipart, p.n_hub + c);
    }
}

// Persistent grid (as many CTAs as fit on the GPU at once).  Phase 1: CTAs
// take the CTA-sized items (hub tiles, then long chunks) round-robin.  Phase
// 2: every warp takes short chunks round-robin from the longest-first order,
// which balances the warps without any atomics.
template <int P, int W, bool I>
__global__ void __launch_bounds__(kThreads) cheb_step_kernel(const StepParams<P, W> p) {
    // columns stopped by the a-posteriori rule no longer accumulate; once
    // every column has stopped the remaining rounds do nothing
    const unsigned active = p.stop ? (p.active & ~*p.stop) : p.active;
    if (p.stop && active == 0 && p.pend == 0) return;
    // sparse frontier: every thread takes the same decision from the same two
    // words (the flag it may set is set only when the count already says so)
    bool filt = false;
    if (p.front) {
        filt = !(*p.front_full || *p.front_entries > p.front_limit);
        if (!filt && blockIdx.x == 0 && threadIdx.x == 0) *p.front_full = 1;
    }
    const int n_cta_items = p.num_hub_tiles + p.num_long_chunks;
    for (int it = blockIdx.x; it < n_cta_items; it += gridDim.x) {
        if (it < p.num_hub_tiles) {
            const int4 t = p.hub_tiles[it];
            if (filt && !hub_in_front(p.front, t.x)) continue;  // the same for the whole CTA
            hub_tile<P, W, I>(p, t, active);
        } else {
            const int4 d = ld_stream4(&p.chunk_desc[it - p.num_hub_tiles].x);
            if (filt && !chunk_in_front(p.front, p.front_hub_words, d.x)) continue;
            long_chunk<P, W, I>(p, d, active);
        }
    }
    const int nwarps = (int)gridDim.x * kWarps;
    for (int idx = p.num_long_chunks + (int)blockIdx.x * kWarps + (int)(threadIdx.x >> 5); idx < p.num_chunks;
         idx += nwarps) {
        const int4 d = ld_stream4(&p.chunk_desc[idx].x);
        if (filt && !chunk_in_front(p.front, p.front_hub_words, d.x)) continue;  // the same for the whole warp
        short_chunk<P, W, I>(p, d, active);
    }
}

// One round over several graphs in one launch (the server's fused mode): the
// CTA items of every graph, then the short chunks of every graph, each work
// list the graphs' lists back to back.  The per-graph parameters sit in the
// launch's constant parameter space and are indexed in place.
constexpr int kMaxFused = 8;
template <int P, int W>
struct MultiParams {
    int ng;
    int cta_off[kMaxFused + 1];   // prefix sums of the graphs' CTA items
    int warp_off[kMaxFused + 1];  // prefix sums of the graphs' short chunks
    StepParams<P, W> g[kMaxFused];
};

template <int P, int W>
__global__ void __launch_bounds__(kThreads) cheb_step_multi_kernel(const __grid_constant__ MultiParams<P, W> mp) {
    for (int it = blockIdx.x; it < mp.cta_off[mp.ng]; it += gridDim.x) {
        int gi = 0;
        while (it >= mp.cta_off[gi + 1]) ++gi;
        const StepParams<P, W> &p = mp.g[gi];
        const unsigned active = p.stop ? (p.active & ~*p.stop) : p.active;
        if (p.stop && active == 0 && p.pend == 0) continue;
        const int local = it - mp.cta_off[gi];
        if (local < p.num_hub_tiles) hub_tile<P, W, false>(p, p.hub_tiles[local], active);
        else long_chunk<P, W, false>(p, ld_stream4(&p.chunk_desc[local - p.num_hub_tiles].x), active);
    }
    const int nwarps = (int)gridDim.x * kWarps;
    for (int idx = (int)blockIdx.x * kWarps + (int)(threadIdx.x >> 5); idx < mp.warp_off[mp.ng]; idx += nwarps) {
        int gi = 0;
        while (idx >= mp.warp_off[gi + 1]) ++gi;
        const StepParams<P, W> &p = mp.g[gi];
        const unsigned active = p.stop ? (p.active & ~*p.stop) : p.active;
        if (p.stop && active == 0 && p.pend == 0) continue;
        short_chunk<P, W, false>(p, ld_stream4(&p.chunk_desc[p.num_long_chunks + idx - mp.warp_off[gi]].x), active);
    }
}

// Per-round sums, level 1: CTA j adds item slots [j per, (j+1) per) -- thread
// t every kThreads-th slot, then a fixed shuffle tree and the warps in order.
template <int W>
__global__ void __launch_bounds__(kThreads) item_sum_kernel(const double *__restrict__ ipart, int64_t items,
                                                            int64_t per, double *out) {
    __shared__ double s_w[kWarps][2 * W];
    double v[2 * W];
#pragma unroll
    for (int q = 0; q < 2 * W; ++q) v[q] = 0.0;
    const int64_t i0 = (int64_t)blockIdx.x * per;
    const int64_t i1 = min(items, i0 + per);
    for (int64_t i = i0 + threadIdx.x; i < i1; i += kThreads)
#pragma unroll
        for (int q = 0; q < 2 * W; ++q) v[q] = __dadd_rn(v[q], ipart[i * 2 * W + q]);
#pragma unroll
    for (int q = 0; q < 2 * W; ++q)
        for (int o = 16; o > 0; o >>= 1) v[q] = __dadd_rn(v[q], __shfl_xor_sync(0xffffffffu, v[q], o));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < 2 * W; ++q) s_w[warp][q] = v[q];
    __syncthreads();
    if (threadIdx.x < 2 * W) {
        double t = s_w[0][threadIdx.x];
        for (int w = 1; w < kWarps; ++w) t = __dadd_rn(t, s_w[w][threadIdx.x]);
        out[(int64_t)blockIdx.x * 2 * W + threadIdx.x] = t;
    }
}

// Level 2 (one CTA): the level-1 sums in block order give the round's
// sum T and sum |T| per column; then the a-posteriori rule's test.
template <int W>
__global__ void item_final_kernel(const double *__restrict__ part, int nblk, double *red, const StopArgs a) {
    const int t = threadIdx.x;
    __shared__ double s_l1[W];
    if (t < 2 * W) {
        double v = 0.0;
        for (int j = 0; j < nblk; ++j) v = __dadd_rn(v, part[j * 2 * W + t]);
        red[t] = v;
        if (t >= W) s_l1[t - W] = v;
    }
    __syncthreads();
    if (t == 0 && a.decide) {
        unsigned stop = *a.stop;
        for (int b = 0; b < W; ++b) {
            if (!(a.decide >> b & 1u) || (stop >> b & 1u)) continue;
            const double m = a.maxl1[b] < s_l1[b] ? s_l1[b] : a.maxl1[b];
            a.maxl1[b] = m;
            const double E = a.err[b];
            const double EK = __dmul_rn(E, __dmul_rn(2.0, m));
            const double bound =
                a.normalize ? EK : __dadd_rn(EK, __ddiv_rn(__dmul_rn(__dadd_rn(1.0, EK), E), __dsub_rn(1.0, E)));
            if (bound < a.tol[b]) {
                stop |= 1u << b;
                a.stop_round[b] = a.k[b];
            }
        }
        *a.stop = stop;
    }
}

// CTAs of cheb_step_kernel<P, W> resident on the whole GPU at once (per
// instantiation, on the current device; computed on first use).
template <int P, int W, bool I>
static int resident_ctas() {
    static int per_sm = 0, sms = 0;
    if (per_sm == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cheb_step_kernel<P, W, I>, kThreads, 0);
        // The kernel's shared arrays take a few KB per CTA.  Left to itself the
        // driver configured more of each SM's L1/shared array as shared memory
        // than that: the smallest carveout (of 10, 15, ... 75%) that keeps the
        // same resident CTAs leaves the rest to L1 for the gathers (measured:
        // the FP64 round on the 16.7M-vertex Chung-Lu graph 2.3-3.1% faster
        // at 10%, DF64 2.1-2.7%; FP32 batches of 8 on the 4M graph 2.4% at 15%,
        // of 16 1%; FP32 single vectors and the lattice unchanged).  If none
        // keeps them, the default stays.
        if (per_sm > 0) {
            bool kept = false;
            for (int pct : {10, 15, 20, 25, 30, 40, 50, 60, 75}) {
                if (cudaFuncSetAttribute(cheb_step_kernel<P, W, I>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         pct) != cudaSuccess)
                    break;
                int after = 0;
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&after, cheb_step_kernel<P, W, I>, kThreads, 0);
                if (after >= per_sm) {
                    kept = true;
                    break;
                }
            }
            if (!kept)
                cudaFuncSetAttribute(cheb_step_kernel<P, W, I>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)cudaSharedmemCarveoutDefault);
        }
        cudaGetLastError();  // a refused hint is not an error of the solve
        if (per_sm < 1) per_sm = 1;
    }
    return per_sm * sms;
}

template <int P, int W>
static int resident_multi_ctas() {
    static int per_sm = 0, sms = 0;
    if (per_sm == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cheb_step_multi_kernel<P, W>, kThreads, 0);
        if (per_sm < 1) per_sm = 1;
    }
    return per_sm * sms;
}

// The kernel parameters of one graph's round.
template <int P, int W>
static void fill_params(const StepLaunch &s, StepParams<P, W> &p) {
    using A = typename Prec<P>::A;
    using S = typename Prec<P>::S;
    using R = typename Prec<P>::R;
    const cpaa_graph *g = s.g;
    p.hub_tiles = g->hub_tiles;
    p.num_hub_tiles = g->num_hub_tiles;
    p.hub_tile = g->hub_tile;
    p.hub_row_ptr = g->hub_row_ptr;
    p.hub_col = g->hub_col;
    p.long_part = reinterpret_cast<A *>(s.long_part);
    p.long_cnt = s.long_cnt ? s.long_cnt : g->long_cnt;
    p.sell_col = g->sell_col;
    p.chunk_desc = g->chunk_desc;
    p.num_chunks = g->num_chunks;
    p.num_long_chunks = g->num_long_chunks;
    p.n_hub = g->n_hub;
    p.n = g->n;
    const A *tab;  // rows: d, 1 / d, 2 / d
    if constexpr (P == CPAA_F64) {
        p.deg = g->deg64;
        p.inv_deg = s.power ? g->inv_deg64 : g->inv2_deg64;
        tab = g->tab64;
    } else if constexpr (P == CPAA_DF64) {
        p.deg = g->deg_df;
        p.inv_deg = s.power ? g->inv_deg_df : g->inv2_deg_df;
        tab = g->tab_df;
    } else {
        p.deg = g->deg32;
        p.inv_deg = s.power ? g->inv_deg32 : g->inv2_deg32;
        tab = g->tab32;
    }
    // the interval series reads its own scaled table
    p.deg16 = g->deg16;
    p.tab_deg = tab;
    p.tab_inv = s.interval ? static_cast<const A *>(s.ivtab) : tab + (size_t)(s.power ? 1 : 2) * g->tab_n;
    p.y_src = static_cast<const S *>(s.y_src);
    p.y_io = static_cast<S *>(s.y_io);
    p.rho = static_cast<R *>(s.rho);
    p.comp = static_cast<R *>(s.comp);
    p.ipart = s.ipart;
    p.stop = s.stop;
    for (int b = 0; b < W; ++b) {
        p.ck[b] = (A)s.ck[b];
        p.ck_prev[b] = (A)s.ck_prev[b];
    }
    p.pend = s.pend;
    p.defer = s.defer;
    p.active = s.active;
    p.reduce = s.reduce;
    p.first = s.first;
    p.power = s.power;
    p.interval = s.interval;
    p.ia = (A)s.ia;
    p.mb = (A)s.mb;
    p.front = s.front;
    p.front_full = s.front_full;
    p.front_entries = s.front_entries;
    p.front_limit = s.front_limit;
    p.front_hub_words = s.front_hub_words;
}

// The two fixed-order sum kernels of a round that takes sums.  The item
// slots are hub rows, then chunks; their split into blocks depends on the
// graph alone, so the sums are the same bits for every tile width.
template <int W>
static void launch_sums(const StepLaunch &s) {
    const cpaa_graph *g = s.g;
    const int64_t items = (int64_t)g->n_hub + g->num_chunks;
    const int nblk = (int)std::max<int64_t>(1, std::min<int64_t>(kSumBlocks, (items + kThreads - 1) / kThreads));
    const int64_t per = (items + nblk - 1) / nblk;
    item_sum_kernel<W><<<nblk, kThreads, 0, s.stream>>>(s.ipart, items, per, s.ipart2);
    item_final_kernel<W><<<1, 64, 0, s.stream>>>(s.ipart2, nblk, s.red, s.sa);
}

template <int P, int W, bool I>
static cudaError_t launch_typed(const StepLaunch &s) {
    const cpaa_graph *g = s.g;
    StepParams<P, W> p;
    fill_params<P, W>(s, p);
    // a small graph needs fewer CTAs than fit: one per CTA item plus one per
    // kWarps short chunks
    const int64_t needed = (int64_t)g->num_hub_tiles + g->num_long_chunks +
                           (g->num_chunks - g->num_long_chunks + kWarps - 1) / kWarps;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(resident_ctas<P, W, I>(), needed));
    cheb_step_kernel<P, W, I><<<grid, kThreads, 0, s.stream>>>(p);
    if (s.reduce) launch_sums<W>(s);
    return cudaGetLastError();
}

// One round of ng graphs (same precision and width, same stream) in one launch.
template <int P, int W>
static cudaError_t launch_multi_typed(const StepLaunch *sl, int ng) {
    MultiParams<P, W> mp;
    mp.ng = ng;
    mp.cta_off[0] = mp.warp_off[0] = 0;
    for (int i = 0; i < ng; ++i) {
        const cpaa_graph *g = sl[i].g;
        fill_params<P, W>(sl[i], mp.g[i]);
        mp.cta_off[i + 1] = mp.cta_off[i] + g->num_hub_tiles + g->num_long_chunks;
        mp.warp_off[i + 1] = mp.warp_off[i] + (g->num_chunks - g->num_long_chunks);
    }
    const int64_t needed = (int64_t)mp.cta_off[ng] + (mp.warp_off[ng] + kWarps - 1) / kWarps;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(resident_multi_ctas<P, W>(), needed));
    cheb_step_multi_kernel<P, W><<<grid, kThreads, 0, sl[0].stream>>>(mp);
    for (int i = 0; i < ng; ++i)
        if (sl[i].reduce) launch_sums<W>(sl[i]);
    return cudaGetLastError();
}

template <int P>
static cudaError_t launch_multi_w(const StepLaunch *sl, int ng) {
    switch (sl[0].width) {
        case 1: return launch_multi_typed<P, 1>(sl, ng);
        case 2: return launch_multi_typed<P, 2>(sl, ng);
        case 4: return launch_multi_typed<P, 4>(sl, ng);
        case 8: return launch_multi_typed<P, 8>(sl, ng);
        case 16: return launch_multi_typed<P, 16>(sl, ng);
    }
    return cudaErrorInvalidValue;
}

template <int P, bool I>
static cudaError_t launch_w(const StepLaunch &s) {
    switch (s.width) {
        case 1: return launch_typed<P, 1, I>(s);
        case 2: return launch_typed<P, 2, I>(s);
        case 4: return launch_typed<P, 4, I>(s);
        case 8: return launch_typed<P, 8, I>(s);
        case 16: return launch_typed<P, 16, I>(s);
    }
    return cudaErrorInvalidValue;
}

template <int P, bool I>
static void prepare_w(int width) {
    switch (width) {
        case 1: resident_ctas<P, 1, I>(); break;
        case 2: resident_ctas<P, 2, I>(); break;
        case 4: resident_ctas<P, 4, I>(); break;
        case 8: resident_ctas<P, 8, I>(); break;
        case 16: resident_ctas<P, 16, I>(); break;
    }
}

// Every round kernel of one form (I: the series on [lambda_lo, 1]) for the
// given precision and width.
template <bool I>
static cudaError_t launch_form(const StepLaunch &s) {
    switch (s.precision) {
        case CPAA_F64: return launch_w<CPAA_F64, I>(s);
        case CPAA_F32: return launch_w<CPAA_F32, I>(s);
        case CPAA_BF16: return launch_w<CPAA_BF16, I>(s);
        case CPAA_DF64: return launch_w<CPAA_DF64, I>(s);
    }
    return cudaErrorInvalidValue;
}

template <bool I>
static void prepare_form(int precision, int width) {
    switch (precision) {
        case CPAA_F64: prepare_w<CPAA_F64, I>(width); break;
        case CPAA_F32: prepare_w<CPAA_F32, I>(width); break;
        case CPAA_BF16: prepare_w<CPAA_BF16, I>(width); break;
        case CPAA_DF64: prepare_w<CPAA_DF64, I>(width); break;
    }
}

}  // namespace cpaa
