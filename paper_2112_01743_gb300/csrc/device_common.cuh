// device_common.cuh -- number formats (FP64, FP32, BF16 storage, and the
// double-float pairs of DF64) and the per-row arithmetic of the round kernel
// (step.cu), which serves single vectors, batched tiles and the server alike.
// Every rounding step is an explicit intrinsic, so a value is the same bits
// whichever of them computed it.
#pragma once

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
template <> struct Prec<CPAA_DF64> {
    using S = df;
    using A = df;
    using R = df;
    static constexpr bool kKahan = false;  // the pair already carries the low bits
};

// ---------------------------------------------------------------------------
// Double-float arithmetic on the FP32 pipes.  The building blocks are the
// classical error-free transformations: Knuth's two-sum (s + e = a + b
// exactly), Dekker's fast two-sum (the same when |a| >= |b|) and the product
// a b = p + e with e from one fused multiply-add.  A double-float sum adds the
// high and the low parts with two-sums and renormalises twice, which keeps
// about 2^-47 relative accuracy even under cancellation (the recurrence
// subtracts y_{k-1}); a product drops only the lo x lo term.  Every step is an
// explicitly rounded intrinsic, so the compiler cannot contract or reorder it.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}
__device__ __forceinline__ df df_add(df a, df b) {
    float s, e, t, f;
    two_sum(a.hi, b.hi, s, e);
    two_sum(a.lo, b.lo, t, f);
    e = __fadd_rn(e, t);
    fast_two_sum(s, e, s, e);
    e = __fadd_rn(e, f);
    fast_two_sum(s, e, s, e);
    return df(s, e);
}
__device__ __forceinline__ df df_mul(df a, df b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    float s;
    fast_two_sum(p, e, s, e);
    return df(s, e);
}
__device__ __forceinline__ df operator-(df a) { return df(-a.hi, -a.lo); }
__device__ __forceinline__ df operator+(df a, df b) { return df_add(a, b); }
__device__ __forceinline__ df &operator+=(df &a, df b) { return a = df_add(a, b); }
__device__ __forceinline__ df operator*(df a, df b) { return df_mul(a, b); }
__device__ __forceinline__ bool operator<(df a, df b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ double to_double(df v) { return __dadd_rn((double)v.hi, (double)v.lo); }
__device__ __forceinline__ double to_double(double v) { return v; }
__device__ __forceinline__ double to_double(float v) { return (double)v; }
// ---------------------------------------------------------------------------

__device__ __forceinline__ double to_acc(double v) { return v; }
__device__ __forceinline__ df to_acc(df v) { return v; }
__device__ __forceinline__ float to_acc(float v) { return v; }
__device__ __forceinline__ float to_acc(__nv_bfloat16 v) { return __bfloat162float(v); }

__device__ __forceinline__ void store_y(double *p, double v) { *p = v; }
__device__ __forceinline__ void store_y(df *p, df v) { *p = v; }
__device__ __forceinline__ df round_y(df v, const df *) { return v; }
__device__ __forceinline__ void store_y(float *p, float v) { *p = v; }
__device__ __forceinline__ void store_y(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
__device__ __forceinline__ double round_y(double v, const double *) { return v; }
__device__ __forceinline__ float round_y(float v, const float *) { return v; }
__device__ __forceinline__ float round_y(float v, const __nv_bfloat16 *) {
    return __bfloat162float(__float2bfloat16_rn(v));
}

// Streaming loads/stores (read or written once per round: evict first).
__device__ __forceinline__ int4 ld_stream4(const int32_t *p) { return __ldcs(reinterpret_cast<const int4 *>(p)); }
template <class T> __device__ __forceinline__ T ld_once(const T *p) { return __ldcs(p); }
__device__ __forceinline__ df ld_once(const df *p) {
    const float2 v = __ldcs(reinterpret_cast<const float2 *>(p));
    return df(v.x, v.y);
}
// Small read-only tables read by every round (kept in cache).
template <class T> __device__ __forceinline__ T ld_ro(const T *p) { return __ldg(p); }
__device__ __forceinline__ df ld_ro(const df *p) {
    const float2 v = __ldg(reinterpret_cast<const float2 *>(p));
    return df(v.x, v.y);
}

// Explicitly rounded arithmetic (no contraction differences between kernels).
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ df add_rn(df a, df b) { return df_add(a, b); }
__device__ __forceinline__ df sub_rn(df a, df b) { return df_add(a, -b); }
__device__ __forceinline__ df mul_rn(df a, df b) { return df_mul(a, b); }
__device__ __forceinline__ df fma_rn(df a, df b, df c) { return df_add(df_mul(a, b), c); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// The new iterate of one row from its gathered sum s (Sec. 4.1), given
// inv2 = 2 / d: k = 1: y = s / d; k >= 2: y = 2 s / d - y_old (one fused
// multiply-add: 2 s (1/d) and s (2/d) are the same exact product); rounded to
// storage.
template <int P, class S = typename Prec<P>::S>
__device__ __forceinline__ typename Prec<P>::A new_iterate(typename Prec<P>::A s, typename Prec<P>::A inv2,
                                                           typename Prec<P>::A y_old, int first) {
    using A = typename Prec<P>::A;
    const A y = first ? mul_rn(mul_rn(s, inv2), A(0.5)) : fma_rn(s, inv2, -y_old);
    return round_y(y, (const S *)nullptr);
}

// The same on the interval [lambda_lo, 1] (Sec. 2.2's general interval): the
// recurrence on Q = (P - mid I) / half, scaled by D^-1 like the rest, with
// iv = ia 2 / d (ia = 1 / half; the caller's factor), mb = -2 mid / half and
// y_cur the row's current iterate y_k[u]:
//   k = 1:  y_1 = ia (s / d) - (mid / half) y_0 = (iv s) / 2 + (mb / 2) y_0
//   k >= 2: y_{k+1} = ia (2 s / d) - 2 (mid / half) y_k - y_{k-1}
//                   = iv s + (mb y_k - y_{k-1})      (two fused multiply-adds)
template <int P, class S = typename Prec<P>::S>
__device__ __forceinline__ typename Prec<P>::A interval_iterate(typename Prec<P>::A s, typename Prec<P>::A iv,
                                                                typename Prec<P>::A y_cur,
                                                                typename Prec<P>::A y_old, int first,
                                                                typename Prec<P>::A mb) {
    using A = typename Prec<P>::A;
    const A y = first ? fma_rn(mul_rn(mb, A(0.5)), y_cur, mul_rn(mul_rn(s, iv), A(0.5)))
                      : fma_rn(s, iv, fma_rn(mb, y_cur, -y_old));
    return round_y(y, (const S *)nullptr);
}

// One power-method round in scaled space (the paper's SPI baseline, Sec. 5.1):
// x' = c P x + (1 - c) p  ->  y' = c s / d + q,  q = (1 - c) p / d.
template <int P, class S = typename Prec<P>::S>
__device__ __forceinline__ typename Prec<P>::A power_iterate(typename Prec<P>::A s, typename Prec<P>::A inv,
                                                             typename Prec<P>::A c, typename Prec<P>::R q) {
    using A = typename Prec<P>::A;
    const A y = fma_rn(mul_rn(c, s), inv, (A)q);
    return round_y(y, (const S *)nullptr);
}

// rho += c_k y (Kahan-compensated for the FP32 accumulator).
template <int P>
__device__ __forceinline__ void accumulate(typename Prec<P>::R &rr, typename Prec<P>::R &cmp,
                                           typename Prec<P>::A ck, typename Prec<P>::A y) {
    using R = typename Prec<P>::R;
    if constexpr (Prec<P>::kKahan) {
        const R t1 = fma_rn(ck, y, -cmp);
        const R t = add_rn(rr, t1);
        cmp = sub_rn(sub_rn(t, rr), t1);
        rr = t;
    } else {
        rr = fma_rn(ck, y, rr);
    }
}

}  // namespace cpaa
