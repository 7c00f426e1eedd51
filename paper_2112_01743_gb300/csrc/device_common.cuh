// device_common.cuh -- number formats and the per-row epilogue arithmetic
// shared by the single-vector round kernel (step.cu) and the batched one
// (batch.cu).  Every rounding step is an explicit intrinsic, so both kernels
// produce bit-identical values for the same inputs.
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

// Gathered iterate: ld.global.nc, allocating in L1 (hub values repeat).
__device__ __forceinline__ double load_y(const double *p) { return __ldg(p); }
__device__ __forceinline__ float load_y(const float *p) { return __ldg(p); }
__device__ __forceinline__ float load_y(const __nv_bfloat16 *p) { return __bfloat162float(__ldg(p)); }

__device__ __forceinline__ double to_acc(double v) { return v; }
__device__ __forceinline__ float to_acc(float v) { return v; }
__device__ __forceinline__ float to_acc(__nv_bfloat16 v) { return __bfloat162float(v); }

__device__ __forceinline__ void store_y(double *p, double v) { *p = v; }
__device__ __forceinline__ void store_y(float *p, float v) { *p = v; }
__device__ __forceinline__ void store_y(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
__device__ __forceinline__ double round_y(double v, const double *) { return v; }
__device__ __forceinline__ float round_y(float v, const float *) { return v; }
__device__ __forceinline__ float round_y(float v, const __nv_bfloat16 *) {
    return __bfloat162float(__float2bfloat16_rn(v));
}

// Streaming loads/stores (read or written once per round: evict first).
__device__ __forceinline__ int ld_stream(const int32_t *p) { return __ldcs(p); }
__device__ __forceinline__ int4 ld_stream4(const int32_t *p) { return __ldcs(reinterpret_cast<const int4 *>(p)); }
template <class T> __device__ __forceinline__ T ld_once(const T *p) { return __ldcs(p); }
template <class T> __device__ __forceinline__ void st_once(T *p, T v) { __stcs(p, v); }

// Explicitly rounded arithmetic (no contraction differences between kernels).
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
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
