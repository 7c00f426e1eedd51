// step_interval.cu -- the round launches of the Chebyshev series on a narrower
// interval [lambda_lo, 1] (Sec. 2.2's general-interval series): the kernels of
// step_impl.cuh with the shifted recurrence in their epilogue
// (interval_iterate, device_common.cuh).
#include "step_impl.cuh"

namespace cpaa {

void prepare_step_interval(int precision, int width) { prepare_form<true>(precision, width); }

cudaError_t launch_step_interval(const StepLaunch &s) { return launch_form<true>(s); }

// ia 2 / d by degree: the product the round kernel takes (row_factor) for the
// rows whose factor it reads from the per-vertex words, so both give the same
// bits.  A is the solve's arithmetic type.
template <class A>
__global__ void ivtab_kernel(const A *__restrict__ inv2tab, int n, double ia, A *out) {
    for (int d = blockIdx.x * blockDim.x + threadIdx.x; d < n; d += gridDim.x * blockDim.x)
        out[d] = mul_rn((A)ia, inv2tab[d]);
}

cudaError_t launch_ivtab(const cpaa_graph *g, int precision, double ia, void *out, cudaStream_t st) {
    const int T = g->tab_n;
    const unsigned blocks = (unsigned)std::min(64, (T + 255) / 256);
    switch (precision) {
        case CPAA_F64:
            ivtab_kernel<double><<<blocks, 256, 0, st>>>(g->tab64 + 2 * (size_t)T, T, ia, (double *)out);
            break;
        case CPAA_F32:
        case CPAA_BF16:
            ivtab_kernel<float><<<blocks, 256, 0, st>>>(g->tab32 + 2 * (size_t)T, T, ia, (float *)out);
            break;
        case CPAA_DF64:
            ivtab_kernel<df><<<blocks, 256, 0, st>>>(g->tab_df + 2 * (size_t)T, T, ia, (df *)out);
            break;
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace cpaa
