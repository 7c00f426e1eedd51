// step.cu -- the round launches of the paper's series on [-1, 1] (Algorithm 1)
// and the server's fused multi-graph round; the kernels are in step_impl.cuh,
// and the series on a narrower interval is launched from step_interval.cu
// (its kernels are separate instantiations, so that neither form's registers
// depend on the other's epilogue).
#include "step_impl.cuh"

namespace cpaa {

cudaError_t launch_step_multi(const StepLaunch *sl, int ng) {
    if (ng < 1 || ng > kMaxFused) return cudaErrorInvalidValue;
    for (int i = 1; i < ng; ++i)
        if (sl[i].precision != sl[0].precision || sl[i].width != sl[0].width || sl[i].stream != sl[0].stream)
            return cudaErrorInvalidValue;
    switch (sl[0].precision) {
        case CPAA_F64: return launch_multi_w<CPAA_F64>(sl, ng);
        case CPAA_F32: return launch_multi_w<CPAA_F32>(sl, ng);
        case CPAA_BF16: return launch_multi_w<CPAA_BF16>(sl, ng);
        case CPAA_DF64: return launch_multi_w<CPAA_DF64>(sl, ng);
    }
    return cudaErrorInvalidValue;
}

// Runs the one-time occupancy queries of a round kernel, so that a later
// launch issues no other CUDA call (as a stream capture wants).
void prepare_step(int precision, int width, bool interval) {
    if (interval) prepare_step_interval(precision, width);
    else prepare_form<false>(precision, width);
}

cudaError_t launch_step(const StepLaunch &s) {
    if (s.interval) return launch_step_interval(s);
    return launch_form<false>(s);
}

}  // namespace cpaa
