// step_interval.cu -- the round launches of the Chebyshev series on a narrower
// interval [lambda_lo, 1] (Sec. 2.2's general-interval series): the kernels of
// step_impl.cuh with the shifted recurrence in their epilogue
// (interval_iterate, device_common.cuh).
#include "step_impl.cuh"

namespace cpaa {

void prepare_step_interval(int precision, int width) { prepare_form<true>(precision, width); }

cudaError_t launch_step_interval(const StepLaunch &s) { return launch_form<true>(s); }

}  // namespace cpaa
