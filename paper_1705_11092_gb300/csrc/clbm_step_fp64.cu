// clbm_step_fp64.cu -- instantiates the step kernel for FP64 storage.
#include "clbm_step.cuh"

namespace clbm {

cudaError_t launch_step_fp64(const StepArgs& a, cudaStream_t s) { return launch_step_format<double>(a, s); }

cudaError_t launch_batch_step_fp64(const BatchLaunch& b, cudaStream_t s) {
    return launch_batch_format<double>(b, s);
}

}  // namespace clbm
