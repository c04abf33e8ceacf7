// clbm_step_fp32.cu -- instantiates the step kernel for FP32 storage.
#include "clbm_step.cuh"

namespace clbm {

cudaError_t launch_step_fp32(const StepArgs& a, cudaStream_t s) { return launch_step_format<float>(a, s); }

}  // namespace clbm
