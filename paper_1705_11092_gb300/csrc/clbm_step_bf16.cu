// clbm_step_bf16.cu -- instantiates the step kernel for BF16 storage.
#include "clbm_step.cuh"

namespace clbm {

cudaError_t launch_step_bf16(const StepArgs& a, cudaStream_t s) { return launch_step_format<__nv_bfloat16>(a, s); }

}  // namespace clbm
