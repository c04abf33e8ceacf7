// clbm_step_fp16.cu -- instantiates the step kernel for FP16 storage.
#include "clbm_step.cuh"

namespace clbm {

cudaError_t launch_step_fp16(const StepArgs& a, cudaStream_t s) { return launch_step_format<__half>(a, s); }

}  // namespace clbm
