// clbm_step_fp64.cu -- instantiates the step kernel for FP64 storage.
#include "clbm_step.cuh"

namespace clbm {

cudaError_t launch_step_fp64(const StepArgs& a, cudaStream_t s) { return launch_step_format<double>(a, s); }

}  // namespace clbm
