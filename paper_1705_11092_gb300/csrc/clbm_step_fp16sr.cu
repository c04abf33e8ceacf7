// clbm_step_fp16sr.cu -- instantiates the step kernel for FP16 storage with
// stochastic rounding of the step's stores (clbm_set_rounding).
#include "clbm_step.cuh"

namespace clbm {

cudaError_t launch_step_fp16sr(const StepArgs& a, cudaStream_t s) { return launch_step_format<HalfSR>(a, s); }

}  // namespace clbm
