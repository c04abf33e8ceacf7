// clbm_batch_fp32.cu -- instantiates the batched step kernels for FP32 storage.
#include "clbm_step.cuh"

namespace clbm {

cudaError_t launch_batch_step_fp32(const BatchLaunch& b, cudaStream_t s) {
    return launch_batch_format<float>(b, s);
}

}  // namespace clbm
