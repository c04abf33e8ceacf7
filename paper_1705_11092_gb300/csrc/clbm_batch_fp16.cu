// clbm_batch_fp16.cu -- instantiates the batched step kernels for FP16 storage.
#include "clbm_step.cuh"

namespace clbm {

cudaError_t launch_batch_step_fp16(const BatchLaunch& b, cudaStream_t s) {
    return launch_batch_format<__half>(b, s);
}

}  // namespace clbm
