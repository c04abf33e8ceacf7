// clbm_batch_bf16.cu -- instantiates the batched step kernels for BF16 storage.
#include "clbm_step.cuh"

namespace clbm {

cudaError_t launch_batch_step_bf16(const BatchLaunch& b, cudaStream_t s) {
    return launch_batch_format<__nv_bfloat16>(b, s);
}

}  // namespace clbm
