// clbm_batch_fp64.cu -- instantiates the batched step kernels for FP64 storage.
#include "clbm_step.cuh"

namespace clbm {

cudaError_t launch_batch_step_fp64(const BatchLaunch& b, cudaStream_t s) {
    return launch_batch_format<double>(b, s);
}

}  // namespace clbm
