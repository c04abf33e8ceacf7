// clbm_micro.cu -- clbm_alu_throughput: measured FMA throughput of the GPU
// for the arithmetic roofs of the step kernels (the FP64 step is bound by
// FP64 arithmetic, the FP32-compute steps come near the FP32 pipe).  No
// counterpart in the paper; a measurement, not part of the time step.
//
// Each thread runs 8 independent chains of fused multiply-adds (enough to
// cover the pipe latency at full occupancy); a launch is timed with CUDA
// events and repeated until the requested time has passed.
#include <cstdint>

#include "../../include/clbm.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kBlocksPerSM = 8;     // 2048 threads per SM

__device__ __forceinline__ double fma64(double a, double b, double c) {
    double r;
    asm volatile("fma.rn.f64 %0, %1, %2, %3;" : "=d"(r) : "d"(a), "d"(b), "d"(c));
    return r;
}
__device__ __forceinline__ double add64(double a, double b) {
    double r;
    asm volatile("add.rn.f64 %0, %1, %2;" : "=d"(r) : "d"(a), "d"(b));
    return r;
}
__device__ __forceinline__ double mul64(double a, double b) {
    double r;
    asm volatile("mul.rn.f64 %0, %1, %2;" : "=d"(r) : "d"(a), "d"(b));
    return r;
}
__device__ __forceinline__ float fma32(float a, float b, float c) {
    float r;
    asm volatile("fma.rn.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ unsigned long long fma32x2(unsigned long long a, unsigned long long b,
                                                      unsigned long long c) {
    unsigned long long r;
    asm volatile("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// KIND 0: FP64 FMA, 1: FP32 FMA, 2: packed FP32x2 FMA, 3: FP64 add,
// 4: FP64 multiply.  Values stay bounded (|b| < 1, alternating signs for
// the add); the sum is written so the chains are not removed.
template <int KIND>
__global__ void __launch_bounds__(kThreads) alu_chains(int iters, double seed, double* out) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    double acc = 0.0;
    if constexpr (KIND == 0 || KIND == 3 || KIND == 4) {
        double a[kChains];
        const double b = 0.999999 - 1e-9 * (tid & 7), c = seed;
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = 1e-3 * (k + 1);
        for (int i = 0; i < iters; ++i) {
            const double d = (i & 1) ? c : -c;
#pragma unroll
            for (int k = 0; k < kChains; ++k) {
                if constexpr (KIND == 0) a[k] = fma64(a[k], b, c);
                else if constexpr (KIND == 3) a[k] = add64(a[k], d);
                else a[k] = mul64(a[k], b);
            }
        }
#pragma unroll
        for (int k = 0; k < kChains; ++k) acc += a[k];
    } else if constexpr (KIND == 1) {
        float a[kChains];
        const float b = 0.999999f - 1e-7f * (tid & 7), c = (float)seed;
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = 1e-3f * (k + 1);
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = fma32(a[k], b, c);
        }
#pragma unroll
        for (int k = 0; k < kChains; ++k) acc += a[k];
    } else {
        unsigned long long a[kChains];
        const float bf = 0.999999f - 1e-7f * (tid & 7), cf = (float)seed;
        const unsigned long long b = ((unsigned long long)__float_as_uint(bf) << 32) | __float_as_uint(bf);
        const unsigned long long c = ((unsigned long long)__float_as_uint(cf) << 32) | __float_as_uint(cf);
#pragma unroll
        for (int k = 0; k < kChains; ++k) {
            const uint32_t v = __float_as_uint(1e-3f * (k + 1));
            a[k] = ((unsigned long long)v << 32) | v;
        }
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = fma32x2(a[k], b, c);
        }
#pragma unroll
        for (int k = 0; k < kChains; ++k)
            acc += __uint_as_float((uint32_t)a[k]) + __uint_as_float((uint32_t)(a[k] >> 32));
    }
    out[tid] = acc;
}

template <int KIND>
cudaError_t launch_chains(int blocks, int iters, double* out, cudaStream_t s) {
    alu_chains<KIND><<<blocks, kThreads, 0, s>>>(iters, 1e-9, out);
    return cudaGetLastError();
}

cudaError_t launch_kind(int kind, int blocks, int iters, double* out, cudaStream_t s) {
    switch (kind) {
        case 0: return launch_chains<0>(blocks, iters, out, s);
        case 1: return launch_chains<1>(blocks, iters, out, s);
        case 2: return launch_chains<2>(blocks, iters, out, s);
        case 3: return launch_chains<3>(blocks, iters, out, s);
        default: return launch_chains<4>(blocks, iters, out, s);
    }
}

}  // namespace

extern "C" int clbm_alu_throughput(int kind, double seconds, double* ops_per_second) {
    if (kind < 0 || kind > 4 || !(seconds > 0.0) || seconds > 60.0 || !ops_per_second) return CLBM_ERR_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return CLBM_ERR_CUDA;
    const int blocks = sms * kBlocksPerSM;
    double* out = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int st = CLBM_OK;
    if (cudaMalloc(&out, (size_t)blocks * kThreads * sizeof(double)) != cudaSuccess) return CLBM_ERR_OOM;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        st = CLBM_ERR_CUDA;
    }
    // calibrate the launch to about 50 ms, then repeat it for `seconds`
    int iters = 1 << 12;
    float ms = 0.0f;
    for (int round = 0; st == CLBM_OK && round < 12; ++round) {
        if (launch_kind(kind, blocks, iters, out, s) != cudaSuccess ||      // warm
            cudaEventRecord(e0, s) != cudaSuccess || launch_kind(kind, blocks, iters, out, s) != cudaSuccess ||
            cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            st = CLBM_ERR_CUDA;
            break;
        }
        if (ms > 20.0f || iters >= (1 << 24)) break;
        iters *= 4;
    }
    if (st == CLBM_OK) {
        const int per = (int)((double)iters * 50.0 / (ms > 0.0f ? ms : 1.0f));
        iters = per < (1 << 12) ? (1 << 12) : (per > (1 << 26) ? (1 << 26) : per);
        const int reps = (int)(seconds * 1e3 / 50.0) + 1;
        if (cudaEventRecord(e0, s) != cudaSuccess) st = CLBM_ERR_CUDA;
        for (int r = 0; st == CLBM_OK && r < reps; ++r)
            if (launch_kind(kind, blocks, iters, out, s) != cudaSuccess) st = CLBM_ERR_CUDA;
        if (st == CLBM_OK && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                              cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
            st = CLBM_ERR_CUDA;
        if (st == CLBM_OK) {
            // operations: lanes x chains x iterations (x2 for the packed form)
            const double ops = (double)blocks * kThreads * kChains * iters * reps * (kind == 2 ? 2.0 : 1.0);
            *ops_per_second = ops / (ms * 1e-3);
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    cudaFree(out);
    return st;
}
