// clbm_noalloc.cu -- clbm_reduce_noalloc: the FP64 mass/momentum reduction
// for callers that cannot allocate device memory.
//
// Who needs it: code that must not call cudaMalloc -- an embedding framework
// that owns every device byte through its own pool or budget, a latency-
// critical loop where an allocation (and the device synchronisation it may
// imply) is not allowed, or a caller that never creates a clbm context
// because creating one allocates.  Such a caller holds the populations
// itself and passes them in; this entry point allocates nothing.
//
// Its scratch (one partial-sum slot per lattice row) is a file-scope device
// array of fixed size: the driver commits it on a device when it loads the
// library's device code there (with lazy loading, CUDA's default, at the
// first call that needs it), and it stays until the context goes.  Host
// code cannot use the array's name as a device address; the address is
// fetched with cudaGetSymbolAddress, with the device current, once per
// device and context, and handed to the kernels.
#include <cuda.h>

#include <cmath>
#include <mutex>

#include "../../include/clbm.h"
#include "clbm_device.cuh"

namespace {

constexpr int kMaxRows = CLBM_NOALLOC_MAX_ROWS;   // 65536 rows
constexpr int kLanes = 4;                          // mass, momentum x, y, non-finite
constexpr int kThreads = 256;
constexpr int kMaxDevices = 64;

// 65536 x 4 doubles = 2 MiB, the whole scratch of this entry point.
static __device__ __align__(256) double noalloc_scratch[kMaxRows * kLanes];

std::mutex g_setup_mutex;
// per device: the context the address was looked up in, and the address
struct ScratchSlot {
    CUcontext ctx = nullptr;
    double* ptr = nullptr;
};
ScratchSlot g_scratch[kMaxDevices];

// fixed-order tree sum of kLanes values over the block
__device__ __forceinline__ void block_sum4(double (&v)[kLanes], double* out) {
    __shared__ double sh[kLanes][kThreads];
#pragma unroll
    for (int k = 0; k < kLanes; ++k) sh[k][threadIdx.x] = v[k];
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
#pragma unroll
            for (int k = 0; k < kLanes; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < kLanes; ++k) out[k] = sh[k][0];
    }
}

// Pass 1: each block sums whole rows (rows b, b + gridDim.x, ...) and
// overwrites that row's slot, so no slot needs clearing beforehand.
__global__ void __launch_bounds__(kThreads)
noalloc_rows(const double* f, int nx, int ny, double fx, double fy, const uint8_t* solid,
             double* rows) {
    const long long n = (long long)nx * ny;
    for (int y = blockIdx.x; y < ny; y += gridDim.x) {
        double acc[kLanes] = {0.0, 0.0, 0.0, 0.0};
        for (int x = threadIdx.x; x < nx; x += blockDim.x) {
            const long long p = (long long)y * nx + x;
            if (solid && solid[p]) continue;
            double r = 0.0, jx = 0.0, jy = 0.0;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const double v = f[i * n + p];
                r += v;
                jx += clbm::ex_of(i) * v;
                jy += clbm::ey_of(i) * v;
            }
            // Eq. 11 and Eq. 15 on the post-collision state: rho = sum f*,
            // rho u = sum f* e - F/2
            const double mx = jx - 0.5 * fx, my = jy - 0.5 * fy;
            acc[0] += r;
            acc[1] += mx;
            acc[2] += my;
            acc[3] += (isfinite(r) && isfinite(mx) && isfinite(my)) ? 0.0 : 1.0;
        }
        block_sum4(acc, rows + (long long)y * kLanes);
        __syncthreads();
    }
}

// Pass 2: one block sums the row slots in a fixed order into out[4].
__global__ void __launch_bounds__(kThreads) noalloc_total(const double* rows, int ny, double* out) {
    double acc[kLanes] = {0.0, 0.0, 0.0, 0.0};
    for (int y = threadIdx.x; y < ny; y += blockDim.x) {
#pragma unroll
        for (int k = 0; k < kLanes; ++k) acc[k] += rows[(long long)y * kLanes + k];
    }
    block_sum4(acc, out);
}

// The context current on this thread (the driver's cuCtxGetCurrent, found
// through the runtime so that the library needs no link to the driver).
CUcontext current_context() {
    using Fn = CUresult (*)(CUcontext*);
    static Fn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !p)
            return nullptr;
        fn = reinterpret_cast<Fn>(p);
    }
    CUcontext c = nullptr;
    return fn(&c) == CUDA_SUCCESS ? c : nullptr;
}

// The scratch's device address on the current device, looked up on the
// first call there and again whenever the device's context has changed
// (after cudaDeviceReset, the module and its array may sit elsewhere).
int scratch_for_current_device(double** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CLBM_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return CLBM_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    ScratchSlot& slot = g_scratch[dev];
    const CUcontext ctx = current_context();
    if (!slot.ptr || !ctx || ctx != slot.ctx) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, noalloc_scratch) != cudaSuccess || !p) return CLBM_ERR_CUDA;
        slot.ptr = static_cast<double*>(p);
        slot.ctx = current_context();    // the runtime makes the primary context current
    }
    *out = slot.ptr;
    return CLBM_OK;
}

}  // namespace

extern "C" int clbm_reduce_noalloc(const double* f, int nx, int ny, double fx, double fy,
                                   const uint8_t* solid, double* out, void* stream) {
    if (!f || !out || nx < 1 || ny < 1) return CLBM_ERR_ARG;
    if (ny > kMaxRows) return CLBM_ERR_ARG;                      // beyond the scratch
    if (!std::isfinite(fx) || !std::isfinite(fy)) return CLBM_ERR_ARG;
    double* rows = nullptr;
    const int st = scratch_for_current_device(&rows);
    if (st != CLBM_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int grid = ny < 1216 ? ny : 1216;                      // 8 blocks per SM on 152 SMs
    // each launch reports its own status (an error left over from the
    // caller's earlier work is neither taken for ours nor cleared)
    void* a1[] = {(void*)&f, (void*)&nx, (void*)&ny, (void*)&fx, (void*)&fy, (void*)&solid, (void*)&rows};
    if (cudaLaunchKernel((const void*)noalloc_rows, dim3(grid), dim3(kThreads), a1, 0, s) != cudaSuccess)
        return CLBM_ERR_CUDA;
    void* a2[] = {(void*)&rows, (void*)&ny, (void*)&out};
    if (cudaLaunchKernel((const void*)noalloc_total, dim3(1), dim3(kThreads), a2, 0, s) != cudaSuccess)
        return CLBM_ERR_CUDA;
    return CLBM_OK;
}
