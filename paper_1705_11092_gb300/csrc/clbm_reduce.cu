// clbm_reduce.cu -- deterministic FP64 reductions over the fluid nodes:
// total mass and momentum (Eq. 11, 15), the NaN/Inf watchdog, and the
// relative L2 velocity error E_2 of Eq. 24 (Fei & Luo, arXiv:1705.11092).
//
// Two passes with a fixed shape: a fixed grid of blocks, each summing a fixed
// set of nodes in a fixed order into one partial per block (global scratch),
// then one block summing the partials in a fixed tree order.  The result does
// not depend on scheduling.
#include "clbm_device.cuh"
#include "clbm_internal.h"

namespace clbm {

constexpr int kReduceBlocks = 608;    // 4 x 152 SMs
constexpr int kReduceThreads = 256;
constexpr int kLanes = 4;             // values reduced together

int reduce_partials_count() { return kReduceBlocks; }

template <class S>
__device__ __forceinline__ double dev_at(const StepArgs& a, int i, long long row_off, int x) {
    const S* p = static_cast<const S*>(a.src) + i * a.geo.plane + row_off + x;
    uint32_t w[4] = {0u, 0u, 0u, 0u};
    if constexpr (sizeof(S) == 8) {
        const unsigned long long v = *reinterpret_cast<const unsigned long long*>(p);
        w[0] = (uint32_t)v; w[1] = (uint32_t)(v >> 32);
    } else if constexpr (sizeof(S) == 4) {
        w[0] = *reinterpret_cast<const uint32_t*>(p);
    } else {
        w[0] = *reinterpret_cast<const unsigned short*>(p);
    }
    return (double)Fmt<S>::get(w, 0) * a.inv_scale;
}

template <class C>
__device__ __forceinline__ void force_d(const StepArgs& a, int x, int y, double& Fx, double& Fy) {
    const C* F = static_cast<const C*>(a.force);
    switch (a.force_kind) {
        case 1: Fx = F[2 * y]; Fy = F[2 * y + 1]; break;
        case 2: Fx = F[2 * x]; Fy = F[2 * x + 1]; break;
        case 3: {
            const long long k = 2 * ((long long)y * a.geo.nx + x);
            Fx = F[k]; Fy = F[k + 1];
            break;
        }
        case 4: {
            C fx, fy;
            sc_force_node<C>(static_cast<const C*>(a.psi), a.geo.pitch, a.geo.nx, a.geo.ny, x, y,
                             (C)a.sc_g, fx, fy);
            Fx = fx;
            Fy = fy;
            break;
        }
        default: Fx = a.fx; Fy = a.fy; break;
    }
}

// block-level fixed-order tree sum of kLanes values per thread
__device__ __forceinline__ void block_sum(double (&v)[kLanes], double* out) {
    __shared__ double sh[kLanes][kReduceThreads];
#pragma unroll
    for (int k = 0; k < kLanes; ++k) sh[k][threadIdx.x] = v[k];
    __syncthreads();
    for (int s = kReduceThreads / 2; s > 0; s >>= 1) {
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

// kind 0: (rho, rho ux, rho uy, nonfinite count); kind 1: (err^2, ref^2, 0, nonfinite)
template <class S>
__global__ void __launch_bounds__(kReduceThreads)
reduce_pass1(const StepArgs a, int kind, const double* ua, const double* va, double* partials) {
    using C = typename Fmt<S>::C;
    const long long n = (long long)a.geo.nx * a.geo.ny;
    const long long per = (n + gridDim.x - 1) / gridDim.x;
    const long long beg = per * blockIdx.x;
    const long long end = min(n, beg + per);
    double acc[kLanes] = {0.0, 0.0, 0.0, 0.0};
    for (long long p = beg + threadIdx.x; p < end; p += blockDim.x) {
        const int y = (int)(p / a.geo.nx), x = (int)(p - (long long)y * a.geo.nx);
        const long long roff = (long long)y * a.geo.pitch;
        const long long q = roff + x;
        if (a.sbits && ((a.sbits[q >> 3] >> (q & 7)) & 1u)) continue;
        double dr = 0.0, jx = 0.0, jy = 0.0;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const double g = dev_at<S>(a, i, roff, x);
            dr += g;
            jx += ex_of(i) * g;
            jy += ey_of(i) * g;
        }
        double Fx, Fy;
        force_d<C>(a, x, y, Fx, Fy);
        const double rho = a.rho0 + dr;
        const double mx = jx - 0.5 * Fx, my = jy - 0.5 * Fy;    // rho u (Eq. 15)
        const bool bad = !isfinite(rho) || !isfinite(mx) || !isfinite(my);
        if (kind == 0) {
            acc[0] += rho;
            acc[1] += mx;
            acc[2] += my;
        } else {
            const double u = mx / rho, v = my / rho;
            const double du = u - ua[p], dv = v - va[p];
            acc[0] += du * du + dv * dv;
            acc[1] += ua[p] * ua[p] + va[p] * va[p];
        }
        acc[3] += bad ? 1.0 : 0.0;
    }
    block_sum(acc, partials + (long long)blockIdx.x * kLanes);
}

__global__ void __launch_bounds__(kReduceThreads)
reduce_pass2(const double* partials, int count, double* out) {
    double acc[kLanes] = {0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < count; b += blockDim.x) {
#pragma unroll
        for (int k = 0; k < kLanes; ++k) acc[k] += partials[(long long)b * kLanes + k];
    }
    block_sum(acc, out);
}

template <class S>
static cudaError_t reduce_t(const StepArgs& a, int kind, const double* ua, const double* va,
                           double* partials, double* out, cudaStream_t s) {
    reduce_pass1<S><<<kReduceBlocks, kReduceThreads, 0, s>>>(a, kind, ua, va, partials);
    reduce_pass2<<<1, kReduceThreads, 0, s>>>(partials, kReduceBlocks, out);
    return cudaGetLastError();
}

static cudaError_t reduce_any(const StepArgs& a, int format, int kind, const double* ua,
                              const double* va, double* partials, double* out, cudaStream_t s) {
    switch (format) {
        case 0: return reduce_t<double>(a, kind, ua, va, partials, out, s);
        case 1: return reduce_t<float>(a, kind, ua, va, partials, out, s);
        case 2: return reduce_t<__half>(a, kind, ua, va, partials, out, s);
        case 3: return reduce_t<__nv_bfloat16>(a, kind, ua, va, partials, out, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_reduce_moments(const StepArgs& a, int format, double* partials, double* out,
                                  cudaStream_t s) {
    return reduce_any(a, format, 0, nullptr, nullptr, partials, out, s);
}

cudaError_t launch_reduce_l2(const StepArgs& a, int format, const double* ua, const double* va,
                             double* partials, double* out, cudaStream_t s) {
    return reduce_any(a, format, 1, ua, va, partials, out, s);
}

}  // namespace clbm
