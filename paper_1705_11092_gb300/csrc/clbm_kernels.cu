// clbm_kernels.cu -- the per-node kernels around the time step
// (initialisation, population get/set, window and macroscopic readout, the
// FP16 scale probe) and the per-format dispatch of the step kernel.
#include "clbm_step.cuh"

namespace clbm {

// ---------------------------------------------------------------------------
// per-node helper kernels (not on the time-step path)
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool node_solid(const StepArgs& a, int x, int y) {
    const long long q = (long long)y * a.geo.pitch + x;
    return a.sbits && ((a.sbits[q >> 3] >> (q & 7)) & 1u);
}

template <class S>
__device__ __forceinline__ void store_elem(const StepArgs& a, int i, int x, int y,
                                           typename Fmt<S>::C v) {
    using F = Fmt<S>;
    uint32_t w[4] = {0u, 0u, 0u, 0u};
    F::set(w, 0, v);
    S* p = static_cast<S*>(a.dst) + i * a.geo.plane + (long long)y * a.geo.pitch + x;
    if constexpr (sizeof(S) == 8) {
        *reinterpret_cast<unsigned long long*>(p) = ((unsigned long long)w[1] << 32) | w[0];
    } else if constexpr (sizeof(S) == 4) {
        *reinterpret_cast<uint32_t*>(p) = w[0];
    } else {
        *reinterpret_cast<unsigned short*>(p) = (unsigned short)(w[0] & 0xffffu);
    }
}

template <class S>
__device__ __forceinline__ double load_dev(const StepArgs& a, int i, int x, int y) {
    using F = Fmt<S>;
    const S* p = static_cast<const S*>(a.src) + i * a.geo.plane + (long long)y * a.geo.pitch + x;
    uint32_t w[4] = {0u, 0u, 0u, 0u};
    if constexpr (sizeof(S) == 8) {
        const unsigned long long v = *reinterpret_cast<const unsigned long long*>(p);
        w[0] = (uint32_t)v; w[1] = (uint32_t)(v >> 32);
    } else if constexpr (sizeof(S) == 4) {
        w[0] = *reinterpret_cast<const uint32_t*>(p);
    } else {
        w[0] = *reinterpret_cast<const unsigned short*>(p);
    }
    return (double)F::get(w, 0) * a.inv_scale;
}

// kind 0: equilibrium of (rho, ux, uy); kind 1: given FP64 populations,
// collided once; kind 2: given FP64 post-collision populations, stored as
// they are.
template <class S>
__global__ void prepare_kernel(const StepArgs a, int kind, const double* rho, const double* ux,
                               const double* uy, const double* f) {
    using F = Fmt<S>;
    using C = typename F::C;
    const long long n = (long long)a.geo.nx * a.geo.ny;
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int y = (int)(p / a.geo.nx), x = (int)(p - (long long)y * a.geo.nx);
    C g[9];
    if (node_solid(a, x, y)) {
#pragma unroll
        for (int i = 0; i < 9; ++i) store_elem<S>(a, i, x, y, C(0));
        return;
    }
    if (kind == 0) {
        const double r = rho ? rho[p] : 1.0;
        const double vx = ux ? ux[p] : 0.0, vy = uy ? uy[p] : 0.0;
        equilibrium_dev<C>((C)(r - a.rho0), (C)vx, (C)vy, (C)a.rho0, g);
    } else {
#pragma unroll
        for (int i = 0; i < 9; ++i) g[i] = (C)(f[i * n + p] - weight(i) * a.rho0);
    }
    if (kind == 2) {
#pragma unroll
        for (int i = 0; i < 9; ++i) store_elem<S>(a, i, x, y, F::encode(g[i], (C)a.scale));
        return;
    }
    C Fx, Fy;
    force_at<C>(a, x, y, Fx, Fy);
    const Coef<C> kc = coef_of<C>(a.relax, a.rho0);
    if (kc.m2)
        collide<C, true>(g, Fx, Fy, kc);
    else
        collide<C, false>(g, Fx, Fy, kc);
#pragma unroll
    for (int i = 0; i < 9; ++i) store_elem<S>(a, i, x, y, F::encode(g[i], (C)a.scale));
}

// pre = 0: the stored post-collision state f*(t).  pre = 1: the
// pre-collision state f(t+1) of the next step, pulled from it (Eq. 10):
// f_i(x) = f*_i(x - e_i), or f*_opp(i)(x) where x - e_i is solid (halfway
// bounce-back, Sec. 4A).  Solid nodes read as 0.
template <class S>
__global__ void get_populations_kernel(const StepArgs a, double* f, int pre) {
    const long long n = (long long)a.geo.nx * a.geo.ny;
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int y = (int)(p / a.geo.nx), x = (int)(p - (long long)y * a.geo.nx);
    const bool solid = node_solid(a, x, y);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        int xs = x, ys = y, is = i;
        if (pre) {
            xs = x - ex_of(i);
            ys = y - ey_of(i);
            xs = xs < 0 ? xs + a.geo.nx : (xs >= a.geo.nx ? xs - a.geo.nx : xs);
            ys = ys < 0 ? ys + a.geo.ny : (ys >= a.geo.ny ? ys - a.geo.ny : ys);
            if (node_solid(a, xs, ys)) {
                xs = x;
                ys = y;
                is = opp_of(i);
            }
        }
        f[i * n + p] = solid ? 0.0 : load_dev<S>(a, is, xs, ys) + weight(is) * a.rho0;
    }
}

// Decoded post-collision populations of a w-by-h window starting at (x0, y0),
// with periodic wrap: out[i][j][k] for node (x0 + k, y0 + j).
template <class S>
__global__ void window_kernel(const StepArgs a, int x0, int y0, int w, int h, double* out) {
    const long long n = (long long)w * h;
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int j = (int)(p / w), k = (int)(p - (long long)j * w);
    const int x = (int)(((long long)x0 + k) % a.geo.nx), y = (int)(((long long)y0 + j) % a.geo.ny);
    const bool solid = node_solid(a, x, y);
#pragma unroll
    for (int i = 0; i < 9; ++i)
        out[i * n + p] = solid ? 0.0 : load_dev<S>(a, i, x, y) + weight(i) * a.rho0;
}

template <class C>
__device__ __forceinline__ void force_at_d(const StepArgs& a, int x, int y, double& Fx, double& Fy) {
    C fx, fy;
    force_at<C>(a, x, y, fx, fy);
    Fx = (double)fx;
    Fy = (double)fy;
}

// Eq. 11 and Eq. 15 from the stored post-collision state:
// rho = sum f*_i, rho u = sum f*_i e_i - F/2.
template <class S>
__global__ void moments_kernel(const StepArgs a, double* rho, double* ux, double* uy) {
    using C = typename Fmt<S>::C;
    const long long n = (long long)a.geo.nx * a.geo.ny;
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int y = (int)(p / a.geo.nx), x = (int)(p - (long long)y * a.geo.nx);
    double r = 0.0, vx = 0.0, vy = 0.0;
    if (!node_solid(a, x, y)) {
        double dr = 0.0, jx = 0.0, jy = 0.0;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const double g = load_dev<S>(a, i, x, y);
            dr += g;
            jx += ex_of(i) * g;
            jy += ey_of(i) * g;
        }
        double Fx, Fy;
        force_at_d<C>(a, x, y, Fx, Fy);
        r = a.rho0 + dr;
        vx = (jx - 0.5 * Fx) / r;
        vy = (jy - 0.5 * Fy) / r;
    }
    if (rho) rho[p] = r;
    if (ux) ux[p] = vx;
    if (uy) uy[p] = vy;
}

__device__ __forceinline__ void atomic_max_pos(double* addr, double v) {
    // v >= 0: the IEEE order of non-negative doubles is their integer order
    atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

// psi(rho) = psi0 exp(-rho0 / rho) in the compute type C.
template <class C>
__device__ __forceinline__ C sc_psi(const StepArgs& a, C rho) {
    const C e = -(C)a.sc_rho0 / rho;
    if constexpr (sizeof(C) == 8) {
        return (C)a.sc_psi0 * exp(e);
    } else {
        return (C)a.sc_psi0 * expf(e);
    }
}

// Decoded deviation of population i at (x, y) of a.src in the compute type.
template <class S>
__device__ __forceinline__ typename Fmt<S>::C load_c(const StepArgs& a, int i, int x, int y) {
    using F = Fmt<S>;
    using C = typename F::C;
    const S* p = static_cast<const S*>(a.src) + i * a.geo.plane + (long long)y * a.geo.pitch + x;
    uint32_t w[4] = {0u, 0u, 0u, 0u};
    if constexpr (sizeof(S) == 8) {
        const unsigned long long v = *reinterpret_cast<const unsigned long long*>(p);
        w[0] = (uint32_t)v; w[1] = (uint32_t)(v >> 32);
    } else if constexpr (sizeof(S) == 4) {
        w[0] = *reinterpret_cast<const uint32_t*>(p);
    } else {
        w[0] = *reinterpret_cast<const unsigned short*>(p);
    }
    return Alg<C>::mul(F::get(w, 0), (C)a.inv_scale);
}

// Shan-Chen psi field (see launch_psi): rho = rho0 + sum_i g_i in the compute
// type, summed in velocity order.
template <class S>
__global__ void psi_kernel(const StepArgs a, int mode, typename Fmt<S>::C* psi) {
    using C = typename Fmt<S>::C;
    const long long n = (long long)a.geo.nx * a.geo.ny;
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int y = (int)(p / a.geo.nx), x = (int)(p - (long long)y * a.geo.nx);
    C dr = C(0);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        int xs = x, ys = y;
        if (mode == 0) {         // f_i(x) = f*_i(x - e_i), periodic
            xs = x - ex_of(i);
            ys = y - ey_of(i);
            xs = xs < 0 ? xs + a.geo.nx : (xs >= a.geo.nx ? xs - a.geo.nx : xs);
            ys = ys < 0 ? ys + a.geo.ny : (ys >= a.geo.ny ? ys - a.geo.ny : ys);
        }
        dr = Alg<C>::add(dr, load_c<S>(a, i, xs, ys));
    }
    psi[(long long)y * a.geo.pitch + x] = sc_psi<C>(a, Alg<C>::add((C)a.rho0, dr));
}

template <class S>
__global__ void psi_prepare_kernel(const StepArgs a, int kind, const double* rho, const double* f,
                                   typename Fmt<S>::C* psi) {
    using C = typename Fmt<S>::C;
    const long long n = (long long)a.geo.nx * a.geo.ny;
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int y = (int)(p / a.geo.nx), x = (int)(p - (long long)y * a.geo.nx);
    double r = 1.0;
    if (kind == 0) {
        if (rho) r = rho[p];
    } else {
        r = 0.0;
#pragma unroll
        for (int i = 0; i < 9; ++i) r += f[i * n + p];
    }
    psi[(long long)y * a.geo.pitch + x] = sc_psi<C>(a, (C)r);
}

template <class S>
__global__ void max_abs_kernel(const StepArgs a, double* out) {
    const long long n = (long long)a.geo.nx * a.geo.ny;
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double mx = 0.0;
    if (p < n) {
        const int y = (int)(p / a.geo.nx), x = (int)(p - (long long)y * a.geo.nx);
        if (!node_solid(a, x, y)) {
#pragma unroll
            for (int i = 0; i < 9; ++i) mx = fmax(mx, fabs(load_dev<S>(a, i, x, y)));
        }
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0 && mx > 0.0) atomic_max_pos(out, mx);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
int element_size(int format) { return format == 0 ? 8 : format == 1 ? 4 : 2; }

cudaError_t launch_step(const StepArgs& a, int format, cudaStream_t s) {
    switch (format) {
        case 0: return launch_step_fp64(a, s);
        case 1: return launch_step_fp32(a, s);
        case 2: return a.sround ? launch_step_fp16sr(a, s) : launch_step_fp16(a, s);
        case 3: return a.sround ? launch_step_bf16sr(a, s) : launch_step_bf16(a, s);
    }
    return cudaErrorInvalidValue;
}

__global__ void sr_tick_kernel(uint32_t* counter) { *counter += 1u; }

cudaError_t launch_sr_tick(uint32_t* counter, cudaStream_t s) {
    sr_tick_kernel<<<1, 1, 0, s>>>(counter);
    return cudaGetLastError();
}

cudaError_t launch_batch_step(const BatchLaunch& b, int format, cudaStream_t s) {
    switch (format) {
        case 0: return launch_batch_step_fp64(b, s);
        case 1: return launch_batch_step_fp32(b, s);
        case 2: return launch_batch_step_fp16(b, s);
        case 3: return launch_batch_step_bf16(b, s);
    }
    return cudaErrorInvalidValue;
}

size_t batch_stage_bytes(int format, int vec_bytes, int stages, int mask_mode) {
    const bool m = mask_mode != 0;
    const int nw = format == 0 ? 4 : vec_bytes / 4;
    int words;
    if (format == 0)
        words = m ? StageOf<double, 4, true, 1>::kWords : StageOf<double, 4, false, 1>::kWords;
    else if (nw == 4)
        words = m ? StageOf<float, 4, true, 1>::kWords : StageOf<float, 4, false, 1>::kWords;
    else
        words = m ? StageOf<float, 2, true, 1>::kWords : StageOf<float, 2, false, 1>::kWords;
    return (size_t)(kStepThreads / 32) * (stages > 0 ? stages : 0) * words * 4;
}

int vector_width_of(int format, int vec_bytes) {
    return (format == 0 ? 16 : vec_bytes) / element_size(format);
}

static unsigned node_blocks(const StepArgs& a, int threads) {
    const long long n = (long long)a.geo.nx * a.geo.ny;
    return (unsigned)((n + threads - 1) / threads);
}

#define CLBM_DISPATCH(format, CALL)                         \
    switch (format) {                                       \
        case 0: { using S = double; CALL; break; }          \
        case 1: { using S = float; CALL; break; }           \
        case 2: { using S = __half; CALL; break; }          \
        case 3: { using S = __nv_bfloat16; CALL; break; }   \
        default: return cudaErrorInvalidValue;              \
    }                                                       \
    return cudaGetLastError();

cudaError_t launch_init(const StepArgs& a, int format, const double* rho, const double* ux,
                        const double* uy, cudaStream_t s) {
    CLBM_DISPATCH(format, (prepare_kernel<S><<<node_blocks(a, 256), 256, 0, s>>>(a, 0, rho, ux, uy, nullptr)))
}

cudaError_t launch_set_populations(const StepArgs& a, int format, const double* f, int collide,
                                   cudaStream_t s) {
    const int kind = collide ? 1 : 2;
    CLBM_DISPATCH(format, (prepare_kernel<S><<<node_blocks(a, 256), 256, 0, s>>>(a, kind, nullptr, nullptr, nullptr, f)))
}

cudaError_t launch_get_populations(const StepArgs& a, int format, double* f, int pre, cudaStream_t s) {
    CLBM_DISPATCH(format, (get_populations_kernel<S><<<node_blocks(a, 256), 256, 0, s>>>(a, f, pre)))
}

cudaError_t launch_window(const StepArgs& a, int format, int x0, int y0, int w, int h,
                          double* out, cudaStream_t s) {
    const long long n = (long long)w * h;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    CLBM_DISPATCH(format, (window_kernel<S><<<blocks, 256, 0, s>>>(a, x0, y0, w, h, out)))
}

cudaError_t launch_moments(const StepArgs& a, int format, double* rho, double* ux, double* uy,
                           cudaStream_t s) {
    CLBM_DISPATCH(format, (moments_kernel<S><<<node_blocks(a, 256), 256, 0, s>>>(a, rho, ux, uy)))
}

cudaError_t launch_psi(const StepArgs& a, int format, int mode, void* psi, cudaStream_t s) {
    CLBM_DISPATCH(format, (psi_kernel<S><<<node_blocks(a, 256), 256, 0, s>>>(
                              a, mode, static_cast<typename Fmt<S>::C*>(psi))))
}

cudaError_t launch_psi_prepare(const StepArgs& a, int format, int kind, const double* rho,
                               const double* f, void* psi, cudaStream_t s) {
    CLBM_DISPATCH(format, (psi_prepare_kernel<S><<<node_blocks(a, 256), 256, 0, s>>>(
                              a, kind, rho, f, static_cast<typename Fmt<S>::C*>(psi))))
}

cudaError_t launch_max_abs_dev(const StepArgs& a, int format, double* out, cudaStream_t s) {
    CLBM_DISPATCH(format, (max_abs_kernel<S><<<node_blocks(a, 256), 256, 0, s>>>(a, out)))
}

}  // namespace clbm
