// clbm_kernels.cu -- the fused pull-stream + collide + force kernel of one
// D2Q9 cascaded LBM time step (Fei & Luo, arXiv:1705.11092, Eq. 9-15 and the
// halfway bounce-back of Sec. 4A), plus the small per-node kernels around it
// (initialisation, population get/set, macroscopic readout).
//
// Layout in HBM: 9 population planes [i][y][x] (structure of arrays), rows
// padded to a multiple of the 16-byte vector width, two copies (ping-pong).
// Each warp owns 32 * V consecutive nodes of one row (V = 16 B / element);
// each lane moves one 16-byte vector per plane, so every plane access is one
// coalesced 512-byte warp transaction.  Pull streaming reads plane i from the
// node x - e_i: the row offset is a different row base, the +-1 column offset
// is one element shifted in from the neighbouring lane (warp shuffle), with a
// scalar load at the warp edges and at the periodic wrap.
#include "clbm_device.cuh"
#include "clbm_internal.h"

namespace clbm {

// ---------------------------------------------------------------------------
// raw element access inside a 16-byte vector held as 4 words
// ---------------------------------------------------------------------------
template <class S> struct Raw {
    using E = uint32_t;   // 16-bit and 32-bit elements travel as one word
};
template <> struct Raw<double> {
    using E = unsigned long long;
};

template <class S>
__device__ __forceinline__ typename Raw<S>::E raw_get(const uint32_t (&w)[4], int j) {
    if constexpr (sizeof(S) == 8) {
        return ((unsigned long long)w[2 * j + 1] << 32) | w[2 * j];
    } else if constexpr (sizeof(S) == 4) {
        return w[j];
    } else {
        return (w[j >> 1] >> ((j & 1) * 16)) & 0xffffu;
    }
}

template <class S>
__device__ __forceinline__ void raw_set(uint32_t (&w)[4], int j, typename Raw<S>::E v) {
    if constexpr (sizeof(S) == 8) {
        w[2 * j] = (uint32_t)v;
        w[2 * j + 1] = (uint32_t)(v >> 32);
    } else if constexpr (sizeof(S) == 4) {
        w[j] = v;
    } else {
        w[j >> 1] = (j & 1) ? ((w[j >> 1] & 0x0000ffffu) | (v << 16))
                            : ((w[j >> 1] & 0xffff0000u) | (v & 0xffffu));
    }
}

// element j <- element j-1, element 0 <- L   (source at x - 1)
template <class S>
__device__ __forceinline__ void shift_in_left(uint32_t (&w)[4], typename Raw<S>::E L) {
    if constexpr (sizeof(S) == 2) {
        // __byte_perm(a, b, 0x5432) = high half of a | low half of b << 16
        w[3] = __byte_perm(w[2], w[3], 0x5432);
        w[2] = __byte_perm(w[1], w[2], 0x5432);
        w[1] = __byte_perm(w[0], w[1], 0x5432);
        w[0] = __byte_perm(L << 16, w[0], 0x5432);
    } else {
        constexpr int V = 16 / sizeof(S);
#pragma unroll
        for (int j = V - 1; j > 0; --j) raw_set<S>(w, j, raw_get<S>(w, j - 1));
        raw_set<S>(w, 0, L);
    }
}

// element j <- element j+1, element V-1 <- R   (source at x + 1)
template <class S>
__device__ __forceinline__ void shift_in_right(uint32_t (&w)[4], typename Raw<S>::E R) {
    if constexpr (sizeof(S) == 2) {
        w[0] = __byte_perm(w[0], w[1], 0x5432);
        w[1] = __byte_perm(w[1], w[2], 0x5432);
        w[2] = __byte_perm(w[2], w[3], 0x5432);
        w[3] = __byte_perm(w[3], R, 0x5432);
    } else {
        constexpr int V = 16 / sizeof(S);
#pragma unroll
        for (int j = 0; j < V - 1; ++j) raw_set<S>(w, j, raw_get<S>(w, j + 1));
        raw_set<S>(w, V - 1, R);
    }
}

__device__ __forceinline__ void ld_vec(const void* p, uint32_t (&w)[4]) {
    const uint4 v = __ldcs(reinterpret_cast<const uint4*>(p));
    w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
}

__device__ __forceinline__ void st_vec(void* p, const uint32_t (&w)[4]) {
    __stcs(reinterpret_cast<uint4*>(p), make_uint4(w[0], w[1], w[2], w[3]));
}

template <class S>
__device__ __forceinline__ typename Raw<S>::E ld_elem(const S* p) {
    if constexpr (sizeof(S) == 8) {
        return __ldg(reinterpret_cast<const unsigned long long*>(p));
    } else if constexpr (sizeof(S) == 4) {
        return __ldg(reinterpret_cast<const unsigned int*>(p));
    } else {
        return (uint32_t)__ldg(reinterpret_cast<const unsigned short*>(p));
    }
}

template <class C> __device__ __forceinline__ Relax<C> relax_of(const RelaxBoth& r);
template <> __device__ __forceinline__ Relax<double> relax_of<double>(const RelaxBoth& r) {
    return Relax<double>{r.d[0], r.d[1], r.d[2], r.d[3], r.d[4], r.d[5], r.d[6]};
}
template <> __device__ __forceinline__ Relax<float> relax_of<float>(const RelaxBoth& r) {
    return Relax<float>{r.f[0], r.f[1], r.f[2], r.f[3], r.f[4], r.f[5], r.f[6]};
}

// Force at node (x, y) for the four force layouts of clbm_force_kind.
template <class C>
__device__ __forceinline__ void force_at(const StepArgs& a, int x, int y, C& Fx, C& Fy) {
    const C* F = static_cast<const C*>(a.force);
    switch (a.force_kind) {
        case 1: Fx = F[2 * y]; Fy = F[2 * y + 1]; break;
        case 2: Fx = F[2 * x]; Fy = F[2 * x + 1]; break;
        case 3: {
            const long long k = 2 * ((long long)y * a.geo.nx + x);
            Fx = F[k]; Fy = F[k + 1];
            break;
        }
        default: Fx = (C)a.fx; Fy = (C)a.fy; break;
    }
}

// ---------------------------------------------------------------------------
// The fused step kernel.  One warp = one 32 * V node chunk of one row.
// MASK = the lattice has solid nodes (link mask present).
// ---------------------------------------------------------------------------
template <class S, bool MASK>
__global__ void __launch_bounds__(256) step_kernel(const StepArgs a) {
    using F = Fmt<S>;
    using C = typename F::C;
    using E = typename Raw<S>::E;
    constexpr int V = F::V;

    const int lane = threadIdx.x & 31;
    const long long task = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (task >= a.ntasks) return;   // uniform per warp
    const int nx = a.geo.nx, ny = a.geo.ny, pitch = a.geo.pitch;
    const long long plane = a.geo.plane;
    const int y = (int)(task / a.chunks);
    const int c = (int)(task - (long long)y * a.chunks);
    const int x0 = c * (32 * V) + lane * V;
    const bool active = x0 < nx;
    const int ym = (y == 0) ? ny - 1 : y - 1;      // source row of e_y = +1
    const int yp = (y == ny - 1) ? 0 : y + 1;      // source row of e_y = -1
    const S* src = static_cast<const S*>(a.src);

    // link mask of the V nodes
    uint32_t m[V];
    bool all_solid = false;
    bool row_solid[3] = {false, false, false};     // source rows e_y = -1, 0, +1 all solid
    if constexpr (MASK) {
        const uint8_t* mp = a.lmask + (long long)y * pitch + x0;
        if (active) {
            if constexpr (V == 2) {
                const uint32_t v = *reinterpret_cast<const unsigned short*>(mp);
                m[0] = v & 0xff; m[1] = v >> 8;
            } else if constexpr (V == 4) {
                const uint32_t v = *reinterpret_cast<const unsigned int*>(mp);
#pragma unroll
                for (int j = 0; j < 4; ++j) m[j] = (v >> (8 * j)) & 0xff;
            } else {
                const uint2 v = *reinterpret_cast<const uint2*>(mp);
#pragma unroll
                for (int j = 0; j < 4; ++j) { m[j] = (v.x >> (8 * j)) & 0xff; m[j + 4] = (v.y >> (8 * j)) & 0xff; }
            }
        } else {
#pragma unroll
            for (int j = 0; j < V; ++j) m[j] = 0xff;
        }
        uint32_t all = 0xff;
#pragma unroll
        for (int j = 0; j < V; ++j) all &= m[j];
        all_solid = all & 1u;
        // bit 2 (source (x, y-1)) and bit 4 (source (x, y+1)) give the
        // solidity of the neighbouring rows under this vector
        row_solid[0] = (all >> 4) & 1u;
        row_solid[1] = all_solid;
        row_solid[2] = (all >> 2) & 1u;
    } else {
#pragma unroll
        for (int j = 0; j < V; ++j) m[j] = 0;
    }

    // ---- a1: pull-stream (Eq. 10) ------------------------------------------
    uint32_t w[9][4];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int ey = ey_of(i);
        const int row = ey > 0 ? ym : (ey < 0 ? yp : y);
        const bool load = active && !row_solid[ey + 1];
        if (load) {
            ld_vec(src + i * plane + (long long)row * pitch + x0, w[i]);
        } else {
            w[i][0] = w[i][1] = w[i][2] = w[i][3] = 0u;
        }
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int ex = ex_of(i), ey = ey_of(i);
        if (ex == 0) continue;
        const int row = ey > 0 ? ym : (ey < 0 ? yp : y);
        const S* rowp = src + i * plane + (long long)row * pitch;
        if (ex > 0) {           // source x - 1
            E L = __shfl_up_sync(0xffffffffu, raw_get<S>(w[i], V - 1), 1);
            if (lane == 0 && active) L = ld_elem<S>(rowp + (x0 == 0 ? nx - 1 : x0 - 1));
            shift_in_left<S>(w[i], L);
        } else {                // source x + 1
            E R = __shfl_down_sync(0xffffffffu, raw_get<S>(w[i], 0), 1);
            const bool edge = (lane == 31) || (x0 + V >= nx);
            if (edge && active) R = ld_elem<S>(rowp + (x0 + V >= nx ? 0 : x0 + V));
            shift_in_right<S>(w[i], R);
            if (active && x0 + V > nx) {   // ragged row end: node nx-1 wraps to x = 0
                const int jr = nx - 1 - x0;
#pragma unroll
                for (int j = 0; j < V - 1; ++j)
                    if (j == jr) raw_set<S>(w[i], j, R);
            }
        }
    }

    // ---- a1: halfway bounce-back (Sec. 4A): f_i(x) = f*_opp(i)(x) ---------
    if constexpr (MASK) {
        if (active) {
#pragma unroll
            for (int i = 1; i < 9; ++i) {
                bool any = false;
#pragma unroll
                for (int j = 0; j < V; ++j) any |= ((m[j] >> i) & 1u) && !(m[j] & 1u);
                if (any) {
                    uint32_t o[4];
                    ld_vec(src + opp_of(i) * plane + (long long)y * pitch + x0, o);
#pragma unroll
                    for (int j = 0; j < V; ++j)
                        if ((m[j] >> i) & 1u) raw_set<S>(w[i], j, raw_get<S>(o, j));
                }
            }
        }
    }

    // ---- a2-a7: collide every node of the vector, encode in place ---------
    const Relax<C> rx = relax_of<C>(a.relax);
    const C rho0 = (C)a.rho0, scale = (C)a.scale, inv_scale = (C)a.inv_scale;
#pragma unroll
    for (int j = 0; j < V; ++j) {
        C g[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) g[i] = F::decode(F::get(w[i], j), inv_scale);
        C Fx, Fy;
        force_at<C>(a, min(x0 + j, nx - 1), y, Fx, Fy);
        collide<C>(g, Fx, Fy, rx, rho0);
        const bool solid = MASK && (m[j] & 1u);
#pragma unroll
        for (int i = 0; i < 9; ++i) F::set(w[i], j, solid ? C(0) : F::encode(g[i], scale));
    }

    // ---- a7: store (a8: fully solid vectors write nothing) -----------------
    if (active && !all_solid) {
        S* dst = static_cast<S*>(a.dst) + (long long)y * pitch + x0;
#pragma unroll
        for (int i = 0; i < 9; ++i) st_vec(dst + i * plane, w[i]);
    }
}

// ---------------------------------------------------------------------------
// per-node helper kernels (not on the time-step path)
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool node_solid(const StepArgs& a, int x, int y) {
    return a.lmask && (a.lmask[(long long)y * a.geo.pitch + x] & 1u);
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

// kind 0: equilibrium of (rho, ux, uy); kind 1: given FP64 populations.
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
    C Fx, Fy;
    force_at<C>(a, x, y, Fx, Fy);
    collide<C>(g, Fx, Fy, relax_of<C>(a.relax), (C)a.rho0);
#pragma unroll
    for (int i = 0; i < 9; ++i) store_elem<S>(a, i, x, y, F::encode(g[i], (C)a.scale));
}

template <class S>
__global__ void get_populations_kernel(const StepArgs a, double* f) {
    const long long n = (long long)a.geo.nx * a.geo.ny;
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int y = (int)(p / a.geo.nx), x = (int)(p - (long long)y * a.geo.nx);
    const bool solid = node_solid(a, x, y);
#pragma unroll
    for (int i = 0; i < 9; ++i)
        f[i * n + p] = solid ? 0.0 : load_dev<S>(a, i, x, y) + weight(i) * a.rho0;
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
int vector_width(int format) { return format == 0 ? 2 : format == 1 ? 4 : 8; }
int element_size(int format) { return format == 0 ? 8 : format == 1 ? 4 : 2; }

template <class S>
static cudaError_t step_t(const StepArgs& a, cudaStream_t s) {
    const int warps = 8;
    const long long blocks = (a.ntasks + warps - 1) / warps;
    if (a.lmask)
        step_kernel<S, true><<<(unsigned)blocks, 32 * warps, 0, s>>>(a);
    else
        step_kernel<S, false><<<(unsigned)blocks, 32 * warps, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_step(const StepArgs& a, int format, cudaStream_t s) {
    switch (format) {
        case 0: return step_t<double>(a, s);
        case 1: return step_t<float>(a, s);
        case 2: return step_t<__half>(a, s);
        case 3: return step_t<__nv_bfloat16>(a, s);
    }
    return cudaErrorInvalidValue;
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

cudaError_t launch_set_populations(const StepArgs& a, int format, const double* f, cudaStream_t s) {
    CLBM_DISPATCH(format, (prepare_kernel<S><<<node_blocks(a, 256), 256, 0, s>>>(a, 1, nullptr, nullptr, nullptr, f)))
}

cudaError_t launch_get_populations(const StepArgs& a, int format, double* f, cudaStream_t s) {
    CLBM_DISPATCH(format, (get_populations_kernel<S><<<node_blocks(a, 256), 256, 0, s>>>(a, f)))
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

cudaError_t launch_max_abs_dev(const StepArgs& a, int format, double* out, cudaStream_t s) {
    CLBM_DISPATCH(format, (max_abs_kernel<S><<<node_blocks(a, 256), 256, 0, s>>>(a, out)))
}

}  // namespace clbm
