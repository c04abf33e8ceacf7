// clbm_device.cuh -- device-side building blocks of the fused D2Q9 cascaded
// LBM step (Fei & Luo, arXiv:1705.11092): storage codecs for the population
// planes and the per-node collision with consistent forcing.
//
// Populations are stored as shifted deviations g_i = (f_i - w_i rho0) * 2^k
// and the collision works on deviations throughout, so FP32 arithmetic never
// forms f_i ~ 0.44 and keeps the small deviation bits.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace clbm {

// ---------------------------------------------------------------------------
// D2Q9 velocities (Eq. 1).  Direction i has velocity (EX[i], EY[i]).
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int ex_of(int i) {
    return (i == 1 || i == 5 || i == 8) ? 1 : (i == 3 || i == 6 || i == 7) ? -1 : 0;
}
__host__ __device__ constexpr int ey_of(int i) {
    return (i == 2 || i == 5 || i == 6) ? 1 : (i == 4 || i == 7 || i == 8) ? -1 : 0;
}
__host__ __device__ constexpr int opp_of(int i) {
    return i == 0 ? 0 : (i <= 4 ? ((i + 1) % 4) + 1 : ((i - 3) % 4) + 5);
}
// Slot of the own vector of plane opp(i) that halfway bounce-back reads for
// link i in {2, 4, 5, 6, 7, 8} (links 1 and 3 read planes of the node's own
// row, which the pull reads anyway).
__host__ __device__ constexpr int own_slot(int i) {
    return i == 2 ? 0 : i == 4 ? 1 : i == 5 ? 2 : i == 6 ? 3 : i == 7 ? 4 : 5;
}
// 1-D weights of the tensor-product D2Q9 rest state: w(-1), w(0), w(+1).
__host__ __device__ constexpr double w1d(int c) { return c == 0 ? 2.0 / 3.0 : 1.0 / 6.0; }
__host__ __device__ constexpr double weight(int i) { return w1d(ex_of(i)) * w1d(ey_of(i)); }

// ---------------------------------------------------------------------------
// Storage formats.  A thread moves one 16-byte vector (4 x 32-bit words) per
// plane, i.e. V = 16 / sizeof(element) consecutive nodes in x.
// ---------------------------------------------------------------------------
template <class S> struct Fmt;

template <> struct Fmt<double> {
    using C = double;                 // compute type
    static constexpr int V = 2;
    __device__ static C get(const uint32_t (&w)[4], int j) {
        return __hiloint2double((int)w[2 * j + 1], (int)w[2 * j]);
    }
    __device__ static void set(uint32_t (&w)[4], int j, C v) {
        w[2 * j] = (uint32_t)__double2loint(v);
        w[2 * j + 1] = (uint32_t)__double2hiint(v);
    }
    __device__ static C decode(C v, C) { return v; }
    __device__ static C encode(C v, C) { return v; }
};

template <> struct Fmt<float> {
    using C = float;
    static constexpr int V = 4;
    __device__ static C get(const uint32_t (&w)[4], int j) { return __uint_as_float(w[j]); }
    __device__ static void set(uint32_t (&w)[4], int j, C v) { w[j] = __float_as_uint(v); }
    __device__ static C decode(C v, C) { return v; }
    __device__ static C encode(C v, C) { return v; }
};

// 16-bit formats: element j sits in half (j & 1) of word j >> 1.  The value
// held is the raw 16-bit pattern; decode/encode convert with the run scale.
template <> struct Fmt<__half> {
    using C = float;
    static constexpr int V = 8;
    __device__ static uint32_t bits(const uint32_t (&w)[4], int j) {
        return (w[j >> 1] >> ((j & 1) * 16)) & 0xffffu;
    }
    __device__ static C get(const uint32_t (&w)[4], int j) {
        return __half2float(__ushort_as_half((unsigned short)bits(w, j)));
    }
    __device__ static void set(uint32_t (&w)[4], int j, C v) {
        uint32_t h = __half_as_ushort(__float2half_rn(v));
        w[j >> 1] = (j & 1) ? ((w[j >> 1] & 0x0000ffffu) | (h << 16)) : ((w[j >> 1] & 0xffff0000u) | h);
    }
    __device__ static C decode(C v, C inv_scale) { return v * inv_scale; }
    __device__ static C encode(C v, C scale) { return v * scale; }
};

template <> struct Fmt<__nv_bfloat16> {
    using C = float;
    static constexpr int V = 8;
    __device__ static uint32_t bits(const uint32_t (&w)[4], int j) {
        return (w[j >> 1] >> ((j & 1) * 16)) & 0xffffu;
    }
    __device__ static C get(const uint32_t (&w)[4], int j) {
        return __uint_as_float(bits(w, j) << 16);
    }
    __device__ static void set(uint32_t (&w)[4], int j, C v) {
        uint32_t h = __bfloat16_as_ushort(__float2bfloat16_rn(v));
        w[j >> 1] = (j & 1) ? ((w[j >> 1] & 0x0000ffffu) | (h << 16)) : ((w[j >> 1] & 0xffff0000u) | h);
    }
    __device__ static C decode(C v, C inv_scale) { return v * inv_scale; }
    __device__ static C encode(C v, C scale) { return v * scale; }
};

// 16-bit storage whose time step rounds stochastically when it stores a
// population (clbm_set_rounding): the same bits in memory as __half and
// __nv_bfloat16, the same decode; only the step's encode differs.
struct HalfSR {
    unsigned short bits;
};
struct Bf16SR {
    unsigned short bits;
};
template <> struct Fmt<HalfSR> : Fmt<__half> {};
template <> struct Fmt<Bf16SR> : Fmt<__nv_bfloat16> {};

template <class S> struct is16 { static constexpr bool value = false; };
template <> struct is16<__half> { static constexpr bool value = true; };
template <> struct is16<__nv_bfloat16> { static constexpr bool value = true; };
template <> struct is16<HalfSR> { static constexpr bool value = true; };
template <> struct is16<Bf16SR> { static constexpr bool value = true; };

template <class S> struct Stochastic { static constexpr bool value = false; };
template <> struct Stochastic<HalfSR> { static constexpr bool value = true; };
template <> struct Stochastic<Bf16SR> { static constexpr bool value = true; };

// ---------------------------------------------------------------------------
// Arithmetic of the collision, generic over the value type: double, float,
// or F2 -- two nodes' FP32 values side by side, computed with the packed
// FP32x2 instructions (add/sub/mul/fma .f32x2) that sm_100-class GPUs
// execute as one instruction for both lanes.  Every operation is written
// out and none is merged by the compiler, so all three forms round alike:
// each mul/add/sub/fma is one IEEE operation with round-to-nearest.
// ---------------------------------------------------------------------------
struct F2 {
    float2 v;
};

template <class T> struct Alg;

template <> struct Alg<double> {
    using S = double;
    __device__ static double splat(double a) { return a; }
    __device__ static double add(double a, double b) { return __dadd_rn(a, b); }
    __device__ static double sub(double a, double b) { return __dsub_rn(a, b); }
    __device__ static double mul(double a, double b) { return __dmul_rn(a, b); }
    __device__ static double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
    __device__ static double recip(double a) { return 1.0 / a; }
};

// FP32 ops are issued as inline PTX as well, so the compiler executes them
// exactly as written (no re-association, fusion or rewriting of a product
// with a reciprocal): scalar and packed forms then round identically.
template <> struct Alg<float> {
    using S = float;
    __device__ static float splat(float a) { return a; }
    __device__ static float add(float a, float b) {
        float r;
        asm("add.rn.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
        return r;
    }
    __device__ static float sub(float a, float b) {
        float r;
        asm("sub.rn.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
        return r;
    }
    __device__ static float mul(float a, float b) {
        float r;
        asm("mul.rn.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
        return r;
    }
    __device__ static float fma(float a, float b, float c) {
        float r;
        asm("fma.rn.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
        return r;
    }
    // hardware reciprocal (within 2 ulp): far below the FP32 path's storage
    // rounding
    __device__ static float recip(float a) { return __fdividef(1.0f, a); }
};

// Packed ops are issued as inline PTX: the compiler cannot merge a separate
// mul and add into one fma there, so the packed form rounds exactly like the
// scalar one (whose __fmul_rn/__fadd_rn are never merged either).
__device__ __forceinline__ unsigned long long f2_bits(F2 a) {
    unsigned long long r;
    memcpy(&r, &a.v, 8);
    return r;
}
__device__ __forceinline__ F2 f2_from(unsigned long long r) {
    F2 out;
    memcpy(&out.v, &r, 8);
    return out;
}

template <> struct Alg<F2> {
    using S = float;
    __device__ static F2 splat(float a) { return F2{make_float2(a, a)}; }
    __device__ static F2 add(F2 a, F2 b) {
        unsigned long long r;
        asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_bits(a)), "l"(f2_bits(b)));
        return f2_from(r);
    }
    __device__ static F2 sub(F2 a, F2 b) {
        unsigned long long r;
        asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_bits(a)), "l"(f2_bits(b)));
        return f2_from(r);
    }
    __device__ static F2 mul(F2 a, F2 b) {
        unsigned long long r;
        asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_bits(a)), "l"(f2_bits(b)));
        return f2_from(r);
    }
    __device__ static F2 fma(F2 a, F2 b, F2 c) {
        unsigned long long r;
        asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(f2_bits(a)), "l"(f2_bits(b)), "l"(f2_bits(c)));
        return f2_from(r);
    }
    __device__ static F2 recip(F2 a) {
        return F2{make_float2(__fdividef(1.0f, a.v.x), __fdividef(1.0f, a.v.y))};
    }
};

// ---------------------------------------------------------------------------
// Per-launch constants of the collision (Eq. 7, 8, 14), in the value type T.
// rho0 is the reference density of the deviation shift, times the run scale.
// ---------------------------------------------------------------------------
template <class T> struct Coef {
    T om_b;    // 1 - s_b   (bulk, T~3)
    T om_2;    // 1 - s_2   (shear, T~4, T~5)
    T om_3;    // 1 - s_3   (third order, T~6, T~7)
    T om_4;    // 1 - s_4   (fourth order, T~8)
    T sb23;    // s_b * 2/3        (T~eq_3 = 2 rho cs^2, Eq. 8)
    T s4_9;    // s_4 / 9          (T~eq_8 = rho cs^4, Eq. 8)
    T f3;      // (1 - s_3/2) / 3  ((I - S/2) C in slots 6, 7; cs^2 = 1/3)
    T rho0;    // rho0
    T rho0_6;  // rho0 / 6   (1-D rest weights 1/6, 2/3, 1/6 times rho0)
    T rho0_23; // rho0 * 2/3
    T rho0_3;  // rho0 / 3   (second 1-D moment of the rest state)
    T half;
    T two;
    T zero;
    T nom_2;   // -(1 - s_2)
    T g1;      // coefficient of F in k~*_10, k~*_01: 1/2; (1 + s1 - s2)/2 for M2
    T c2;      // (1 - s2/2): weight of Guo's moments in M2
    bool m2;   // forcing of Lycett-Brown and Luo (Eq. 21) instead of Eq. 12
};

// raw constants (see RelaxBoth): om_b, om_2, om_3, om_4, sb23, s4_9, f3,
// g1, c2, m2
template <class T>
__device__ __forceinline__ Coef<T> make_coef(const typename Alg<T>::S (&r)[10],
                                             typename Alg<T>::S rho0) {
    using A = Alg<T>;
    using S = typename A::S;
    Coef<T> k;
    k.om_b = A::splat(r[0]);
    k.om_2 = A::splat(r[1]);
    k.om_3 = A::splat(r[2]);
    k.om_4 = A::splat(r[3]);
    k.sb23 = A::splat(r[4]);
    k.s4_9 = A::splat(r[5]);
    k.f3 = A::splat(r[6]);
    k.rho0 = A::splat(rho0);
    k.rho0_6 = A::splat(rho0 / S(6));
    k.rho0_23 = A::splat(rho0 * S(2) / S(3));
    k.rho0_3 = A::splat(rho0 / S(3));
    k.half = A::splat(S(0.5));
    k.two = A::splat(S(2));
    k.zero = A::splat(S(0));
    k.nom_2 = A::splat(-r[1]);
    k.g1 = A::splat(r[7]);
    k.c2 = A::splat(r[8]);
    k.m2 = r[9] != S(0);
    return k;
}

// Shan-Chen interaction force at node (x, y) (Sec. 4C):
//   F = -G psi(x) sum_i w_i psi(x + e_i) e_i,
// w_i = 1/3 on the axes and 1/12 on the diagonals, from a periodic psi field
// [ny][pitch] in the compute type C.  Every operation is a rounded add, sub
// or mul (no contraction), so all kernels that call it agree bit for bit.
template <class C>
__device__ __forceinline__ void sc_force_node(const C* __restrict__ psi, int pitch, int nx, int ny,
                                              int x, int y, C G, C& Fx, C& Fy) {
    using A = Alg<C>;
    const int xl = x == 0 ? nx - 1 : x - 1, xr = x == nx - 1 ? 0 : x + 1;
    const int yd = y == 0 ? ny - 1 : y - 1, yu = y == ny - 1 ? 0 : y + 1;
    const C* r0 = psi + (long long)yd * pitch;   // row y - 1 (e_y = -1)
    const C* r1 = psi + (long long)y * pitch;
    const C* r2 = psi + (long long)yu * pitch;   // row y + 1 (e_y = +1)
    const C third = C(1) / C(3), twelfth = C(1) / C(12);
    const C ax = A::sub(r1[xr], r1[xl]);
    const C dx = A::add(A::sub(r2[xr], r2[xl]), A::sub(r0[xr], r0[xl]));
    const C ay = A::sub(r2[x], r0[x]);
    const C dy = A::sub(A::add(r2[xr], r2[xl]), A::add(r0[xr], r0[xl]));
    const C sx = A::add(A::mul(third, ax), A::mul(twelfth, dx));
    const C sy = A::add(A::mul(third, ay), A::mul(twelfth, dy));
    const C g = A::mul(-G, r1[x]);
    Fx = A::mul(g, sx);
    Fy = A::mul(g, sy);
}

// ---------------------------------------------------------------------------
// One collision at one node (or one pair of nodes for F2), in place on the
// deviations g[9] (Eq. 11-15).
//
// The map f -> T~ = N(u) M f of Eq. 4-6 is applied as a tensor product of two
// 1-D shifts: along x for each row of velocities (e_y = -1, 0, 1), then along
// y for each x-moment order m = 0, 1, 2.  This yields the central moments
// k~_mn (m, n <= 2) of Eq. 2, from which T~ is the recombination of Eq. 3;
// the back-transform M^-1 N^-1 (Eq. 9) is the inverse of the same two
// shifts.  All moments are carried as deviations from rho0 c_m c_n with
// c = (1, 0, 1/3), the moments of rho0 w_i.
//
// Relaxation (Eq. 12 with Eq. 8 and the forcing moments of Eq. 14):
//   T~*_0 = rho,  T~*_1 = Fx/2, T~*_2 = Fy/2   (conserved; any s0, s1)
//   T~*_3 = (1-sb) T~_3 + sb 2 rho/3
//   T~*_4,5 = (1-s2) T~_4,5
//   T~*_6 = (1-s3) T~_6 + (1-s3/2) Fy/3   (k~21 of R_i, Eq. 13)
//   T~*_7 = (1-s3) T~_7 + (1-s3/2) Fx/3   (k~12 of R_i, Eq. 13)
//   T~*_8 = (1-s4) T~_8 + s4 rho/9
// The velocity is the force-corrected one of Eq. 15.
// ---------------------------------------------------------------------------
// GUO: the M2 forcing moments (compiled only where M2 is launched).
template <class T, bool GUO = false>
__device__ __forceinline__ void collide(T (&g)[9], T Fx, T Fy, const Coef<T>& k) {
    using A = Alg<T>;
    // q[a][b]: population with velocity (a-1, b-1)
    T q[3][3];
    q[0][0] = g[7]; q[1][0] = g[4]; q[2][0] = g[8];
    q[0][1] = g[3]; q[1][1] = g[0]; q[2][1] = g[1];
    q[0][2] = g[6]; q[1][2] = g[2]; q[2][2] = g[5];

    // per velocity row b: sum, difference and sum of the e_x = +-1 entries
    T sx[3], dx[3], d0[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        sx[b] = A::add(q[2][b], q[0][b]);
        dx[b] = A::sub(q[2][b], q[0][b]);
        d0[b] = A::add(sx[b], q[1][b]);
    }
    // Eq. 11 and Eq. 15
    const T drho = A::add(A::add(d0[0], d0[2]), d0[1]);
    const T jx = A::add(A::add(dx[0], dx[2]), dx[1]);
    const T jy = A::sub(d0[2], d0[0]);
    const T rho = A::add(k.rho0, drho);
    const T inv_rho = A::recip(rho);
    const T ux = A::mul(A::fma(k.half, Fx, jx), inv_rho);
    const T uy = A::mul(A::fma(k.half, Fy, jy), inv_rho);
    // Every rounded product below is consumed as an fma operand, never by a
    // separate add: a compiler may not fuse a separate mul and add the same
    // way in every instantiation, and only exact products (by 1/2 or 2) may
    // feed an add.
    const T ux2 = A::mul(ux, ux), uy2 = A::mul(uy, uy);
    const T ux_2 = A::mul(k.two, ux), uy_2 = A::mul(k.two, uy);
    const T nux = A::sub(k.zero, ux), nuy = A::sub(k.zero, uy);
    const T nux_2 = A::sub(k.zero, ux_2), nuy_2 = A::sub(k.zero, uy_2);
    const T w0[3] = {k.rho0_6, k.rho0_23, k.rho0_6};

    // x shift (central moments in x of each row): h[m][b]
    T h[3][3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        const T K0 = A::add(w0[b], d0[b]);
        h[0][b] = d0[b];
        h[1][b] = A::fma(nux, K0, dx[b]);
        h[2][b] = A::fma(ux2, K0, A::fma(nux_2, dx[b], sx[b]));
    }
    // y shift for each x order m: D[m][n] = k~_mn - rho0 c_m c_n
    T D[3][3];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        const T s = A::add(h[m][2], h[m][0]);
        const T d = A::sub(h[m][2], h[m][0]);
        const T D0 = A::add(s, h[m][1]);
        const T K0 = (m == 0) ? rho : (m == 1) ? D0 : A::add(k.rho0_3, D0);
        D[m][0] = D0;
        D[m][1] = A::fma(nuy, K0, d);
        D[m][2] = A::fma(uy2, K0, A::fma(nuy_2, d, s));
    }

    // relaxation with consistent forcing (Eq. 12), in deviation form
    // T~*_3 - 2 rho0/3 = t3;  T~*_4 = (1 - s2) dd;  k~*_20, k~*_02 = (t3 +- T~*_4)/2
    const T t3 = A::fma(k.om_b, A::add(D[2][0], D[0][2]), A::mul(k.sb23, drho));
    const T dd = A::sub(D[2][0], D[0][2]);
    T E[3][3];
    E[0][0] = drho;
    E[1][0] = A::mul(k.g1, Fx);
    E[0][1] = A::mul(k.g1, Fy);
    E[2][0] = A::mul(k.half, A::fma(k.om_2, dd, t3));
    E[0][2] = A::mul(k.half, A::fma(k.nom_2, dd, t3));
    E[1][1] = A::mul(k.om_2, D[1][1]);
    E[2][1] = A::fma(k.om_3, D[2][1], A::mul(k.f3, Fy));
    E[1][2] = A::fma(k.om_3, D[1][2], A::mul(k.f3, Fx));
    E[2][2] = A::fma(k.om_4, D[2][2], A::mul(k.s4_9, drho));
    if constexpr (GUO) {
        // M2 (Eq. 21): (1 - s2/2) times the central moments of Guo's R_G,
        // [0, Fx, Fy, 0, 0, 0, Fy/3 - 2 ux uy Fx - ux^2 Fy,
        //  Fx/3 - 2 ux uy Fy - uy^2 Fx, 4 ux uy (uy Fx + ux Fy)]; the Fy/3, Fx/3
        // parts sit in f3 and the first-order parts in g1
        const T uxy = A::mul(ux, uy);
        const T a21 = A::fma(ux2, Fy, A::mul(A::mul(k.two, uxy), Fx));   // 2 ux uy Fx + ux^2 Fy
        const T a12 = A::fma(uy2, Fx, A::mul(A::mul(k.two, uxy), Fy));   // 2 ux uy Fy + uy^2 Fx
        const T a22 = A::mul(A::mul(k.two, k.two), A::mul(uxy, A::fma(uy, Fx, A::mul(ux, Fy))));
        const T nc2 = A::sub(k.zero, k.c2);
        E[2][1] = A::fma(nc2, a21, E[2][1]);
        E[1][2] = A::fma(nc2, a12, E[1][2]);
        E[2][2] = A::fma(k.c2, a22, E[2][2]);
    }

    // inverse y shift: back to x-moments of each velocity row
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        const T K0 = (m == 0) ? rho : (m == 1) ? E[1][0] : A::add(k.rho0_3, E[2][0]);
        const T r1 = A::fma(uy, K0, E[m][1]);
        const T R2 = A::fma(uy2, K0, A::fma(uy_2, E[m][1], E[m][2]));
        h[m][1] = A::sub(E[m][0], R2);
        h[m][2] = A::mul(k.half, A::add(R2, r1));
        h[m][0] = A::mul(k.half, A::sub(R2, r1));
    }
    // inverse x shift: back to populations
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        const T K0 = A::add(w0[b], h[0][b]);
        const T r1 = A::fma(ux, K0, h[1][b]);
        const T R2 = A::fma(ux2, K0, A::fma(ux_2, h[1][b], h[2][b]));
        q[1][b] = A::sub(h[0][b], R2);
        q[2][b] = A::mul(k.half, A::add(R2, r1));
        q[0][b] = A::mul(k.half, A::sub(R2, r1));
    }
    g[7] = q[0][0]; g[4] = q[1][0]; g[8] = q[2][0];
    g[3] = q[0][1]; g[0] = q[1][1]; g[1] = q[2][1];
    g[6] = q[0][2]; g[2] = q[1][2]; g[5] = q[2][2];
}

// Deviations of the generalized equilibrium (central moments Eq. 8) about
// (rho0 + drho, u): the inverse of the two shifts applied to D = drho c_m c_n.
template <class C>
__device__ __forceinline__ void equilibrium_dev(C drho, C ux, C uy, C rho0, C (&g)[9]) {
    using A = Alg<C>;
    const C half = C(0.5), two = C(2), third = C(1) / C(3);
    const C wr[3] = {C(1) / C(6), C(2) / C(3), C(1) / C(6)};
    const C ux2 = ux * ux, uy2 = uy * uy;
    C h[3][3];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        const C cm = (m == 0) ? C(1) : (m == 1) ? C(0) : third;
        const C E0 = drho * cm, E1 = C(0), E2 = drho * cm * third;
        const C K0 = A::fma(rho0, cm, E0);
        const C r1 = A::fma(uy, K0, E1);
        const C R2 = A::fma(uy2, K0, A::fma(two * uy, E1, E2));
        h[m][1] = E0 - R2;
        h[m][2] = half * (R2 + r1);
        h[m][0] = half * (R2 - r1);
    }
    C q[3][3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        const C K0 = A::fma(rho0, wr[b], h[0][b]);
        const C r1 = A::fma(ux, K0, h[1][b]);
        const C R2 = A::fma(ux2, K0, A::fma(two * ux, h[1][b], h[2][b]));
        q[1][b] = h[0][b] - R2;
        q[2][b] = half * (R2 + r1);
        q[0][b] = half * (R2 - r1);
    }
    g[7] = q[0][0]; g[4] = q[1][0]; g[8] = q[2][0];
    g[3] = q[0][1]; g[0] = q[1][1]; g[1] = q[2][1];
    g[6] = q[0][2]; g[2] = q[1][2]; g[5] = q[2][2];
}

}  // namespace clbm
