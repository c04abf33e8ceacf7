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

template <class S> struct is16 { static constexpr bool value = false; };
template <> struct is16<__half> { static constexpr bool value = true; };
template <> struct is16<__nv_bfloat16> { static constexpr bool value = true; };

// ---------------------------------------------------------------------------
// Relaxation parameters of Eq. 7 in the form the collision uses.
// ---------------------------------------------------------------------------
template <class C> struct Relax {
    C om_b;   // 1 - s_b   (bulk, T~3)
    C om_2;   // 1 - s_2   (shear, T~4, T~5)
    C om_3;   // 1 - s_3   (third order, T~6, T~7)
    C om_4;   // 1 - s_4   (fourth order, T~8)
    C sb23;   // s_b * 2/3     (T~eq_3 = 2 rho cs^2, Eq. 8)
    C s4_9;   // s_4 / 9       (T~eq_8 = rho cs^4, Eq. 8)
    C f3;     // (1 - s_3/2) / 3  (forcing weight of C6, C7: (I - S/2) C, cs^2 = 1/3)
};

// ---------------------------------------------------------------------------
// One collision at one node, in place on the deviations g[9] (Eq. 11-15).
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
template <class C>
__device__ __forceinline__ void collide(C (&g)[9], C Fx, C Fy, const Relax<C>& r, C rho0) {
    const C half = C(0.5), two = C(2), third = C(1) / C(3);
    const C wr[3] = {C(1) / C(6), C(2) / C(3), C(1) / C(6)};   // 1-D weights, index c+1
    // q[a][b]: population with velocity (a-1, b-1)
    C q[3][3];
    q[0][0] = g[7]; q[1][0] = g[4]; q[2][0] = g[8];
    q[0][1] = g[3]; q[1][1] = g[0]; q[2][1] = g[1];
    q[0][2] = g[6]; q[1][2] = g[2]; q[2][2] = g[5];

    // per velocity row b: sum, difference and sum of the e_x = +-1 entries
    C sx[3], dx[3], d0[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        sx[b] = q[2][b] + q[0][b];
        dx[b] = q[2][b] - q[0][b];
        d0[b] = sx[b] + q[1][b];
    }
    // Eq. 11 and Eq. 15
    const C drho = (d0[0] + d0[2]) + d0[1];
    const C jx = (dx[0] + dx[2]) + dx[1];
    const C jy = d0[2] - d0[0];
    const C rho = rho0 + drho;
    const C inv_rho = C(1) / rho;
    const C ux = (jx + half * Fx) * inv_rho;
    const C uy = (jy + half * Fy) * inv_rho;
    const C ux2 = ux * ux, uy2 = uy * uy;

    // x shift (central moments in x of each row): h[m][b]
    C h[3][3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        const C K0 = rho0 * wr[b] + d0[b];
        h[0][b] = d0[b];
        h[1][b] = dx[b] - ux * K0;
        h[2][b] = (sx[b] - two * ux * dx[b]) + ux2 * K0;
    }
    // y shift for each x order m: D[m][n] = k~_mn - rho0 c_m c_n
    C D[3][3];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        const C cm = (m == 0) ? C(1) : (m == 1) ? C(0) : third;
        const C s = h[m][2] + h[m][0];
        const C d = h[m][2] - h[m][0];
        const C D0 = s + h[m][1];
        const C K0 = rho0 * cm + D0;
        D[m][0] = D0;
        D[m][1] = d - uy * K0;
        D[m][2] = (s - two * uy * d) + uy2 * K0;
    }

    // relaxation with consistent forcing (Eq. 12), in deviation form
    const C t3 = r.om_b * (D[2][0] + D[0][2]) + r.sb23 * drho;   // T~*_3 - 2 rho0/3
    const C t4 = r.om_2 * (D[2][0] - D[0][2]);                    // T~*_4
    C E[3][3];
    E[0][0] = drho;
    E[1][0] = half * Fx;
    E[0][1] = half * Fy;
    E[2][0] = half * (t3 + t4);
    E[0][2] = half * (t3 - t4);
    E[1][1] = r.om_2 * D[1][1];
    E[2][1] = r.om_3 * D[2][1] + r.f3 * Fy;
    E[1][2] = r.om_3 * D[1][2] + r.f3 * Fx;
    E[2][2] = r.om_4 * D[2][2] + r.s4_9 * drho;

    // inverse y shift: back to x-moments of each velocity row
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        const C cm = (m == 0) ? C(1) : (m == 1) ? C(0) : third;
        const C K0 = rho0 * cm + E[m][0];
        const C r1 = E[m][1] + uy * K0;
        const C R2 = (E[m][2] + two * uy * E[m][1]) + uy2 * K0;
        h[m][1] = E[m][0] - R2;
        h[m][2] = half * (R2 + r1);
        h[m][0] = half * (R2 - r1);
    }
    // inverse x shift: back to populations
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        const C K0 = rho0 * wr[b] + h[0][b];
        const C r1 = h[1][b] + ux * K0;
        const C R2 = (h[2][b] + two * ux * h[1][b]) + ux2 * K0;
        q[1][b] = h[0][b] - R2;
        q[2][b] = half * (R2 + r1);
        q[0][b] = half * (R2 - r1);
    }
    g[7] = q[0][0]; g[4] = q[1][0]; g[8] = q[2][0];
    g[3] = q[0][1]; g[0] = q[1][1]; g[1] = q[2][1];
    g[6] = q[0][2]; g[2] = q[1][2]; g[5] = q[2][2];
}

// Deviations of the generalized equilibrium (central moments Eq. 8) about
// (rho0 + drho, u): the inverse of the two shifts applied to D = drho c_m c_n.
template <class C>
__device__ __forceinline__ void equilibrium_dev(C drho, C ux, C uy, C rho0, C (&g)[9]) {
    const C half = C(0.5), two = C(2), third = C(1) / C(3);
    const C wr[3] = {C(1) / C(6), C(2) / C(3), C(1) / C(6)};
    const C ux2 = ux * ux, uy2 = uy * uy;
    C h[3][3];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        const C cm = (m == 0) ? C(1) : (m == 1) ? C(0) : third;
        const C E0 = drho * cm, E1 = C(0), E2 = drho * cm * third;
        const C K0 = rho0 * cm + E0;
        const C r1 = E1 + uy * K0;
        const C R2 = (E2 + two * uy * E1) + uy2 * K0;
        h[m][1] = E0 - R2;
        h[m][2] = half * (R2 + r1);
        h[m][0] = half * (R2 - r1);
    }
    C q[3][3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        const C K0 = rho0 * wr[b] + h[0][b];
        const C r1 = h[1][b] + ux * K0;
        const C R2 = (h[2][b] + two * ux * h[1][b]) + ux2 * K0;
        q[1][b] = h[0][b] - R2;
        q[2][b] = half * (R2 + r1);
        q[0][b] = half * (R2 - r1);
    }
    g[7] = q[0][0]; g[4] = q[1][0]; g[8] = q[2][0];
    g[3] = q[0][1]; g[0] = q[1][1]; g[1] = q[2][1];
    g[6] = q[0][2]; g[2] = q[1][2]; g[5] = q[2][2];
}

}  // namespace clbm
