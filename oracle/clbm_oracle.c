/*
 * clbm_oracle.c -- plain, slow FP64 CPU oracle for one time step of the D2Q9
 * cascaded lattice Boltzmann method (CLBM) with the consistent forcing scheme
 * of Fei & Luo, "Consistent forcing scheme in the cascaded lattice Boltzmann
 * method" (arXiv:1705.11092).
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark may load this library.  It shares no code, table or
 * header with the CUDA path and it is never a fallback for it.
 *
 * Everything here follows the paper's formulas in the paper's order, in FP64,
 * with no blocking, fusion or reordering:
 *   - lattice: Sec. 2A, Eq. 1 (D2Q9 velocities, c = 1, cs^2 = 1/3);
 *   - moments: Eq. 2 (raw k_mn, central k~_mn) recombined as in Eq. 3;
 *   - "definition" mode computes the central moments T~ directly from Eq. 2-3
 *     and recovers f* by solving K(u) f* = T~* with K(u) = N(u) M built from
 *     the same definitions (Eq. 4), by LU with partial pivoting;
 *   - "printed" mode uses the matrices as printed: M (Eq. 5), N(u) (Eq. 6),
 *     M^-1 and N^-1(u) (Appendix);
 *   - collision with consistent forcing: Eq. 12 (first line), equilibrium
 *     central moments Eq. 8, forcing central moments Eq. 14 (see C_MODE_*);
 *   - macroscopic variables: Eq. 11 (density) and Eq. 15 (velocity);
 *   - streaming: Eq. 10 (push form), with halfway bounce-back at solid nodes
 *     (Sec. 4A: the wall lies half-way between a fluid node and a solid one);
 *   - equilibrium: the product-form "generalized local equilibrium" whose
 *     central moments are exactly Eq. 8 (the paper names it, Sec. 2A, but does
 *     not write it out; its 1-D factors are psi(0,u) = 2/3 - u^2 and
 *     psi(+-1,u) = (1/3 + u^2 +- u)/2).
 *   - reference steps for the algebraic reductions (Remarks 2 and 3): a raw
 *     moment MRT step with Guo-type forcing written in population space, and
 *     a BGK step with the force term R_i of Eq. 13 or Guo's R_Gi;
 *   - the comparison forcing schemes M1 (Eq. 17-19) and M2 (Eq. 21);
 *   - the Shan-Chen interaction force of Sec. 4C with the exponential
 *     pseudopotential, recomputed from the density before every collision.
 *
 * Layout: populations are 9 planes f[i][y][x] (index i*nx*ny + y*nx + x),
 * forces are per-node arrays fx[y*nx + x], fy[y*nx + x], the solid mask is
 * solid[y*nx + x] (nonzero = solid).  The lattice is periodic in x and y.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>
#include <stdlib.h>

/* ---- Eq. 1: D2Q9 discrete velocities ----------------------------------- */
static const int OR_EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int OR_EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

/* Direction with the opposite velocity (used by halfway bounce-back). */
static int or_opposite(int i)
{
    for (int j = 0; j < 9; ++j)
        if (OR_EX[j] == -OR_EX[i] && OR_EY[j] == -OR_EY[i]) return j;
    return -1;
}

/* Forcing schemes of Sec. 3, for the comparisons of Sec. 4:
 * FORCING_M1: Premnath et al. (Eq. 17-19): T~* = (I-S) T~ + S (T~eq - C_P/2),
 *   f* = M^-1 N^-1 T~* + Delta f, C_P = [0,Fx,Fy,0,0,0,0,0,0].  Delta f is the
 *   discrete distribution whose central moments are C_P (Delta f = (NM)^-1
 *   C_P); its rest component is -2 F.u + O(u^3), as Eq. 20 states.
 * FORCING_M2: Lycett-Brown and Luo (Eq. 21): T~* = (I-S) T~ + S T~eq
 *   + (1 - s2/2) N M R_G with Guo's R_G of Remark 3. */
enum { FORCING_M1 = 3, FORCING_M2 = 4 };

/* Forcing central moments C (Eq. 14).
 * C_MODE_DERIVED: C = [0,Fx,Fy,0,0,0,cs^2 Fy,cs^2 Fx,0].  This is what the
 *   central moments of R_i (Eq. 13) with the generalized equilibrium give in
 *   slots k~21 and k~12 (Eq. 2-3 order); at u = 0 it is exact.
 * C_MODE_PRINTED: the order as printed in Eq. 14, [..,cs^2 Fx,cs^2 Fy,0].
 * C_MODE_EXACT: C = N M R, the exact central moments of R_i computed from
 *   Eq. 13 by definition (used to check the BGK limit of Remark 3). */
enum { C_MODE_DERIVED = 0, C_MODE_PRINTED = 1, C_MODE_EXACT = 2 };

/* Collision modes. */
enum {
    MODE_DEFINITION = 0, /* Eq. 2-4 definitions, LU back-transform          */
    MODE_PRINTED = 1,    /* printed M, N, M^-1, N^-1                         */
    MODE_RAW_MRT = 2     /* N = I (Remark 2): raw moments relaxed towards
                            M f^eq, forcing term M R; definition + LU        */
};

static const double CS2 = 1.0 / 3.0;

/* integer power by repeated multiplication */
static double ipow(double b, int e)
{
    double r = 1.0;
    for (int k = 0; k < e; ++k) r *= b;
    return r;
}

/* Eq. 3: recombined moment k of the monomials (cx)^m (cy)^n. */
static double recombined_monomial(int k, double cx, double cy)
{
    switch (k) {
    case 0: return 1.0;                                   /* k00        */
    case 1: return cx;                                    /* k10        */
    case 2: return cy;                                    /* k01        */
    case 3: return ipow(cx, 2) + ipow(cy, 2);             /* k20 + k02  */
    case 4: return ipow(cx, 2) - ipow(cy, 2);             /* k20 - k02  */
    case 5: return cx * cy;                               /* k11        */
    case 6: return ipow(cx, 2) * cy;                      /* k21        */
    case 7: return cx * ipow(cy, 2);                      /* k12        */
    case 8: return ipow(cx, 2) * ipow(cy, 2);             /* k22        */
    }
    return 0.0;
}

/* K(u)[k][i]: row k of the map f -> T~ for shift velocity u (Eq. 2-4).
 * With u = 0 this is the raw-moment matrix M of Eq. 5. */
static void build_K(double ux, double uy, double K[9][9])
{
    for (int k = 0; k < 9; ++k)
        for (int i = 0; i < 9; ++i)
            K[k][i] = recombined_monomial(k, OR_EX[i] - ux, OR_EY[i] - uy);
}

/* Eq. 2-3 by definition: recombined central moments about (ux, uy). */
void oracle_central_moments(const double f[9], double ux, double uy, double T[9])
{
    for (int k = 0; k < 9; ++k) {
        double s = 0.0;
        for (int i = 0; i < 9; ++i)
            s += f[i] * recombined_monomial(k, OR_EX[i] - ux, OR_EY[i] - uy);
        T[k] = s;
    }
}

/* Solve A x = b (9x9) by LU with partial pivoting.  A and b are copied. */
static int lu_solve9(const double Ain[9][9], const double bin[9], double x[9])
{
    double A[9][9], b[9];
    memcpy(A, Ain, sizeof(A));
    memcpy(b, bin, sizeof(b));
    for (int c = 0; c < 9; ++c) {
        int p = c;
        for (int r = c + 1; r < 9; ++r)
            if (fabs(A[r][c]) > fabs(A[p][c])) p = r;
        if (A[p][c] == 0.0) return -1;
        if (p != c) {
            for (int j = 0; j < 9; ++j) { double t = A[c][j]; A[c][j] = A[p][j]; A[p][j] = t; }
            double t = b[c]; b[c] = b[p]; b[p] = t;
        }
        for (int r = c + 1; r < 9; ++r) {
            double l = A[r][c] / A[c][c];
            for (int j = c; j < 9; ++j) A[r][j] -= l * A[c][j];
            b[r] -= l * b[c];
        }
    }
    for (int r = 8; r >= 0; --r) {
        double s = b[r];
        for (int j = r + 1; j < 9; ++j) s -= A[r][j] * x[j];
        x[r] = s / A[r][r];
    }
    return 0;
}

/* Product-form generalized local equilibrium (its central moments are
 * Eq. 8 exactly): f^eq_i = rho psi(ex_i, ux) psi(ey_i, uy). */
static double psi1d(int c, double u)
{
    if (c == 0) return 2.0 / 3.0 - u * u;
    return (1.0 / 3.0 + u * u + c * u) / 2.0;
}

void oracle_equilibrium(double rho, double ux, double uy, double feq[9])
{
    for (int i = 0; i < 9; ++i)
        feq[i] = rho * psi1d(OR_EX[i], ux) * psi1d(OR_EY[i], uy);
}

/* Eq. 13: force effect term R_i = F.(e_i - u)/(rho cs^2) f^eq_i. */
void oracle_force_term(double rho, double ux, double uy, double Fx, double Fy, double R[9])
{
    double feq[9];
    oracle_equilibrium(rho, ux, uy, feq);
    for (int i = 0; i < 9; ++i)
        R[i] = (Fx * (OR_EX[i] - ux) + Fy * (OR_EY[i] - uy)) / (rho * CS2) * feq[i];
}

/* Remark 3: Guo's force term R_Gi = w_i[(e_i - u)/cs^2 + (e_i.u) e_i/cs^4].F */
static double weight(int i)
{
    /* the weights are the u = 0 equilibrium at rho = 1 */
    return psi1d(OR_EX[i], 0.0) * psi1d(OR_EY[i], 0.0);
}

void oracle_guo_term(double ux, double uy, double Fx, double Fy, double RG[9])
{
    for (int i = 0; i < 9; ++i) {
        double ex = OR_EX[i], ey = OR_EY[i];
        double eu = ex * ux + ey * uy;
        double ax = (ex - ux) / CS2 + eu * ex / (CS2 * CS2);
        double ay = (ey - uy) / CS2 + eu * ey / (CS2 * CS2);
        RG[i] = weight(i) * (ax * Fx + ay * Fy);
    }
}

/* Eq. 11 and Eq. 15: density and force-corrected velocity of a node. */
void oracle_macroscopic(const double f[9], double Fx, double Fy,
                        double* rho, double* ux, double* uy)
{
    double r = 0.0, jx = 0.0, jy = 0.0;
    for (int i = 0; i < 9; ++i) {
        r += f[i];
        jx += f[i] * OR_EX[i];
        jy += f[i] * OR_EY[i];
    }
    *rho = r;
    *ux = (jx + 0.5 * Fx) / r;
    *uy = (jy + 0.5 * Fy) / r;
}

/* ---- printed matrices ---------------------------------------------------- */

/* Eq. 5 */
static const double M_PRINTED[9][9] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1},
    {0, 1, 0, -1, 0, 1, -1, -1, 1},
    {0, 0, 1, 0, -1, 1, 1, -1, -1},
    {0, 1, 1, 1, 1, 2, 2, 2, 2},
    {0, 1, -1, 1, -1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 1, -1, 1, -1},
    {0, 0, 0, 0, 0, 1, 1, -1, -1},
    {0, 0, 0, 0, 0, 1, -1, -1, 1},
    {0, 0, 0, 0, 0, 1, 1, 1, 1},
};

/* Appendix: M^-1 */
static const double MINV_PRINTED[9][9] = {
    {1, 0, 0, -1, 0, 0, 0, 0, 1},
    {0, 0.5, 0, 0.25, 0.25, 0, 0, -0.5, -0.5},
    {0, 0, 0.5, 0.25, -0.25, 0, -0.5, 0, -0.5},
    {0, -0.5, 0, 0.25, 0.25, 0, 0, 0.5, -0.5},
    {0, 0, -0.5, 0.25, -0.25, 0, 0.5, 0, -0.5},
    {0, 0, 0, 0, 0, 0.25, 0.25, 0.25, 0.25},
    {0, 0, 0, 0, 0, -0.25, 0.25, -0.25, 0.25},
    {0, 0, 0, 0, 0, 0.25, -0.25, -0.25, 0.25},
    {0, 0, 0, 0, 0, -0.25, -0.25, 0.25, 0.25},
};

/* Eq. 6: shift matrix N(u), as printed */
void oracle_shift_matrix(double ux, double uy, double N[9][9])
{
    double x2 = ux * ux, y2 = uy * uy, xy = ux * uy;
    double R[9][9] = {
        {1, 0, 0, 0, 0, 0, 0, 0, 0},
        {-ux, 1, 0, 0, 0, 0, 0, 0, 0},
        {-uy, 0, 1, 0, 0, 0, 0, 0, 0},
        {x2 + y2, -2 * ux, -2 * uy, 1, 0, 0, 0, 0, 0},
        {x2 - y2, -2 * ux, 2 * uy, 0, 1, 0, 0, 0, 0},
        {xy, -uy, -ux, 0, 0, 1, 0, 0, 0},
        {-x2 * uy, 2 * xy, x2, -uy / 2, -uy / 2, -2 * ux, 1, 0, 0},
        {-y2 * ux, y2, 2 * xy, -ux / 2, ux / 2, -2 * uy, 0, 1, 0},
        {x2 * y2, -2 * ux * y2, -2 * uy * x2, x2 / 2 + y2 / 2, y2 / 2 - x2 / 2,
         4 * xy, -2 * uy, -2 * ux, 1},
    };
    memcpy(N, R, sizeof(R));
}

/* Appendix: N^-1(u), as printed */
void oracle_shift_matrix_inverse(double ux, double uy, double Ni[9][9])
{
    double x2 = ux * ux, y2 = uy * uy, xy = ux * uy;
    double R[9][9] = {
        {1, 0, 0, 0, 0, 0, 0, 0, 0},
        {ux, 1, 0, 0, 0, 0, 0, 0, 0},
        {uy, 0, 1, 0, 0, 0, 0, 0, 0},
        {x2 + y2, 2 * ux, 2 * uy, 1, 0, 0, 0, 0, 0},
        {x2 - y2, 2 * ux, -2 * uy, 0, 1, 0, 0, 0, 0},
        {xy, uy, ux, 0, 0, 1, 0, 0, 0},
        {x2 * uy, 2 * xy, x2, uy / 2, uy / 2, 2 * ux, 1, 0, 0},
        {y2 * ux, y2, 2 * xy, ux / 2, -ux / 2, 2 * uy, 0, 1, 0},
        {x2 * y2, 2 * ux * y2, 2 * uy * x2, x2 / 2 + y2 / 2, y2 / 2 - x2 / 2,
         4 * xy, 2 * uy, 2 * ux, 1},
    };
    memcpy(Ni, R, sizeof(R));
}

void oracle_transform_matrix(double M[9][9]) { memcpy(M, M_PRINTED, sizeof(M_PRINTED)); }
void oracle_transform_matrix_inverse(double Mi[9][9]) { memcpy(Mi, MINV_PRINTED, sizeof(MINV_PRINTED)); }

/* K(u) = N(u) M from the definitions (exported for the matrix pins). */
void oracle_definition_matrix(double ux, double uy, double K[9][9]) { build_K(ux, uy, K); }

static void matvec9(const double A[9][9], const double x[9], double y[9])
{
    for (int r = 0; r < 9; ++r) {
        double s = 0.0;
        for (int c = 0; c < 9; ++c) s += A[r][c] * x[c];
        y[r] = s;
    }
}

/* Eq. 14 forcing central moments, per the chosen reading. */
static void forcing_moments(int c_mode, double rho, double ux, double uy,
                            double Fx, double Fy, double C[9])
{
    for (int k = 0; k < 9; ++k) C[k] = 0.0;
    if (c_mode == C_MODE_EXACT) {
        double R[9];
        oracle_force_term(rho, ux, uy, Fx, Fy, R);
        oracle_central_moments(R, ux, uy, C);
        return;
    }
    C[1] = Fx;
    C[2] = Fy;
    if (c_mode == C_MODE_PRINTED) {
        C[6] = CS2 * Fx;
        C[7] = CS2 * Fy;
    } else {
        C[6] = CS2 * Fy;
        C[7] = CS2 * Fx;
    }
}

/*
 * One collision at one node: f (pre-collision) -> fstar (post-collision).
 * s[9] is the diagonal of S in Eq. 7 order (s0, s1, s1, sb, s2, s2, s3, s3, s4).
 * Returns 0, or -1 if the back-transform is singular.
 */
int oracle_collide_node(const double f[9], double Fx, double Fy, const double s[9],
                        int mode, int c_mode, double fstar[9])
{
    double rho, ux, uy;
    oracle_macroscopic(f, Fx, Fy, &rho, &ux, &uy);          /* Eq. 11, 15 */

    if (c_mode == FORCING_M1 || c_mode == FORCING_M2) {
        double Tt[9], K[9][9];
        oracle_central_moments(f, ux, uy, Tt);                 /* Eq. 2-3 */
        build_K(ux, uy, K);
        double Teq[9] = {rho, 0, 0, 2.0 * rho * CS2, 0, 0, 0, 0, rho * CS2 * CS2};
        double Ts[9];
        if (c_mode == FORCING_M1) {
            const double CP[9] = {0, Fx, Fy, 0, 0, 0, 0, 0, 0};            /* Eq. 19 */
            for (int k = 0; k < 9; ++k)
                Ts[k] = (1.0 - s[k]) * Tt[k] + s[k] * (Teq[k] - 0.5 * CP[k]);  /* Eq. 17 */
            double fs[9], df[9];
            if (lu_solve9((const double(*)[9])K, Ts, fs)) return -1;
            if (lu_solve9((const double(*)[9])K, CP, df)) return -1;
            for (int i = 0; i < 9; ++i) fstar[i] = fs[i] + df[i];        /* Eq. 18 */
            return 0;
        }
        double RG[9], CG[9];
        oracle_guo_term(ux, uy, Fx, Fy, RG);                   /* Remark 3 */
        oracle_central_moments(RG, ux, uy, CG);                /* N M R_G */
        for (int k = 0; k < 9; ++k)
            Ts[k] = (1.0 - s[k]) * Tt[k] + s[k] * Teq[k] + (1.0 - 0.5 * s[4]) * CG[k];   /* Eq. 21 */
        return lu_solve9((const double(*)[9])K, Ts, fstar);
    }

    if (mode == MODE_RAW_MRT) {
        /* Remark 2: N = I.  T* = (I-S) M f + S M f^eq + (I - S/2) M R. */
        double K0[9][9], T[9], Teq[9], TR[9], feq[9], R[9], Ts[9];
        build_K(0.0, 0.0, K0);
        oracle_equilibrium(rho, ux, uy, feq);
        oracle_force_term(rho, ux, uy, Fx, Fy, R);
        matvec9(K0, f, T);
        matvec9(K0, feq, Teq);
        matvec9(K0, R, TR);
        for (int k = 0; k < 9; ++k)
            Ts[k] = (1.0 - s[k]) * T[k] + s[k] * Teq[k] + (1.0 - 0.5 * s[k]) * TR[k];
        return lu_solve9((const double(*)[9])K0, Ts, fstar);
    }

    double Tt[9];
    if (mode == MODE_PRINTED) {
        double N[9][9], T[9];
        matvec9(M_PRINTED, f, T);                              /* Eq. 4  */
        oracle_shift_matrix(ux, uy, N);
        matvec9((const double(*)[9])N, T, Tt);                 /* Eq. 4  */
    } else {
        oracle_central_moments(f, ux, uy, Tt);                 /* Eq. 2-3 */
    }

    /* Eq. 8: equilibrium central moments */
    double Teq[9] = {rho, 0, 0, 2.0 * rho * CS2, 0, 0, 0, 0, rho * CS2 * CS2};
    double C[9];
    forcing_moments(c_mode, rho, ux, uy, Fx, Fy, C);           /* Eq. 14 */

    /* Eq. 12 (first line) */
    double Ts[9];
    for (int k = 0; k < 9; ++k)
        Ts[k] = (1.0 - s[k]) * Tt[k] + s[k] * Teq[k] + (1.0 - 0.5 * s[k]) * C[k];

    /* Eq. 9: f* = M^-1 N^-1 T~* */
    if (mode == MODE_PRINTED) {
        double Ni[9][9], T[9];
        oracle_shift_matrix_inverse(ux, uy, Ni);
        matvec9((const double(*)[9])Ni, Ts, T);
        matvec9(MINV_PRINTED, T, fstar);
        return 0;
    }
    double K[9][9];
    build_K(ux, uy, K);
    return lu_solve9((const double(*)[9])K, Ts, fstar);
}

/*
 * Reference MRT step with N = I written in population space (Remark 2):
 *   f* = f - M^-1 S M (f - f^eq) + M^-1 (I - S/2) M R,
 * with the printed M and M^-1, the product-form f^eq and R_i of Eq. 13.
 */
void oracle_mrt_guo_node(const double f[9], double Fx, double Fy, const double s[9],
                         double fstar[9])
{
    double rho, ux, uy, feq[9], R[9], d[9], Md[9], MR[9], w[9], out[9];
    oracle_macroscopic(f, Fx, Fy, &rho, &ux, &uy);
    oracle_equilibrium(rho, ux, uy, feq);
    oracle_force_term(rho, ux, uy, Fx, Fy, R);
    for (int i = 0; i < 9; ++i) d[i] = f[i] - feq[i];
    matvec9(M_PRINTED, d, Md);
    matvec9(M_PRINTED, R, MR);
    for (int k = 0; k < 9; ++k) w[k] = -s[k] * Md[k] + (1.0 - 0.5 * s[k]) * MR[k];
    matvec9(MINV_PRINTED, w, out);
    for (int i = 0; i < 9; ++i) fstar[i] = f[i] + out[i];
}

/*
 * Reference BGK step (Remark 3): f* = f - s (f - f^eq) + (1 - s/2) Q, where
 * Q is R_i of Eq. 13 (guo = 0) or Guo's R_Gi (guo = 1).
 */
void oracle_bgk_node(const double f[9], double Fx, double Fy, double s, int guo,
                     double fstar[9])
{
    double rho, ux, uy, feq[9], Q[9];
    oracle_macroscopic(f, Fx, Fy, &rho, &ux, &uy);
    oracle_equilibrium(rho, ux, uy, feq);
    if (guo) oracle_guo_term(ux, uy, Fx, Fy, Q);
    else oracle_force_term(rho, ux, uy, Fx, Fy, Q);
    for (int i = 0; i < 9; ++i)
        fstar[i] = f[i] - s * (f[i] - feq[i]) + (1.0 - 0.5 * s) * Q[i];
}

/* ---- lattice drivers ----------------------------------------------------- */

static size_t idx(int nx, int x, int y) { return (size_t)y * (size_t)nx + (size_t)x; }

/*
 * Collision at every fluid node: f_pre -> f_post (same layout).
 * Solid nodes are set to zero.  Returns 0 or -1 on a singular solve.
 */
int oracle_collide_lattice(int nx, int ny, const double s[9],
                           const double* fx, const double* fy,
                           const uint8_t* solid, int mode, int c_mode,
                           const double* f_pre, double* f_post)
{
    size_t n = (size_t)nx * (size_t)ny;
    int err = 0;
#pragma omp parallel for schedule(static) reduction(| : err)
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            size_t p = idx(nx, x, y);
            if (solid && solid[p]) {
                for (int i = 0; i < 9; ++i) f_post[i * n + p] = 0.0;
                continue;
            }
            double f[9], fs[9];
            for (int i = 0; i < 9; ++i) f[i] = f_pre[i * n + p];
            if (oracle_collide_node(f, fx[p], fy[p], s, mode, c_mode, fs)) err = 1;
            for (int i = 0; i < 9; ++i) f_post[i * n + p] = fs[i];
        }
    }
    return err ? -1 : 0;
}

/*
 * Eq. 10 streaming in push form with halfway bounce-back:
 *   f_i(x + e_i, t+1) = f*_i(x, t)        if x + e_i is fluid,
 *   f_opp(i)(x, t+1)  = f*_i(x, t)        if x + e_i is solid.
 * Periodic wrap in x and y.  Solid nodes of f_next are zero.
 */
void oracle_stream(int nx, int ny, const uint8_t* solid, const double* f_post, double* f_next)
{
    size_t n = (size_t)nx * (size_t)ny;
    for (size_t k = 0; k < 9 * n; ++k) f_next[k] = 0.0;
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            size_t p = idx(nx, x, y);
            if (solid && solid[p]) continue;
            for (int i = 0; i < 9; ++i) {
                int xt = ((x + OR_EX[i]) % nx + nx) % nx;
                int yt = ((y + OR_EY[i]) % ny + ny) % ny;
                size_t q = idx(nx, xt, yt);
                if (solid && solid[q])
                    f_next[(size_t)or_opposite(i) * n + p] = f_post[i * n + p];
                else
                    f_next[i * n + q] = f_post[i * n + p];
            }
        }
    }
}

/*
 * nsteps full time steps (collide, then stream) on the pre-collision state f,
 * in place.  Returns 0 or -1.
 */
int oracle_run(int nx, int ny, const double s[9], const double* fx, const double* fy,
               const uint8_t* solid, int mode, int c_mode, double* f, int nsteps)
{
    size_t n = 9 * (size_t)nx * (size_t)ny;
    double* post = (double*)malloc(n * sizeof(double));
    if (!post) return -2;
    int err = 0;
    for (int t = 0; t < nsteps && !err; ++t) {
        err = oracle_collide_lattice(nx, ny, s, fx, fy, solid, mode, c_mode, f, post);
        oracle_stream(nx, ny, solid, post, f);
    }
    free(post);
    return err;
}

/*
 * Macroscopic fields of a pre-collision state (Eq. 11, Eq. 15).  Solid
 * nodes get rho = ux = uy = 0.
 */
void oracle_moments(int nx, int ny, const double* fx, const double* fy,
                    const uint8_t* solid, const double* f, double* rho, double* ux, double* uy)
{
    size_t n = (size_t)nx * (size_t)ny;
    for (size_t p = 0; p < n; ++p) {
        if (solid && solid[p]) { rho[p] = ux[p] = uy[p] = 0.0; continue; }
        double g[9];
        for (int i = 0; i < 9; ++i) g[i] = f[i * n + p];
        oracle_macroscopic(g, fx[p], fy[p], &rho[p], &ux[p], &uy[p]);
    }
}

/* Product-form equilibrium on every fluid node (solid nodes zero). */
void oracle_equilibrium_lattice(int nx, int ny, const uint8_t* solid, const double* rho,
                                const double* ux, const double* uy, double* f)
{
    size_t n = (size_t)nx * (size_t)ny;
    for (size_t p = 0; p < n; ++p) {
        double feq[9];
        if (solid && solid[p]) { for (int i = 0; i < 9; ++i) f[i * n + p] = 0.0; continue; }
        oracle_equilibrium(rho[p], ux[p], uy[p], feq);
        for (int i = 0; i < 9; ++i) f[i * n + p] = feq[i];
    }
}

/* ---- Sec. 4C: Shan-Chen pseudopotential force --------------------------- */

/* psi(rho) = psi0 exp(-rho0 / rho): the exponential pseudopotential. */
double oracle_sc_psi(double rho, double psi0, double rho0)
{
    return psi0 * exp(-rho0 / rho);
}

/* Pressure of the Shan-Chen fluid, p = rho cs^2 + G psi^2 / 2. */
double oracle_sc_pressure(double rho, double G, double psi0, double rho0)
{
    double psi = oracle_sc_psi(rho, psi0, rho0);
    return rho * CS2 + 0.5 * G * psi * psi;
}

/*
 * Interaction force of every node of a periodic nx-by-ny density field:
 *   F(x) = -G psi(x) sum_i w_i psi(x + e_i) e_i,
 * nearest-neighbour weights w_i = 1/3 for |e_i|^2 = 1 and 1/12 for
 * |e_i|^2 = 2, summed over i = 1..8 in the velocity order of Eq. 1.
 */
void oracle_sc_force(int nx, int ny, const double* rho, double G, double psi0, double rho0,
                     double* Fx, double* Fy)
{
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            double sx = 0.0, sy = 0.0;
            for (int i = 1; i < 9; ++i) {
                int xt = ((x + OR_EX[i]) % nx + nx) % nx;
                int yt = ((y + OR_EY[i]) % ny + ny) % ny;
                double w = (OR_EX[i] * OR_EX[i] + OR_EY[i] * OR_EY[i] == 1) ? 1.0 / 3.0 : 1.0 / 12.0;
                double ps = oracle_sc_psi(rho[idx(nx, xt, yt)], psi0, rho0);
                sx += w * ps * OR_EX[i];
                sy += w * ps * OR_EY[i];
            }
            double pc = oracle_sc_psi(rho[idx(nx, x, y)], psi0, rho0);
            Fx[idx(nx, x, y)] = -G * pc * sx;
            Fy[idx(nx, x, y)] = -G * pc * sy;
        }
    }
}

/* Density (Eq. 11) of every node of a pre-collision state. */
void oracle_density(int nx, int ny, const double* f, double* rho)
{
    size_t n = (size_t)nx * (size_t)ny;
    for (size_t p = 0; p < n; ++p) {
        double r = 0.0;
        for (int i = 0; i < 9; ++i) r += f[i * n + p];
        rho[p] = r;
    }
}

/*
 * nsteps time steps of a Shan-Chen fluid on a periodic lattice without solid
 * nodes, in place on the pre-collision state f: each step takes the density
 * of f, the interaction force from it, then collides with that force (Eq. 12)
 * and streams (Eq. 10).  Returns 0, -1 (singular solve) or -2 (no memory).
 */
int oracle_run_sc(int nx, int ny, const double s[9], double G, double psi0, double rho0,
                  int mode, int c_mode, double* f, int nsteps)
{
    size_t n = (size_t)nx * (size_t)ny;
    double* post = (double*)malloc(9 * n * sizeof(double));
    double* rho = (double*)malloc(n * sizeof(double));
    double* Fx = (double*)malloc(n * sizeof(double));
    double* Fy = (double*)malloc(n * sizeof(double));
    int err = (!post || !rho || !Fx || !Fy) ? -2 : 0;
    for (int t = 0; t < nsteps && !err; ++t) {
        oracle_density(nx, ny, f, rho);
        oracle_sc_force(nx, ny, rho, G, psi0, rho0, Fx, Fy);
        err = oracle_collide_lattice(nx, ny, s, Fx, Fy, NULL, mode, c_mode, f, post);
        oracle_stream(nx, ny, NULL, post, f);
    }
    free(post);
    free(rho);
    free(Fx);
    free(Fy);
    return err;
}

int oracle_has_openmp(void)
{
#ifdef _OPENMP
    return 1;
#else
    return 0;
#endif
}
