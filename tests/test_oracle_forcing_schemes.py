"""Pins of the oracle's comparison forcing schemes (Sec. 3 of Fei & Luo,
arXiv:1705.11092): M1 of Premnath et al. (Eq. 17-20) and M2 of Lycett-Brown
and Luo (Eq. 21), checked against the M1 and M2 columns of Table 1 and
Table 2, Remarks 5 and 6, and a closed form of the central moments of
Guo's force term.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from oracle import analytic as A
from paper_1705_11092_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], dtype=float)
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1], dtype=float)


def read_table2(column):
    out = {}
    with open(os.path.join(GOLDEN, "table2_taylor_green_m1_m2.txt")) as fh:
        for line in fh:
            f = line.split("#")[0].split()
            if f and f[0] == column:
                out[(int(f[1]), int(f[2]))] = float(f[3]) * 1e-2
    return out


def taylor_green_e2(N, Re, c_mode, u0=0.05, tol=1e-9):
    """Sec. 4B run for a forcing scheme (s1 = s2 for M2, 1 otherwise; Sec. 4).
    Stop when E_R < 1e-9 (every 1000 steps); if the symmetric state turns
    unstable first (E_R rises again after falling below 1e-8), E2 is read at
    the E_R minimum."""
    nu = u0 * N / Re
    s2 = A.shear_rate(nu)
    s1 = s2 if c_mode == O.FORCING_M2 else 1.0
    S = O.rates(1.0, s1, s2, s2, 1.0, 1.0)
    phi = 2 * math.pi / N
    ux, uy = A.taylor_green(N, N, u0, phi)
    Fx, Fy = A.taylor_green_force(N, N, u0, phi, nu)
    L = O.Lattice(N, N, S, Fx, Fy, c_mode=c_mode)
    f = L.equilibrium(1.0, ux, uy)
    _, uo, vo = L.moments(f)
    best = (np.inf, None)
    for _ in range(1000):
        f = L.run(f, 1000)
        _, u, v = L.moments(f)
        er = A.e_r(u, v, uo, vo)
        uo, vo = u, v
        e2 = A.e2(u, v, ux, uy)
        if er < tol:
            return e2
        if er < best[0]:
            best = (er, e2)
        elif best[0] < 1e-8 and er > 10 * best[0]:
            return best[1]
    return best[1]


T2_M1 = read_table2("M1")
T2_M2 = read_table2("M2")


@pytest.mark.parametrize("N,Re", [(10, 50), (10, 100), (10, 150), (20, 50), (20, 100), (20, 150)])
def test_table2_m1_column(N, Re):
    e = taylor_green_e2(N, Re, O.FORCING_M1)
    assert round(e * 1e2, 4) == pytest.approx(T2_M1[(N, Re)] * 1e2, abs=1e-12), e


@pytest.mark.parametrize("N,Re", [(10, 50), (10, 100), (10, 150), (20, 50), (20, 100), (20, 150)])
def test_table2_m2_column(N, Re):
    e = taylor_green_e2(N, Re, O.FORCING_M2)
    assert round(e * 1e2, 4) == pytest.approx(T2_M2[(N, Re)] * 1e2, abs=1e-12), e


def channel_e2(Fx, c_mode, tol=1e-9):
    """Table 1 channel: 50 fluid nodes across, s3 from the non-slip rule,
    other rates 1.754 (s1 = s2 for M2, 1 otherwise)."""
    s2 = 1.754
    s1 = s2 if c_mode == O.FORCING_M2 else 1.0
    S = O.rates(1.0, s1, s2, s2, A.nonslip_s3(s2), s2)
    H, nx = 50, 3
    solid = inputs.channel_mask(nx, H + 1)
    L = O.Lattice(nx, H + 1, S, Fx, 0.0, solid=solid, c_mode=c_mode)
    f = L.equilibrium(1.0, 0.0, 0.0)
    _, uo, vo = L.moments(f)
    for _ in range(3000):
        f = L.run(f, 1000)
        _, u, v = L.moments(f)
        er = A.e_r(u, v, uo, vo)
        uo, vo = u, v
        if er < tol:
            break
    y = np.arange(H + 1) - 0.5
    ua = A.poiseuille_steady(y, H, Fx, A.viscosity(s2))[:, None] * np.ones((1, nx))
    return A.e2(u, v, ua, 0 * ua, solid == 0)


def test_table1_m1_m2_columns():
    """Table 1: M1 2.739e-4 and M2 2.339e-4, the same for every Fx."""
    e1 = channel_e2(1e-6, O.FORCING_M1)
    e2 = channel_e2(1e-6, O.FORCING_M2)
    assert round(e1 * 1e4, 3) == 2.739
    assert round(e2 * 1e4, 3) == 2.339
    assert channel_e2(7e-6, O.FORCING_M1) == pytest.approx(e1, rel=1e-4)


def _state(rng):
    return O.equilibrium(rng.uniform(0.9, 1.1), *rng.uniform(-0.1, 0.1, 2)) * (
        1 + rng.uniform(-0.05, 0.05, 9))


def test_remark6_m1_equals_present_scheme_at_s3_2():
    rng = np.random.default_rng(6)
    for _ in range(20):
        f = _state(rng)
        Fx, Fy = rng.uniform(-1e-2, 1e-2, 2)
        S = O.rates(1.0, 1.0, 1.3, 1.6, 2.0, 1.1)
        a = O.collide_node(f, Fx, Fy, S, c_mode=O.C_DERIVED)
        b = O.collide_node(f, Fx, Fy, S, c_mode=O.FORCING_M1)
        np.testing.assert_allclose(a, b, rtol=0, atol=2e-15)
        S3 = O.rates(1.0, 1.0, 1.3, 1.6, 1.2, 1.1)
        a = O.collide_node(f, Fx, Fy, S3, c_mode=O.C_DERIVED)
        b = O.collide_node(f, Fx, Fy, S3, c_mode=O.FORCING_M1)
        assert np.abs(a - b).max() > 1e-6


def test_eq20_m1_rest_component():
    """Eq. 20: the rest component of Premnath's Delta f is -2 F.u + O(u^3).
    In the oracle's M1, Delta f is the distribution whose central moments
    are C_P, i.e. (N M)^-1 C_P; its rest component must have that form."""
    rng = np.random.default_rng(20)
    for _ in range(10):
        ux, uy = rng.uniform(-0.1, 0.1, 2)
        Fx, Fy = rng.uniform(-1e-3, 1e-3, 2)
        K = O.definition_matrix(ux, uy)
        df = np.linalg.solve(K, [0, Fx, Fy, 0, 0, 0, 0, 0, 0])
        lead = -2 * (Fx * ux + Fy * uy)
        assert abs(df[0] - lead) <= 4 * max(abs(Fx), abs(Fy)) * (abs(ux) + abs(uy)) ** 3


def test_remark5_momentum_for_each_scheme():
    """M1 keeps momentum (gains F) for any s1; M2 only when s1 = s2."""
    rng = np.random.default_rng(5)
    f = _state(rng)
    Fx, Fy = 3e-3, -1e-3
    for s1 in (0.7, 1.0, 1.6):
        S = O.rates(1.0, s1, 1.3, 1.6, 1.2, 1.1)
        fs = O.collide_node(f, Fx, Fy, S, c_mode=O.FORCING_M1)
        assert abs((fs * EX).sum() - (f * EX).sum() - Fx) < 1e-15
    S = O.rates(1.0, 1.6, 1.3, 1.6, 1.2, 1.1)
    fs = O.collide_node(f, Fx, Fy, S, c_mode=O.FORCING_M2)
    assert abs((fs * EX).sum() - (f * EX).sum() - Fx) < 1e-15
    S = O.rates(1.0, 1.0, 1.3, 1.6, 1.2, 1.1)
    fs = O.collide_node(f, Fx, Fy, S, c_mode=O.FORCING_M2)
    assert abs((fs * EX).sum() - (f * EX).sum() - Fx) > 1e-5


def test_guo_term_central_moments_closed_form():
    """Central moments of Guo's R_G (Remark 3), by brute force, equal
    [0, Fx, Fy, 0, 0, 0, Fy/3 - 2 ux uy Fx - ux^2 Fy,
     Fx/3 - 2 ux uy Fy - uy^2 Fx, 4 ux uy (uy Fx + ux Fy)]."""
    rng = np.random.default_rng(3)
    for _ in range(20):
        ux, uy = rng.uniform(-0.2, 0.2, 2)
        Fx, Fy = rng.uniform(-1e-2, 1e-2, 2)
        RG = O.guo_term(ux, uy, Fx, Fy)
        cx, cy = EX - ux, EY - uy
        k = lambda m, n: float(np.sum(RG * cx ** m * cy ** n))
        got = [k(0, 0), k(1, 0), k(0, 1), k(2, 0) + k(0, 2), k(2, 0) - k(0, 2), k(1, 1),
               k(2, 1), k(1, 2), k(2, 2)]
        expect = [0, Fx, Fy, 0, 0, 0, Fy / 3 - 2 * ux * uy * Fx - ux * ux * Fy,
                  Fx / 3 - 2 * ux * uy * Fy - uy * uy * Fx, 4 * ux * uy * (uy * Fx + ux * Fy)]
        np.testing.assert_allclose(got, expect, rtol=0, atol=1e-17)
