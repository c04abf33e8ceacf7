"""Pins of the oracle's per-node algebra against what the paper fixes.

Fei & Luo, arXiv:1705.11092: Eq. 1-9 (moments, shift matrix, collision),
Eq. 12-15 (consistent forcing), Appendix (printed inverses), Remarks 2, 3, 5.
Every expected value here is either printed in the paper or follows from a
closed form; the brute-force moment sums are written out in numpy in this
file, independently of the oracle's C code.
"""
import numpy as np
import pytest

import oracle as O

EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], dtype=float)  # Eq. 1
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1], dtype=float)
CS2 = 1.0 / 3.0


def brute_central(f, ux, uy):
    """Eq. 2 then Eq. 3, by direct summation in numpy."""
    cx, cy = EX - ux, EY - uy
    k = lambda m, n: float(np.sum(f * cx ** m * cy ** n))
    return np.array([k(0, 0), k(1, 0), k(0, 1), k(2, 0) + k(0, 2), k(2, 0) - k(0, 2),
                     k(1, 1), k(2, 1), k(1, 2), k(2, 2)])


@pytest.fixture(scope="module")
def rng():
    return np.random.default_rng(20170531)


# ---- P1: printed matrices -------------------------------------------------

def test_printed_M_times_printed_Minv_is_identity():
    M, Mi = O.transform_matrix(), O.transform_matrix_inverse()
    assert np.array_equal(M @ Mi, np.eye(9))
    assert np.array_equal(Mi @ M, np.eye(9))


def test_printed_M_is_raw_moment_definition():
    # Eq. 4-5: row k of M is the recombined monomial of e_i (Eq. 2-3, u = 0)
    M = O.transform_matrix()
    for i in range(9):
        e = np.zeros(9)
        e[i] = 1.0
        assert np.array_equal(M[:, i], brute_central(e, 0.0, 0.0))


def test_printed_N_is_shift_definition(rng):
    # Eq. 4 and 6: T~ = N(u) M f for every f, with T~ the central moments.
    M = O.transform_matrix()
    for _ in range(20):
        ux, uy = rng.uniform(-0.4, 0.4, 2)
        f = rng.uniform(0.0, 1.0, 9)
        N = O.shift_matrix(ux, uy)
        np.testing.assert_allclose(N @ (M @ f), brute_central(f, ux, uy), rtol=0, atol=2e-15)
        np.testing.assert_allclose(O.definition_matrix(ux, uy), N @ M, rtol=0, atol=1e-15)


def test_printed_Ninv_is_inverse_and_N_of_minus_u(rng):
    for _ in range(20):
        ux, uy = rng.uniform(-0.4, 0.4, 2)
        N, Ni = O.shift_matrix(ux, uy), O.shift_matrix_inverse(ux, uy)
        np.testing.assert_allclose(N @ Ni, np.eye(9), rtol=0, atol=1e-15)
        np.testing.assert_allclose(Ni @ N, np.eye(9), rtol=0, atol=1e-15)
        np.testing.assert_array_equal(Ni, O.shift_matrix(-ux, -uy))


def test_oracle_central_moments_match_brute_force(rng):
    for _ in range(20):
        ux, uy = rng.uniform(-0.3, 0.3, 2)
        f = rng.uniform(0.0, 1.0, 9)
        np.testing.assert_allclose(O.central_moments(f, ux, uy), brute_central(f, ux, uy),
                                   rtol=1e-14, atol=1e-15)


# ---- P2: equilibrium has the central moments of Eq. 8 ---------------------

def test_equilibrium_central_moments_are_eq8(rng):
    for _ in range(20):
        rho = rng.uniform(0.5, 2.0)
        ux, uy = rng.uniform(-0.3, 0.3, 2)
        feq = O.equilibrium(rho, ux, uy)
        expect = np.array([rho, 0, 0, 2 * rho * CS2, 0, 0, 0, 0, rho * CS2 * CS2])
        np.testing.assert_allclose(brute_central(feq, ux, uy), expect, rtol=0, atol=1e-15)
        # and its raw first moments are rho u (Eq. 11)
        assert abs(np.sum(feq * EX) - rho * ux) < 1e-15
        assert abs(np.sum(feq * EY) - rho * uy) < 1e-15


def test_equilibrium_at_rest_is_d2q9_weights():
    w = O.equilibrium(1.0, 0.0, 0.0)
    np.testing.assert_allclose(w, [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4, rtol=0, atol=1e-16)


# ---- P3: forcing central moments (Eq. 13-14) --------------------------------

def test_force_term_central_moments(rng):
    """Central moments of R_i (Eq. 13) = C (derived slot order) plus the
    closed-form O(F u^3) terms of the product-form equilibrium."""
    for _ in range(30):
        rho = rng.uniform(0.7, 1.5)
        ux, uy = rng.uniform(-0.2, 0.2, 2)
        Fx, Fy = rng.uniform(-1e-2, 1e-2, 2)
        R = O.force_term(rho, ux, uy, Fx, Fy)
        got = brute_central(R, ux, uy)
        C = np.array([0, Fx, Fy, 0, 0, 0, CS2 * Fy, CS2 * Fx, 0])
        a = Fx * ux ** 3
        b = Fy * uy ** 3
        extra = np.array([0, 0, 0, -3 * (a + b), -3 * (a - b), 0, 0, 0, -(a + b)])
        np.testing.assert_allclose(got, C + extra, rtol=0, atol=1e-16)


def test_force_moments_at_rest_pin_slot_order():
    """At u = 0 central = raw moments and M R = C exactly: k~21 carries Fy/3
    and k~12 carries Fx/3 (the printed Eq. 14 lists them the other way)."""
    Fx, Fy = 3e-3, -7e-3
    R = O.force_term(1.0, 0.0, 0.0, Fx, Fy)
    MR = O.transform_matrix() @ R
    np.testing.assert_allclose(MR, [0, Fx, Fy, 0, 0, 0, Fy / 3, Fx / 3, 0], rtol=0, atol=1e-18)


# ---- collision invariants (Eq. 12, Remark 5) ------------------------------

def _random_state(rng):
    rho = rng.uniform(0.8, 1.2)
    ux, uy = rng.uniform(-0.1, 0.1, 2)
    return O.equilibrium(rho, ux, uy) * (1.0 + rng.uniform(-0.05, 0.05, 9))


@pytest.mark.parametrize("mode", [O.MODE_DEFINITION, O.MODE_PRINTED])
def test_mass_conserved_momentum_gains_force(rng, mode):
    for _ in range(20):
        f = _random_state(rng)
        Fx, Fy = rng.uniform(-1e-3, 1e-3, 2)
        s = rng.uniform(0.3, 1.9, 6)
        S = O.rates(*s)
        fs = O.collide_node(f, Fx, Fy, S, mode)
        assert abs(fs.sum() - f.sum()) < 2e-15
        assert abs((fs * EX).sum() - (f * EX).sum() - Fx) < 2e-15
        assert abs((fs * EY).sum() - (f * EY).sum() - Fy) < 2e-15


def test_independent_of_s0_and_s1(rng):
    """Remark 5: the conserved-moment rates can be chosen freely."""
    for _ in range(10):
        f = _random_state(rng)
        Fx, Fy = rng.uniform(-1e-3, 1e-3, 2)
        base = dict(sb=1.3, s2=1.6, s3=0.9, s4=1.1)
        a = O.collide_node(f, Fx, Fy, O.rates(s0=1.0, s1=1.0, **base))
        b = O.collide_node(f, Fx, Fy, O.rates(s0=0.4, s1=1.7, **base))
        np.testing.assert_allclose(a, b, rtol=0, atol=2e-15)


def test_definition_and_printed_modes_agree(rng):
    """P14: LU on the definition matrix vs the printed M, N, M^-1, N^-1."""
    for _ in range(50):
        f = _random_state(rng)
        Fx, Fy = rng.uniform(-1e-2, 1e-2, 2)
        S = O.rates(*rng.uniform(0.2, 1.95, 6))
        a = O.collide_node(f, Fx, Fy, S, O.MODE_DEFINITION)
        b = O.collide_node(f, Fx, Fy, S, O.MODE_PRINTED)
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-15)


def test_relaxed_central_moments_follow_eq12(rng):
    """Central moments of f* about the same u equal Eq. 12's T~*."""
    for _ in range(20):
        f = _random_state(rng)
        Fx, Fy = rng.uniform(-1e-2, 1e-2, 2)
        s = rng.uniform(0.3, 1.9, 6)
        S = O.rates(*s)
        rho, ux, uy = O.macroscopic(f, Fx, Fy)
        T = brute_central(f, ux, uy)
        Teq = np.array([rho, 0, 0, 2 * rho / 3, 0, 0, 0, 0, rho / 9])
        C = np.array([0, Fx, Fy, 0, 0, 0, Fy / 3, Fx / 3, 0])
        expect = (1 - S) * T + S * Teq + (1 - S / 2) * C
        got = brute_central(O.collide_node(f, Fx, Fy, S), ux, uy)
        np.testing.assert_allclose(got, expect, rtol=0, atol=2e-15)


# ---- P6: algebraic reductions (Remarks 2 and 3) ---------------------------

def test_shift_off_is_population_space_mrt(rng):
    """Remark 2: with N = I the scheme is MRT with force term M R."""
    for _ in range(20):
        f = _random_state(rng)
        Fx, Fy = rng.uniform(-1e-2, 1e-2, 2)
        S = O.rates(*rng.uniform(0.3, 1.9, 6))
        a = O.collide_node(f, Fx, Fy, S, O.MODE_RAW_MRT)
        b = O.mrt_guo_node(f, Fx, Fy, S)
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-15)


def test_bgk_limit_with_exact_forcing_moments(rng):
    """Remark 3: all rates equal and C = N M R exactly -> BGK with R_i."""
    for _ in range(20):
        f = _random_state(rng)
        Fx, Fy = rng.uniform(-1e-2, 1e-2, 2)
        s = rng.uniform(0.3, 1.9)
        a = O.collide_node(f, Fx, Fy, O.rates(s, s, s, s, s, s), c_mode=O.C_EXACT)
        b = O.bgk_node(f, Fx, Fy, s)
        np.testing.assert_allclose(a, b, rtol=0, atol=2e-15)


def test_bgk_limit_with_eq14_differs_by_closed_form(rng):
    """With the Eq. 14 moments the BGK-limit difference is
    -(1 - s/2) (N M)^-1 [extra O(F u^3) moments], built from the printed
    inverses."""
    Mi = O.transform_matrix_inverse()
    for _ in range(20):
        f = _random_state(rng)
        Fx, Fy = rng.uniform(-1e-2, 1e-2, 2)
        s = rng.uniform(0.3, 1.9)
        rho, ux, uy = O.macroscopic(f, Fx, Fy)
        a = O.collide_node(f, Fx, Fy, O.rates(s, s, s, s, s, s))
        b = O.bgk_node(f, Fx, Fy, s)
        p, q = Fx * ux ** 3, Fy * uy ** 3
        extra = np.array([0, 0, 0, -3 * (p + q), -3 * (p - q), 0, 0, 0, -(p + q)])
        expect = -(1 - s / 2) * (Mi @ O.shift_matrix_inverse(ux, uy) @ extra)
        np.testing.assert_allclose(a - b, expect, rtol=0, atol=1e-15)


def test_force_term_is_guo_plus_high_order(rng):
    """Remark 3: R_i = R_Gi + O(F u^2)."""
    Fx, Fy = 1e-3, -2e-3
    d = rng.uniform(-1, 1, 2)
    d /= np.linalg.norm(d)
    prev = None
    for scale in [0.08, 0.04, 0.02, 0.01]:
        ux, uy = scale * d
        diff = np.abs(O.force_term(1.0, ux, uy, Fx, Fy) - O.guo_term(ux, uy, Fx, Fy)).max()
        if prev is not None:
            assert 3.5 < prev / diff < 4.5  # halves u -> quarter difference
        prev = diff
    assert np.allclose(O.force_term(1.0, 0, 0, Fx, Fy), O.guo_term(0, 0, Fx, Fy), atol=1e-18)


def test_printed_c_order_changes_the_result(rng):
    """The two readings of Eq. 14 differ whenever Fx != Fy and s3 != 2."""
    f = _random_state(rng)
    S = O.rates(1, 1, 1.2, 1.5, 1.1, 1)
    a = O.collide_node(f, 1e-3, -1e-3, S, c_mode=O.C_DERIVED)
    b = O.collide_node(f, 1e-3, -1e-3, S, c_mode=O.C_PRINTED)
    assert np.abs(a - b).max() > 1e-5
    S2 = O.rates(1, 1, 1.2, 1.5, 2.0, 1)   # Remark 6: s3 = 2 removes the term
    a = O.collide_node(f, 1e-3, -1e-3, S2, c_mode=O.C_DERIVED)
    b = O.collide_node(f, 1e-3, -1e-3, S2, c_mode=O.C_PRINTED)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-16)
