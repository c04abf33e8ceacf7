"""Pins of the oracle's start-up series (``oracle.analytic.poiseuille_startup``)
against what the mathematics fixes, without the package's own closed forms.

Sec. 4A of Fei & Luo (arXiv:1705.11092) drives a channel with a uniform body
force; a channel started from rest follows u_t = nu u_yy + F / rho with
u(0, t) = u(H, t) = 0 and u(y, 0) = 0.  The series must therefore

* vanish at t = 0 (the sine series of the parabola sums to the parabola; at
  the centre this is the identity sum_k (-1)^k / (2k+1)^3 = pi^3 / 32, which
  fixes the coefficient 4 / pi^3 and the power n^3),
* grow as F t / rho in the bulk at early times (the force alone acts there),
* reach the steady parabola as t -> infinity (sign of the decay exponent),
* satisfy the diffusion equation with the force at interior points (the
  decay rate n^2 pi^2 nu / H^2 of every mode), and
* vanish at both walls for every t.
"""
import math

import numpy as np
import pytest

from oracle import analytic as A

H, F, NU = 32.0, 1e-6, 0.1


def test_startup_vanishes_at_t0_by_the_centre_identity():
    # centre: steady F H^2 / (8 nu); the series' t = 0 sum there is
    # (4 F H^2 / (nu pi^3)) sum_k (-1)^k / (2k+1)^3 = F H^2 / (8 nu)
    centre = A.poiseuille_startup(np.array([H / 2]), 0.0, H, F, NU)[0]
    steady = F * H * H / (8.0 * NU)
    # the series is truncated after n = 2001: the remainder is below
    # 4 F H^2 / (nu pi^3) * 1 / (2 * 2001^2)
    bound = 4 * F * H * H / (NU * math.pi ** 3) / (2 * 2001 ** 2)
    assert abs(centre) <= bound
    assert abs(centre) < 1e-6 * steady


def test_startup_vanishes_everywhere_at_t0():
    y = np.linspace(0.5, H - 0.5, 64)
    u0 = A.poiseuille_startup(y, 0.0, H, F, NU)
    steady = A.poiseuille_steady(y, H, F, NU)
    assert np.abs(u0).max() < 1e-5 * steady.max()


def test_startup_grows_with_the_force_alone_in_the_bulk():
    # before the walls are felt (nu t << (H/2)^2) the centre moves as F t
    for t in (1.0, 5.0, 20.0):
        centre = A.poiseuille_startup(np.array([H / 2]), t, H, F, NU)[0]
        assert centre == pytest.approx(F * t, rel=1e-5)


def test_startup_reaches_the_steady_parabola():
    y = np.linspace(0.5, H - 0.5, 33)
    t = 60.0 * H * H / NU
    np.testing.assert_allclose(A.poiseuille_startup(y, t, H, F, NU),
                               F * y * (H - y) / (2 * NU), rtol=1e-12)


def test_startup_solves_the_forced_diffusion_equation():
    y = np.linspace(3.0, H - 3.0, 14)
    h, dt = 1e-2, 1e-2
    for t in (50.0, 400.0, 3000.0):
        u = lambda yy, tt: A.poiseuille_startup(yy, tt, H, F, NU)
        ut = (u(y, t + dt) - u(y, t - dt)) / (2 * dt)
        uyy = (u(y + h, t) - 2 * u(y, t) + u(y - h, t)) / h ** 2
        np.testing.assert_allclose(ut, NU * uyy + F, rtol=2e-4, atol=1e-14)


def test_startup_vanishes_at_the_walls():
    for t in (0.0, 10.0, 1e3, 1e5):
        w = A.poiseuille_startup(np.array([0.0, H]), t, H, F, NU)
        assert np.abs(w).max() < 1e-12 * F * H * H / NU


def test_slowest_mode_decays_at_the_diffusion_rate():
    # late enough that only n = 1 is left: (steady - u) / sin(pi y / H)
    # decays by exp(-pi^2 nu dt / H^2) over dt
    y = np.array([H / 4, H / 2])
    t0, dt = 2000.0, 1000.0
    d0 = A.poiseuille_steady(y, H, F, NU) - A.poiseuille_startup(y, t0, H, F, NU)
    d1 = A.poiseuille_steady(y, H, F, NU) - A.poiseuille_startup(y, t0 + dt, H, F, NU)
    np.testing.assert_allclose(d1 / d0, math.exp(-(math.pi / H) ** 2 * NU * dt), rtol=1e-6)
