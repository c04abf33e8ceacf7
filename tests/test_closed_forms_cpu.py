"""The library's closed-form reference flows (paper_1705_11092_gb300/
closed_forms.py) against the oracle's independently written ones and
against their limits: the start-up series at t = 0 and t -> infinity, the
non-slip rule of Remark 4 (Fei & Luo, arXiv:1705.11092), and a known order."""
import math

import numpy as np
import pytest

from oracle import analytic as A
from paper_1705_11092_gb300 import closed_forms as C


def test_steady_profile_matches_the_oracle_closed_form():
    H, F, nu = 32.0, 1e-6, 0.1
    y = np.arange(33) - 0.5
    np.testing.assert_allclose(C.channel_steady(y, H, F, nu), A.poiseuille_steady(y, H, F, nu),
                               rtol=1e-14, atol=0)


def test_startup_series_limits():
    H, F, nu = 32.0, 1e-6, 0.1
    y = np.arange(1, 32) - 0.5
    steady = C.channel_steady(y, H, F, nu)
    assert np.abs(C.channel_startup(y, H, F, nu, 0.0)).max() < 2e-3 * steady.max()
    np.testing.assert_allclose(C.channel_startup(y, H, F, nu, 1e6), steady, rtol=1e-12)
    # the leading transient decays as exp(-pi^2 nu t / H^2)
    t = 2000.0
    d = steady - C.channel_startup(y, H, F, nu, t)
    lead = 4 * F * H * H / (nu * math.pi ** 3) * math.exp(-(math.pi / H) ** 2 * nu * t)
    assert d.max() == pytest.approx(lead * np.sin(math.pi * y / H).max(), rel=1e-3)


def test_startup_series_solves_the_diffusion_equation():
    """du/dt = nu u'' + F at interior points (finite differences)."""
    H, F, nu, t = 40.0, 1e-5, 0.2, 300.0
    y = np.linspace(2.0, 38.0, 19)
    h, dt = 1e-2, 1e-2
    ut = (C.channel_startup(y, H, F, nu, t + dt) - C.channel_startup(y, H, F, nu, t - dt)) / (2 * dt)
    uyy = (C.channel_startup(y + h, H, F, nu, t) - 2 * C.channel_startup(y, H, F, nu, t)
           + C.channel_startup(y - h, H, F, nu, t)) / h ** 2
    np.testing.assert_allclose(ut, nu * uyy + F, rtol=1e-4, atol=1e-12)


def test_slip_vanishes_on_the_non_slip_rule_and_matches_the_oracle():
    s2 = 1.754
    s3 = A.nonslip_s3(s2)
    assert abs(C.halfway_slip(1e-6, C.viscosity(s2), s2, s3)) < 1e-20
    for s3 in (0.8, 1.0, 1.6):
        assert C.halfway_slip(1e-6, C.viscosity(s2), s2, s3) == pytest.approx(
            A.bounce_back_slip(1e-6, s2, s3), rel=1e-14)


def test_fitted_order():
    h = np.array([16, 32, 64, 128])
    assert C.fitted_order(h, 3.0 * h ** -2.0) == pytest.approx(2.0, abs=1e-12)
