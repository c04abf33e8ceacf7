"""Closed-form reference flows for the library's error diagnostics.

The library reports E_2 errors (Eq. 24 of Fei & Luo, arXiv:1705.11092)
through ``clbm_l2_error`` / ``clbm_batch_l2_error``; these functions give the
fields to compare with, for the force-driven channel of Sec. 4A with walls at
y = 0 and y = H (halfway bounce-back: the wall lies half-way between the last
fluid node and the first solid one, so a fluid row j sits at y = j - 1/2
when row 0 is the solid row).  All quantities are in lattice units.
"""
from __future__ import annotations

import math

import numpy as np


def viscosity(s2: float) -> float:
    """Kinematic viscosity of the shear rate s2: nu = (1/s2 - 1/2) / 3."""
    return (1.0 / s2 - 0.5) / 3.0


def channel_steady(y, H: float, F: float, nu: float, rho: float = 1.0):
    """Steady plane Poiseuille profile u(y) = F y (H - y) / (2 rho nu)."""
    y = np.asarray(y, dtype=np.float64)
    return F * y * (H - y) / (2.0 * rho * nu)


def channel_startup(y, H: float, F: float, nu: float, t: float, rho: float = 1.0,
                    rel_tol: float = 1e-16):
    """Profile of the channel started from rest at t = 0 with a constant
    body force: the steady profile minus the decaying odd sine modes,
    u(y, t) = u_s(y) - sum_{n odd} 4 F H^2 / (rho nu pi^3 n^3)
                       sin(n pi y / H) exp(-n^2 pi^2 nu t / H^2),
    summed until a term falls below rel_tol of the first."""
    y = np.asarray(y, dtype=np.float64)
    u = channel_steady(y, H, F, nu, rho)
    a1 = 4.0 * F * H * H / (rho * nu * math.pi ** 3)
    n = 1
    while True:
        amp = a1 / n ** 3 * math.exp(-(n * math.pi / H) ** 2 * nu * t)
        if amp <= rel_tol * a1:
            break
        u = u - amp * np.sin(n * math.pi * y / H)
        n += 2
    return u


def halfway_slip(F: float, nu: float, s2: float, s3: float, rho: float = 1.0) -> float:
    """Wall slip of the steady channel with halfway bounce-back under a
    two-rate collision (shear rate s2, third-order rate s3):
    F (16 Lambda - 3) / (24 rho nu), Lambda = (1/s2 - 1/2)(1/s3 - 1/2).
    It vanishes on the non-slip rule Lambda = 3/16 (Remark 4)."""
    lam = (1.0 / s2 - 0.5) * (1.0 / s3 - 0.5)
    return F * (16.0 * lam - 3.0) / (24.0 * rho * nu)


def fitted_order(h, err) -> float:
    """Convergence order p of err ~ h^-p over resolutions h (nodes across):
    minus the least-squares slope of log(err) against log(h)."""
    x = np.log(np.asarray(h, dtype=np.float64))
    y = np.log(np.asarray(err, dtype=np.float64))
    return -float(np.polyfit(x, y, 1)[0])
