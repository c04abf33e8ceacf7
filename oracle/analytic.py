"""Closed-form solutions and error norms used to pin the oracle.

TEST INFRASTRUCTURE (part of the oracle package; see ``oracle/__init__.py``).

Paper: Fei & Luo, arXiv:1705.11092.
  - Sec. 4A, Eq. 23: steady force-driven Poiseuille flow.  The printed form
    u = Fx/(2 nu)(1 - y^2/L^2) lacks a factor L^2; with the walls at y = 0 and
    y = H (H = 2L) the steady profile is u(y) = F y (H - y) / (2 rho nu).
  - Remark 4: the non-slip rule s3 = (16 - 8 s2)/(8 - s2), which is
    Lambda = (1/s2 - 1/2)(1/s3 - 1/2) = 3/16.
  - Eq. 24: the residual E_R and the relative L2 error E_2.
  - Sec. 4B: the steady Taylor-Green (four-roll mill) flow and its force.
"""
from __future__ import annotations

import math

import numpy as np


def viscosity(s2: float) -> float:
    """Kinematic viscosity from the shear rate, s2 = 1/(3 nu + 1/2) (Eq. 7)."""
    return (1.0 / s2 - 0.5) / 3.0


def shear_rate(nu: float) -> float:
    return 1.0 / (3.0 * nu + 0.5)


def nonslip_s3(s2: float) -> float:
    """Remark 4: s3 giving zero slip with halfway bounce-back."""
    return (16.0 - 8.0 * s2) / (8.0 - s2)


def magic_lambda(s2: float, s3: float) -> float:
    """Lambda = (1/s2 - 1/2)(1/s3 - 1/2); the non-slip rule is Lambda = 3/16."""
    return (1.0 / s2 - 0.5) * (1.0 / s3 - 0.5)


def poiseuille_steady(y, H, F, nu, rho=1.0):
    """Steady channel profile with walls at y = 0 and y = H (Eq. 23 with L^2)."""
    y = np.asarray(y, dtype=np.float64)
    return F * y * (H - y) / (2.0 * rho * nu)


def poiseuille_startup(y, t, H, F, nu, rho=1.0, nterms=2001):
    """Start-up flow from rest: u_t = nu u_yy + F/rho, u(0) = u(H) = 0.

    u(y, t) = steady - sum_{n odd} 4 F H^2 / (rho nu pi^3 n^3)
                        sin(n pi y / H) exp(-n^2 pi^2 nu t / H^2).
    """
    y = np.asarray(y, dtype=np.float64)
    u = poiseuille_steady(y, H, F, nu, rho)
    for n in range(1, nterms + 1, 2):
        b = 4.0 * F * H * H / (rho * nu * math.pi ** 3 * n ** 3)
        decay = math.exp(-(n * math.pi / H) ** 2 * nu * t)
        if decay == 0.0:
            break
        u = u - b * np.sin(n * math.pi * y / H) * decay
    return u


def bounce_back_slip(F, s2, s3, rho=1.0):
    """Slip velocity of halfway bounce-back in steady Poiseuille flow for a
    two-relaxation-rate scheme: F (16 Lambda - 3) / (24 rho nu).

    Closed form from the two-relaxation-time literature (Ginzburg and
    d'Humieres); it vanishes at Lambda = 3/16, the paper's non-slip rule.
    """
    nu = viscosity(s2)
    return F * (16.0 * magic_lambda(s2, s3) - 3.0) / (24.0 * rho * nu)


def taylor_green(nx, ny, u0, phi, offset=0.0):
    """Steady Taylor-Green velocity (Sec. 4B) at nodes x = i + offset."""
    x = np.arange(nx, dtype=np.float64) + offset
    y = np.arange(ny, dtype=np.float64) + offset
    X, Y = np.meshgrid(x, y)
    ux = u0 * np.sin(phi * X) * np.sin(phi * Y)
    uy = u0 * np.cos(phi * X) * np.cos(phi * Y)
    return ux, uy


def taylor_green_force(nx, ny, u0, phi, nu, rho=1.0, offset=0.0):
    """Body force that holds the Taylor-Green field steady.

    The viscous balance needs F = -rho nu lap(u) = 2 rho nu phi^2 u_a, i.e.
    components [sin sin, cos cos]; the printed force of Sec. 4B lists
    [cos cos, sin sin], which does not balance the printed u_a.
    """
    ux, uy = taylor_green(nx, ny, u0, phi, offset)
    k = 2.0 * rho * nu * phi * phi
    return k * ux, k * uy


def e2(ux, uy, ux_a, uy_a, fluid=None) -> float:
    """Eq. 24: relative L2 error over the fluid nodes (both components)."""
    ux, uy, ux_a, uy_a = (np.asarray(a, dtype=np.float64) for a in (ux, uy, ux_a, uy_a))
    if fluid is not None:
        fluid = np.asarray(fluid, dtype=bool)
        ux, uy, ux_a, uy_a = ux[fluid], uy[fluid], ux_a[fluid], uy_a[fluid]
    num = np.sum((ux - ux_a) ** 2 + (uy - uy_a) ** 2)
    den = np.sum(ux_a ** 2 + uy_a ** 2)
    return math.sqrt(num / den)


def e_r(ux_new, uy_new, ux_old, uy_old) -> float:
    """Eq. 24: relative change of the velocity field over an interval."""
    num = np.sum((ux_new - ux_old) ** 2 + (uy_new - uy_old) ** 2)
    den = np.sum(ux_new ** 2 + uy_new ** 2)
    return math.sqrt(num / den) if den > 0 else math.sqrt(num)


def convergence_rate(n, err) -> float:
    """Least-squares slope of log(E2) against log(1/N) (Table 2's CR)."""
    x = np.log(np.asarray(n, dtype=np.float64))
    y = np.log(np.asarray(err, dtype=np.float64))
    slope = np.polyfit(x, y, 1)[0]
    return -float(slope)
