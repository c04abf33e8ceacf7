"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle's
callers.

This module holds none of the method's arithmetic: no moments, equilibria,
collision or streaming.  It only builds input fields -- density noise,
velocity fields, body-force fields and solid masks -- for the canonical
problems of Sec. 4 of Fei & Luo (arXiv:1705.11092) and the large synthetic
lattices shaped like them.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), a counter-based generator:
value k of stream ``seed`` is mix(seed + (k + 1) * 0x9E3779B97F4A7C15).  Noise
fields are consumed in node order y * nx + x.
"""
from __future__ import annotations

import math

import numpy as np

DEFAULT_SEED = 1705

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# D2Q9 rest-state populations at unit density (the lattice weights,
# velocities ordered as in Eq. 1): used only to build random test states.
REST_WEIGHTS = np.array([4 / 9, 1 / 9, 1 / 9, 1 / 9, 1 / 9,
                         1 / 36, 1 / 36, 1 / 36, 1 / 36], dtype=np.float64)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Values offset..offset+n-1 of the SplitMix64 stream ``seed`` (uint64)."""
    with np.errstate(over="ignore"):
        k = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed) + k * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int, lo: float = -1.0, hi: float = 1.0, offset: int = 0) -> np.ndarray:
    """n doubles uniform in [lo, hi): the top 53 bits of each draw."""
    z = splitmix64(seed, n, offset)
    u01 = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return lo + (hi - lo) * u01


def density_noise(nx: int, ny: int, amp: float, seed: int = DEFAULT_SEED, rho0: float = 1.0):
    """rho = rho0 + amp * U(-1, 1), drawn in node order y * nx + x."""
    return (rho0 + amp * uniform(seed, nx * ny)).reshape(ny, nx)


def random_populations(nx: int, ny: int, amp: float = 0.05, seed: int = DEFAULT_SEED):
    """A random pre-collision state f[9][ny][nx] = w_i (1 + amp U(-1,1)).

    Mean velocity is O(amp/10); used by the parity tests as a generic
    non-equilibrium state.
    """
    r = uniform(seed, 9 * nx * ny).reshape(9, ny, nx)
    return REST_WEIGHTS[:, None, None] * (1.0 + amp * r)


def taylor_green_velocity(nx: int, ny: int, u0: float):
    """u = u0 [sin(phi_x x) sin(phi_y y), cos(phi_x x) cos(phi_y y)], phi = 2 pi/n.

    The steady Taylor-Green (four-roll mill) field of Sec. 4B on an nx-by-ny
    periodic lattice with nodes at integer coordinates.
    """
    x = np.arange(nx, dtype=np.float64)
    y = np.arange(ny, dtype=np.float64)
    px, py = 2 * math.pi / nx, 2 * math.pi / ny
    X, Y = np.meshgrid(x, y)
    return u0 * np.sin(px * X) * np.sin(py * Y), u0 * np.cos(px * X) * np.cos(py * Y)


def sinusoidal_force_rows(ny: int, F0: float, k: int = 1):
    """Per-row force [ny][2]: F = F0 sin(2 pi k y / ny) e_x."""
    y = np.arange(ny, dtype=np.float64)
    out = np.zeros((ny, 2))
    out[:, 0] = F0 * np.sin(2 * math.pi * k * y / ny)
    return out


def sinusoidal_force_columns(nx: int, F0: float, k: int = 1):
    """Per-column force [nx][2]: F = F0 sin(2 pi k x / nx) e_y (the first
    force turned by 90 degrees)."""
    x = np.arange(nx, dtype=np.float64)
    out = np.zeros((nx, 2))
    out[:, 1] = F0 * np.sin(2 * math.pi * k * x / nx)
    return out


def modulated_force_rows(ny: int, F0: float, a: float = 0.1):
    """Per-row force [ny][2]: Fx = F0 (1 + a sin(2 pi y / ny)), Fy = 0."""
    y = np.arange(ny, dtype=np.float64)
    out = np.zeros((ny, 2))
    out[:, 0] = F0 * (1.0 + a * np.sin(2 * math.pi * y / ny))
    return out


def channel_mask(nx: int, ny: int):
    """Periodic channel: row 0 solid, fluid rows 1..ny-1.  Row 0 is both
    walls; with halfway bounce-back they sit at y = 1/2 and y = ny - 1/2, so
    the channel width is H = ny - 1."""
    m = np.zeros((ny, nx), np.uint8)
    m[0, :] = 1
    return m


def obstacle_mask(nx: int, ny: int, size: int = 32, pitch: int = 64):
    """Periodic array of size-by-size solid squares on a pitch-by-pitch grid
    (25 % solid for size 32, pitch 64)."""
    x = np.arange(nx) % pitch
    y = np.arange(ny) % pitch
    return ((y[:, None] < size) & (x[None, :] < size)).astype(np.uint8)


CHANNEL_SWEEP_HEIGHTS = (17, 33, 65, 129, 257, 513)


def channel_sweep(count: int = 256, seed: int = DEFAULT_SEED, heights=CHANNEL_SWEEP_HEIGHTS):
    """Parameters of a batched resolution/parameter sweep of force-driven
    channels: ladders of the given ny values (nx = 2 ny), each ladder sharing
    one draw of tau ~ U[0.55, 1.5] and Fx ~ log-U[1e-7, 1e-5]; when `count`
    is not a multiple of the ladder length the remainder are single channels
    with a random height.  Returns a list of dicts (nx, ny, tau, fx, ladder).
    """
    per = len(heights)
    ladders = count // per
    u = uniform(seed, 2 * (ladders + count), 0.0, 1.0)
    out = []
    for k in range(ladders):
        tau = 0.55 + 0.95 * u[2 * k]
        fx = 10.0 ** (-7.0 + 2.0 * u[2 * k + 1])
        for ny in heights:
            out.append({"nx": 2 * ny, "ny": ny, "tau": tau, "fx": fx, "ladder": k})
    j = 2 * ladders
    while len(out) < count:
        ny = heights[int(u[j] * per) % per]
        tau = 0.55 + 0.95 * u[j + 1]
        fx = 10.0 ** (-7.0 + 2.0 * u[j + 2])
        out.append({"nx": 2 * ny, "ny": ny, "tau": tau, "fx": fx, "ladder": -1})
        j += 3
    return out
