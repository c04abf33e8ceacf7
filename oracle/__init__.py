"""Plain FP64 CPU oracle for the D2Q9 cascaded LBM with consistent forcing.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA path (``paper_1705_11092_gb300``) and neither imports the other.

The arithmetic lives in ``clbm_oracle.c`` (plain C, FP64, built by
``oracle/build.py``); this module only marshals numpy arrays into it.  The
closed-form solutions used by the pins are in ``oracle/analytic.py``.

Paper: L. Fei and K. H. Luo, "Consistent forcing scheme in the cascaded
lattice Boltzmann method", arXiv:1705.11092.  Section, equation and remark
numbers below refer to it.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

# collision modes (see clbm_oracle.c)
MODE_DEFINITION = 0  # Eq. 2-4 definitions, LU back-transform
MODE_PRINTED = 1     # printed M (Eq. 5), N (Eq. 6), M^-1, N^-1 (Appendix)
MODE_RAW_MRT = 2     # N = I (Remark 2)

# readings of the forcing central moments C (Eq. 14)
C_DERIVED = 0  # [0,Fx,Fy,0,0,0,Fy/3,Fx/3,0] -- from Eq. 13 (default)
C_PRINTED = 1  # [0,Fx,Fy,0,0,0,Fx/3,Fy/3,0] -- literal print of Eq. 14
C_EXACT = 2    # N M R computed by definition from Eq. 13
# comparison forcing schemes of Sec. 3 (passed as c_mode)
FORCING_M1 = 3  # Premnath et al., Eq. 17-19
FORCING_M2 = 4  # Lycett-Brown and Luo, Eq. 21

EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])  # Eq. 1
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])

_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_U8 = ctypes.POINTER(ctypes.c_uint8)


def _load():
    global _lib
    if _lib is not None:
        return _lib
    path = _build.library_path()
    if not os.path.exists(path):
        _build.build()
    lib = ctypes.CDLL(path)
    d, i = ctypes.c_double, ctypes.c_int
    sig = {
        "oracle_central_moments": (None, [_D, d, d, _D]),
        "oracle_equilibrium": (None, [d, d, d, _D]),
        "oracle_force_term": (None, [d, d, d, d, d, _D]),
        "oracle_guo_term": (None, [d, d, d, d, _D]),
        "oracle_macroscopic": (None, [_D, d, d, _D, _D, _D]),
        "oracle_shift_matrix": (None, [d, d, _D]),
        "oracle_shift_matrix_inverse": (None, [d, d, _D]),
        "oracle_transform_matrix": (None, [_D]),
        "oracle_transform_matrix_inverse": (None, [_D]),
        "oracle_definition_matrix": (None, [d, d, _D]),
        "oracle_collide_node": (i, [_D, d, d, _D, i, i, _D]),
        "oracle_mrt_guo_node": (None, [_D, d, d, _D, _D]),
        "oracle_bgk_node": (None, [_D, d, d, d, i, _D]),
        "oracle_collide_lattice": (i, [i, i, _D, _D, _D, _U8, i, i, _D, _D]),
        "oracle_stream": (None, [i, i, _U8, _D, _D]),
        "oracle_run": (i, [i, i, _D, _D, _D, _U8, i, i, _D, i]),
        "oracle_moments": (None, [i, i, _D, _D, _U8, _D, _D, _D, _D]),
        "oracle_equilibrium_lattice": (None, [i, i, _U8, _D, _D, _D, _D]),
        "oracle_has_openmp": (i, []),
        "oracle_sc_psi": (d, [d, d, d]),
        "oracle_sc_pressure": (d, [d, d, d, d]),
        "oracle_sc_force": (None, [i, i, _D, d, d, d, _D, _D]),
        "oracle_density": (None, [i, i, _D, _D]),
        "oracle_run_sc": (i, [i, i, _D, d, d, d, i, i, _D, i]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _f64(a, shape=None) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def rates(s0=1.0, s1=1.0, sb=1.0, s2=1.0, s3=1.0, s4=1.0) -> np.ndarray:
    """Diagonal of S in Eq. 7: (s0, s1, s1, sb, s2, s2, s3, s3, s4)."""
    return np.array([s0, s1, s1, sb, s2, s2, s3, s3, s4], dtype=np.float64)


def has_openmp() -> bool:
    return bool(_load().oracle_has_openmp())


# ---- per-node functions --------------------------------------------------

def central_moments(f, ux, uy) -> np.ndarray:
    """Recombined central moments T~ of Eq. 2-3 about (ux, uy)."""
    f = _f64(f, (9,))
    out = np.zeros(9)
    _load().oracle_central_moments(_dp(f), ux, uy, _dp(out))
    return out


def equilibrium(rho, ux, uy) -> np.ndarray:
    """Product-form generalized equilibrium (central moments = Eq. 8)."""
    out = np.zeros(9)
    _load().oracle_equilibrium(rho, ux, uy, _dp(out))
    return out


def force_term(rho, ux, uy, Fx, Fy) -> np.ndarray:
    """R_i of Eq. 13."""
    out = np.zeros(9)
    _load().oracle_force_term(rho, ux, uy, Fx, Fy, _dp(out))
    return out


def guo_term(ux, uy, Fx, Fy) -> np.ndarray:
    """Guo's R_Gi (Remark 3)."""
    out = np.zeros(9)
    _load().oracle_guo_term(ux, uy, Fx, Fy, _dp(out))
    return out


def macroscopic(f, Fx, Fy):
    """(rho, ux, uy) of Eq. 11 and Eq. 15."""
    f = _f64(f, (9,))
    r, x, y = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _load().oracle_macroscopic(_dp(f), Fx, Fy, ctypes.byref(r), ctypes.byref(x), ctypes.byref(y))
    return r.value, x.value, y.value


def _mat(fn, *args) -> np.ndarray:
    out = np.zeros((9, 9))
    fn(*args, _dp(out))
    return out


def shift_matrix(ux, uy) -> np.ndarray:
    """N(u) as printed in Eq. 6."""
    return _mat(_load().oracle_shift_matrix, ux, uy)


def shift_matrix_inverse(ux, uy) -> np.ndarray:
    """N^-1(u) as printed in the Appendix."""
    return _mat(_load().oracle_shift_matrix_inverse, ux, uy)


def transform_matrix() -> np.ndarray:
    """M as printed in Eq. 5."""
    return _mat(_load().oracle_transform_matrix)


def transform_matrix_inverse() -> np.ndarray:
    """M^-1 as printed in the Appendix."""
    return _mat(_load().oracle_transform_matrix_inverse)


def definition_matrix(ux, uy) -> np.ndarray:
    """K(u) = N(u) M built from the definitions of Eq. 2-4."""
    return _mat(_load().oracle_definition_matrix, ux, uy)


def collide_node(f, Fx, Fy, s, mode=MODE_DEFINITION, c_mode=C_DERIVED) -> np.ndarray:
    """One collision with consistent forcing (Eq. 12) at one node."""
    f = _f64(f, (9,))
    s = _f64(s, (9,))
    out = np.zeros(9)
    rc = _load().oracle_collide_node(_dp(f), Fx, Fy, _dp(s), mode, c_mode, _dp(out))
    if rc != 0:
        raise FloatingPointError("singular back-transform")
    return out


def mrt_guo_node(f, Fx, Fy, s) -> np.ndarray:
    """Population-space MRT step with N = I and force term M R (Remark 2)."""
    f = _f64(f, (9,))
    s = _f64(s, (9,))
    out = np.zeros(9)
    _load().oracle_mrt_guo_node(_dp(f), Fx, Fy, _dp(s), _dp(out))
    return out


def bgk_node(f, Fx, Fy, s, guo=False) -> np.ndarray:
    """BGK step with R_i of Eq. 13 (guo=False) or Guo's R_Gi (guo=True)."""
    f = _f64(f, (9,))
    out = np.zeros(9)
    _load().oracle_bgk_node(_dp(f), Fx, Fy, float(s), int(bool(guo)), _dp(out))
    return out


# ---- Shan-Chen pseudopotential (Sec. 4C) ---------------------------------

def sc_psi(rho, psi0=1.0, rho0=1.0) -> float:
    """psi(rho) = psi0 exp(-rho0 / rho)."""
    return _load().oracle_sc_psi(float(rho), psi0, rho0)


def sc_pressure(rho, G, psi0=1.0, rho0=1.0) -> float:
    """p = rho cs^2 + G psi^2 / 2."""
    return _load().oracle_sc_pressure(float(rho), G, psi0, rho0)


def sc_force(rho, G, psi0=1.0, rho0=1.0):
    """Interaction force (Fx, Fy) of a periodic density field rho[ny][nx]."""
    rho = _f64(rho)
    ny, nx = rho.shape
    fx = np.zeros_like(rho)
    fy = np.zeros_like(rho)
    _load().oracle_sc_force(nx, ny, _dp(rho), G, psi0, rho0, _dp(fx), _dp(fy))
    return fx, fy


# ---- lattice functions ---------------------------------------------------

class Lattice:
    """An nx-by-ny periodic lattice with an optional solid mask and a
    per-node force field, for the oracle's lattice drivers.

    ``fx``/``fy`` may be scalars or arrays broadcastable to (ny, nx).
    """

    def __init__(self, nx, ny, s, fx=0.0, fy=0.0, solid=None,
                 mode=MODE_DEFINITION, c_mode=C_DERIVED):
        self.nx, self.ny = int(nx), int(ny)
        self.s = _f64(s, (9,))
        shape = (self.ny, self.nx)
        self.fx = np.ascontiguousarray(np.broadcast_to(np.asarray(fx, np.float64), shape))
        self.fy = np.ascontiguousarray(np.broadcast_to(np.asarray(fy, np.float64), shape))
        if solid is None:
            self.solid = np.zeros(shape, np.uint8)
        else:
            self.solid = np.ascontiguousarray(np.asarray(solid).astype(np.uint8).reshape(shape))
        self.mode = mode
        self.c_mode = c_mode

    def _u8(self):
        return self.solid.ctypes.data_as(_U8)

    def equilibrium(self, rho, ux, uy) -> np.ndarray:
        shape = (self.ny, self.nx)
        rho = np.ascontiguousarray(np.broadcast_to(np.asarray(rho, np.float64), shape))
        ux = np.ascontiguousarray(np.broadcast_to(np.asarray(ux, np.float64), shape))
        uy = np.ascontiguousarray(np.broadcast_to(np.asarray(uy, np.float64), shape))
        f = np.zeros((9, self.ny, self.nx))
        _load().oracle_equilibrium_lattice(self.nx, self.ny, self._u8(), _dp(rho), _dp(ux),
                                           _dp(uy), _dp(f))
        return f

    def collide(self, f) -> np.ndarray:
        """Post-collision state of a pre-collision state (solid nodes zero)."""
        f = _f64(f, (9, self.ny, self.nx))
        out = np.zeros_like(f)
        rc = _load().oracle_collide_lattice(self.nx, self.ny, _dp(self.s), _dp(self.fx),
                                            _dp(self.fy), self._u8(), self.mode, self.c_mode,
                                            _dp(f), _dp(out))
        if rc != 0:
            raise FloatingPointError("singular back-transform")
        return out

    def stream(self, f_post) -> np.ndarray:
        """Eq. 10 with halfway bounce-back."""
        f_post = _f64(f_post, (9, self.ny, self.nx))
        out = np.zeros_like(f_post)
        _load().oracle_stream(self.nx, self.ny, self._u8(), _dp(f_post), _dp(out))
        return out

    def run(self, f, nsteps) -> np.ndarray:
        """nsteps time steps (collide, stream) from the pre-collision state f."""
        f = _f64(f, (9, self.ny, self.nx)).copy()
        rc = _load().oracle_run(self.nx, self.ny, _dp(self.s), _dp(self.fx), _dp(self.fy),
                                self._u8(), self.mode, self.c_mode, _dp(f), int(nsteps))
        if rc != 0:
            raise FloatingPointError("oracle run failed (%d)" % rc)
        return f

    def run_sc(self, f, nsteps, G, psi0=1.0, rho0=1.0) -> np.ndarray:
        """nsteps Shan-Chen steps: the force is recomputed from the density
        of the pre-collision state before every collision (no solid nodes;
        the lattice's own force arrays are not used)."""
        if self.solid.any():
            raise ValueError("Shan-Chen runs take no solid nodes")
        f = _f64(f, (9, self.ny, self.nx)).copy()
        rc = _load().oracle_run_sc(self.nx, self.ny, _dp(self.s), G, psi0, rho0, self.mode,
                                   self.c_mode, _dp(f), int(nsteps))
        if rc != 0:
            raise FloatingPointError("oracle run failed (%d)" % rc)
        return f

    def moments_sc(self, f, G, psi0=1.0, rho0=1.0):
        """(rho, ux, uy) of a pre-collision state of a Shan-Chen run: Eq. 11
        and Eq. 15 with the force of that state's density."""
        f = _f64(f, (9, self.ny, self.nx))
        rho = f.sum(axis=0)
        fx, fy = sc_force(rho, G, psi0, rho0)
        rho = np.zeros((self.ny, self.nx))
        ux = np.zeros_like(rho)
        uy = np.zeros_like(rho)
        _load().oracle_moments(self.nx, self.ny, _dp(fx), _dp(fy), self._u8(),
                               _dp(f), _dp(rho), _dp(ux), _dp(uy))
        return rho, ux, uy

    def moments(self, f):
        """(rho, ux, uy) fields of a pre-collision state, Eq. 11 and Eq. 15."""
        f = _f64(f, (9, self.ny, self.nx))
        rho = np.zeros((self.ny, self.nx))
        ux = np.zeros_like(rho)
        uy = np.zeros_like(rho)
        _load().oracle_moments(self.nx, self.ny, _dp(self.fx), _dp(self.fy), self._u8(),
                               _dp(f), _dp(rho), _dp(ux), _dp(uy))
        return rho, ux, uy
