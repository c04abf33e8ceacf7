"""Thin ctypes binding of the C ABI in ``include/clbm.h``.

Every function here has the name of the C entry point it calls and does
argument marshalling only: numpy arrays (host) or torch CUDA tensors (device)
become pointers, the torch stream becomes a ``cudaStream_t``.  All
arithmetic of the time step runs in the CUDA library.  If the library is
missing this module raises; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

CLBM_FP64, CLBM_FP32, CLBM_FP16, CLBM_BF16 = 0, 1, 2, 3
FORMATS = {"fp64": CLBM_FP64, "fp32": CLBM_FP32, "fp16": CLBM_FP16, "bf16": CLBM_BF16}
CLBM_FORCE_UNIFORM, CLBM_FORCE_ROWS, CLBM_FORCE_COLUMNS, CLBM_FORCE_FIELD = 0, 1, 2, 3
CLBM_FORCE_SHAN_CHEN = 4
CLBM_FORCING_CONSISTENT, CLBM_FORCING_M1, CLBM_FORCING_M2 = 0, 1, 2
CLBM_SCHEDULE_CONTIGUOUS, CLBM_SCHEDULE_INTERLEAVED = 0, 1
CLBM_SPARSE_OFF, CLBM_SPARSE_ON, CLBM_SPARSE_AUTO = 0, 1, 2
CLBM_ROUND_NEAREST, CLBM_ROUND_STOCHASTIC = 0, 1
CLBM_FAIL_NONE, CLBM_FAIL_ALLOC, CLBM_FAIL_LAUNCH = 0, 1, 2

CLBM_OK = 0
CLBM_ERR_ARG = -1
CLBM_ERR_OOM = -2
CLBM_ERR_CUDA = -3
CLBM_ERR_DIVERGED = -4
CLBM_ERR_TIMEOUT = -5
CLBM_ERR_STATE = -6

# every symbol the header declares, with (restype, argtypes)
_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_SIGNATURES = {
    "clbm_create": (_I, [ctypes.POINTER(_P), _I, _I, _P, _I, _P, _D, _D, _P, _I, _P]),
    "clbm_init": (_I, [_P, _P, _P, _P]),
    "clbm_init_dev": (_I, [_P, _P, _P, _P]),
    "clbm_set_populations": (_I, [_P, _P, _I]),
    "clbm_get_populations": (_I, [_P, _P, _I]),
    "clbm_get_window": (_I, [_P, _I, _I, _I, _I, _P]),
    "clbm_get_window_async": (_I, [_P, _I, _I, _I, _I, _P]),
    "clbm_step": (_I, [_P, _I]),
    "clbm_moments": (_I, [_P, _P, _P, _P]),
    "clbm_moments_dev": (_I, [_P, _P, _P, _P]),
    "clbm_reduce": (_I, [_P, _P]),
    "clbm_l2_error": (_I, [_P, _P, _P, _P]),
    "clbm_set_forcing_scheme": (_I, [_P, _I]),
    "clbm_synchronize": (_I, [_P]),
    "clbm_scale_exponent": (_I, [_P]),
    "clbm_set_scale_exponent": (_I, [_P, _I]),
    "clbm_set_tuning": (_I, [_P, _I, _I, _I, _I]),
    "clbm_set_sparse": (_I, [_P, _I]),
    "clbm_set_rounding": (_I, [_P, _I]),
    "clbm_sparse_tasks": (_I, [_P]),
    "clbm_get_tuning": (_I, [_P, _P, _P, _P, _P]),
    "clbm_bytes_per_update": (_D, [_P]),
    "clbm_fluid_nodes": (ctypes.c_longlong, [_P]),
    "clbm_get_size": (_I, [_P, _P, _P]),
    "clbm_debug_fail_next": (_I, [_I]),
    "clbm_batch_create": (_I, [ctypes.POINTER(_P), _I, _P, _I, _P]),
    "clbm_batch_init": (_I, [_P, _I, _P, _P, _P]),
    "clbm_batch_set_populations": (_I, [_P, _I, _P, _I]),
    "clbm_batch_get_populations": (_I, [_P, _I, _P, _I]),
    "clbm_batch_moments": (_I, [_P, _I, _P, _P, _P]),
    "clbm_batch_reduce": (_I, [_P, _I, _P]),
    "clbm_batch_l2_error": (_I, [_P, _I, _P, _P, _P]),
    "clbm_batch_step": (_I, [_P, _I]),
    "clbm_batch_set_tuning": (_I, [_P, _I, _I, _I, _I]),
    "clbm_batch_get_tuning": (_I, [_P, _P, _P, _P, _P]),
    "clbm_batch_autotune": (_I, [_P, _I, _P]),
    "clbm_batch_set_mode": (_I, [_P, _I, _I, _I]),
    "clbm_batch_get_mode": (_I, [_P, _P, _P, _P]),
    "clbm_batch_resident_lattices": (_I, [_P]),
    "clbm_batch_set_wait": (_I, [_P, ctypes.c_longlong, ctypes.c_longlong]),
    "clbm_batch_synchronize": (_I, [_P]),
    "clbm_batch_fluid_nodes": (ctypes.c_longlong, [_P]),
    "clbm_batch_bytes_per_step": (_D, [_P]),
    "clbm_batch_scale_exponent": (_I, [_P, _I]),
    "clbm_batch_destroy": (_I, [_P]),
    "clbm_reduce_noalloc": (_I, [_P, _I, _I, _D, _D, _P, _P, _P]),
    "clbm_alu_throughput": (_I, [_I, _D, _P]),
    "clbm_destroy": (_I, [_P]),
    "clbm_status_string": (ctypes.c_char_p, [_I]),
}

_lib = None


class ClbmError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__("%s: %s (%d)" % (where, clbm_status_string(status), status))


def library_path() -> str:
    return _build.library_path()


def load():
    """Load ``libclbm.so``; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise ImportError("CUDA library %s is not built; run __graft_entry__.build()" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status: int, where: str):
    if status != CLBM_OK:
        raise ClbmError(status, where)


def _host(a, dtype=np.float64, size=None):
    """A C-contiguous host array of dtype and its pointer (None -> NULL)."""
    if a is None:
        return None, None
    a = np.ascontiguousarray(np.asarray(a, dtype=dtype))
    if size is not None and a.size != size:
        raise ValueError("expected %d values, got %d" % (size, a.size))
    return a, a.ctypes.data_as(_P)


def _current_device():
    import torch
    return torch.cuda.current_device()


def _dev(t, numel=None, min_numel=None, dtype="float64"):
    """Pointer of a contiguous torch CUDA tensor on the current device
    (None -> NULL), after checking its element type and size: the C ABI
    takes bare pointers and cannot see a tensor that is too small or lives
    on another GPU."""
    if t is None:
        return None
    if dtype == "float64":
        ok = t.dtype.is_floating_point and t.element_size() == 8
    else:
        ok = (not t.dtype.is_floating_point) and t.element_size() == 1
    if not (t.is_cuda and ok and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA %s tensor" % ("float64" if dtype == "float64" else "uint8"))
    if t.device.index != _current_device():
        raise ValueError("tensor on cuda:%s, but the current device is cuda:%d"
                         % (t.device.index, _current_device()))
    if numel is not None and t.numel() != numel:
        raise ValueError("expected %d elements, got %d" % (numel, t.numel()))
    if min_numel is not None and t.numel() < min_numel:
        raise ValueError("expected at least %d elements, got %d" % (min_numel, t.numel()))
    return ctypes.c_void_p(t.data_ptr())


CUDA_STREAM_LEGACY = 1   # cudaStreamLegacy: the legacy default stream


def current_stream():
    """cudaStream_t of torch's current stream on the current device.

    torch reports its default stream as handle 0, which the C ABI reads as
    "use a private stream"; it is passed as cudaStreamLegacy instead, so the
    library's work is ordered with torch's work on that stream."""
    import torch
    h = torch.cuda.current_stream().cuda_stream
    return ctypes.c_void_p(h if h else CUDA_STREAM_LEGACY)


def clbm_status_string(status: int) -> str:
    return load().clbm_status_string(int(status)).decode()


def clbm_create(nx, ny, rates, force_kind=CLBM_FORCE_UNIFORM, force=None, fx=0.0, fy=0.0,
                solid=None, fmt=CLBM_FP32, stream=None):
    """clbm_create; returns the context handle.  ``stream`` is a cudaStream_t
    (e.g. from :func:`current_stream`) or None for a private stream."""
    lib = load()
    rates_a, rates_p = _host(rates, size=9)
    nforce = {CLBM_FORCE_UNIFORM: None, CLBM_FORCE_ROWS: 2 * ny,
              CLBM_FORCE_COLUMNS: 2 * nx, CLBM_FORCE_FIELD: 2 * nx * ny,
              CLBM_FORCE_SHAN_CHEN: 3}[force_kind]
    force_a, force_p = _host(force, size=nforce) if nforce else (None, None)
    solid_a, solid_p = _host(solid, dtype=np.uint8, size=nx * ny)
    h = ctypes.c_void_p()
    _check(lib.clbm_create(ctypes.byref(h), int(nx), int(ny), rates_p, int(force_kind), force_p,
                           float(fx), float(fy), solid_p, int(fmt), stream), "clbm_create")
    return h


def clbm_destroy(h):
    return load().clbm_destroy(h)


def clbm_init(h, rho=None, ux=None, uy=None):
    _, r = _host(rho)
    _, x = _host(ux)
    _, y = _host(uy)
    _check(load().clbm_init(h, r, x, y), "clbm_init")


def clbm_get_size(h):
    nx, ny = ctypes.c_int(), ctypes.c_int()
    _check(load().clbm_get_size(h, ctypes.byref(nx), ctypes.byref(ny)), "clbm_get_size")
    return nx.value, ny.value


def clbm_debug_fail_next(what):
    """Test hook: the next device allocation (CLBM_FAIL_ALLOC) or step launch
    (CLBM_FAIL_LAUNCH) of the library reports failure."""
    _check(load().clbm_debug_fail_next(int(what)), "clbm_debug_fail_next")


def _nodes(h):
    nx, ny = clbm_get_size(h)
    return nx * ny


def clbm_init_dev(h, rho=None, ux=None, uy=None):
    n = _nodes(h)
    _check(load().clbm_init_dev(h, _dev(rho, n), _dev(ux, n), _dev(uy, n)), "clbm_init_dev")


def clbm_set_populations(h, f, pre_collision=True):
    """Set the state from host FP64 f [9][ny][nx]: a pre-collision state
    that is collided once (pre_collision=True), or a post-collision state
    stored as given (False)."""
    _, p = _host(f, size=9 * _nodes(h))
    _check(load().clbm_set_populations(h, p, int(bool(pre_collision))), "clbm_set_populations")


def clbm_get_populations(h, out, pre_collision=False):
    """Fill ``out`` (float64, 9*ny*nx, host) with the post-collision state
    (pre_collision=False) or the pre-collision state the next step collides
    (True)."""
    if not (isinstance(out, np.ndarray) and out.dtype == np.float64 and out.flags.c_contiguous
            and out.size == 9 * _nodes(h)):
        raise ValueError("out must be a C-contiguous float64 numpy array of 9*nx*ny values")
    _check(load().clbm_get_populations(h, out.ctypes.data_as(_P), int(bool(pre_collision))),
           "clbm_get_populations")
    return out


def clbm_get_window(h, x0, y0, w, hh, out):
    """Fill ``out`` (float64 [9][hh][w], host) with a periodic window."""
    if not (isinstance(out, np.ndarray) and out.dtype == np.float64 and out.flags.c_contiguous
            and out.size == 9 * w * hh):
        raise ValueError("out must be a C-contiguous float64 array of 9*w*h values")
    _check(load().clbm_get_window(h, int(x0), int(y0), int(w), int(hh), out.ctypes.data_as(_P)),
           "clbm_get_window")
    return out


def clbm_get_window_async(h, x0, y0, w, hh, out):
    """Enqueue the window read into ``out`` (float64 [9][hh][w], host; page-
    locked for the copy to overlap later work) on the lattice's stream; the
    values are there once the stream has passed it (an event recorded on
    the stream after this call, or clbm_synchronize).  The caller keeps
    ``out`` alive until then."""
    if not (isinstance(out, np.ndarray) and out.dtype == np.float64 and out.flags.c_contiguous
            and out.size == 9 * w * hh):
        raise ValueError("out must be a C-contiguous float64 array of 9*w*h values")
    _check(load().clbm_get_window_async(h, int(x0), int(y0), int(w), int(hh), out.ctypes.data_as(_P)),
           "clbm_get_window_async")
    return out


def clbm_step(h, n):
    _check(load().clbm_step(h, int(n)), "clbm_step")


def clbm_moments(h, rho=None, ux=None, uy=None):
    """Fill host float64 arrays (any may be None) with rho, ux, uy."""
    ptrs = []
    for a in (rho, ux, uy):
        if a is None:
            ptrs.append(None)
        else:
            if not (a.dtype == np.float64 and a.flags.c_contiguous):
                raise ValueError("outputs must be C-contiguous float64")
            ptrs.append(a.ctypes.data_as(_P))
    _check(load().clbm_moments(h, *ptrs), "clbm_moments")


def clbm_moments_dev(h, rho=None, ux=None, uy=None):
    n = _nodes(h)
    _check(load().clbm_moments_dev(h, _dev(rho, n), _dev(ux, n), _dev(uy, n)), "clbm_moments_dev")


def clbm_reduce(h):
    out = (ctypes.c_double * 3)()
    st = load().clbm_reduce(h, out)
    _check(st, "clbm_reduce")
    return out[0], out[1], out[2]


def clbm_l2_error(h, ua, va):
    a, pa = _host(ua)
    b, pb = _host(va)
    out = ctypes.c_double()
    _check(load().clbm_l2_error(h, pa, pb, ctypes.byref(out)), "clbm_l2_error")
    return out.value


def clbm_reduce_noalloc(f, nx, ny, fx, fy, solid, out, stream=None):
    """FP64 totals of a caller-held device population field, without any
    device allocation (for callers that may not allocate).  ``f``: contiguous
    CUDA float64 [9][ny][nx]; ``solid``: CUDA uint8 [ny][nx] or None; ``out``:
    CUDA float64 with 4 elements, written on ``stream`` (a cudaStream_t, None
    for the legacy default stream).  Asynchronous; marshals pointers only."""
    nx, ny = int(nx), int(ny)
    fp = _dev(f, numel=9 * nx * ny)
    sp = _dev(solid, numel=nx * ny, dtype="uint8")
    op = _dev(out, min_numel=4)
    _check(load().clbm_reduce_noalloc(fp, nx, ny, float(fx), float(fy), sp, op, stream),
           "clbm_reduce_noalloc")


ALU_FP64, ALU_FP32, ALU_FP32X2, ALU_FP64_ADD, ALU_FP64_MUL = 0, 1, 2, 3, 4


def clbm_alu_throughput(kind, seconds=1.5):
    """Measured operations per second of the current GPU (kind: ALU_FP64,
    ALU_FP32 or ALU_FP32X2 fused multiply-adds, ALU_FP64_ADD, ALU_FP64_MUL)."""
    out = ctypes.c_double()
    _check(load().clbm_alu_throughput(int(kind), float(seconds), ctypes.byref(out)), "clbm_alu_throughput")
    return out.value


def clbm_set_forcing_scheme(h, scheme):
    _check(load().clbm_set_forcing_scheme(h, int(scheme)), "clbm_set_forcing_scheme")


def clbm_synchronize(h):
    _check(load().clbm_synchronize(h), "clbm_synchronize")


def clbm_scale_exponent(h) -> int:
    return load().clbm_scale_exponent(h)


def clbm_set_scale_exponent(h, k):
    _check(load().clbm_set_scale_exponent(h, int(k)), "clbm_set_scale_exponent")


def clbm_set_tuning(h, vec_bytes=16, packed=0, prefetch=0, stages=0):
    _check(load().clbm_set_tuning(h, int(vec_bytes), int(packed), int(prefetch), int(stages)),
           "clbm_set_tuning")


def clbm_get_tuning(h):
    v, p, d, st = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load().clbm_get_tuning(h, ctypes.byref(v), ctypes.byref(p), ctypes.byref(d),
                                  ctypes.byref(st)), "clbm_get_tuning")
    return v.value, p.value, d.value, st.value


def clbm_set_sparse(h, mode):
    _check(load().clbm_set_sparse(h, int(mode)), "clbm_set_sparse")


def clbm_sparse_tasks(h) -> int:
    return load().clbm_sparse_tasks(h)


def clbm_set_rounding(h, mode):
    _check(load().clbm_set_rounding(h, int(mode)), "clbm_set_rounding")


def clbm_bytes_per_update(h) -> float:
    return load().clbm_bytes_per_update(h)


def clbm_fluid_nodes(h) -> int:
    return load().clbm_fluid_nodes(h)


class _DomainDesc(ctypes.Structure):
    """clbm_domain_desc of include/clbm.h."""
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("rates", ctypes.c_double * 9),
                ("force_kind", ctypes.c_int), ("force", ctypes.c_void_p),
                ("fx", ctypes.c_double), ("fy", ctypes.c_double), ("solid", ctypes.c_void_p),
                ("forcing", ctypes.c_int)]


def clbm_batch_create(domains, fmt=CLBM_FP32, stream=None):
    """clbm_batch_create.  ``domains``: list of dicts with keys nx, ny, rates
    and optionally force_kind, force, fx, fy, solid (numpy arrays)."""
    lib = load()
    keep = []
    arr = (_DomainDesc * len(domains))()
    for k, d in enumerate(domains):
        nx, ny = int(d["nx"]), int(d["ny"])
        arr[k].nx, arr[k].ny = nx, ny
        r, _ = _host(d["rates"], size=9)
        for i in range(9):
            arr[k].rates[i] = float(r[i])
        kind = int(d.get("force_kind", CLBM_FORCE_UNIFORM))
        arr[k].force_kind = kind
        nforce = {CLBM_FORCE_UNIFORM: None, CLBM_FORCE_ROWS: 2 * ny,
                  CLBM_FORCE_COLUMNS: 2 * nx, CLBM_FORCE_FIELD: 2 * nx * ny}[kind]
        fa, fp = _host(d.get("force"), size=nforce) if nforce else (None, None)
        sa, sp = _host(d.get("solid"), dtype=np.uint8, size=nx * ny)
        keep += [fa, sa]
        arr[k].force = fp
        arr[k].fx, arr[k].fy = float(d.get("fx", 0.0)), float(d.get("fy", 0.0))
        arr[k].solid = sp
        arr[k].forcing = int(d.get("forcing", CLBM_FORCING_CONSISTENT))
    h = ctypes.c_void_p()
    _check(lib.clbm_batch_create(ctypes.byref(h), len(domains), ctypes.cast(arr, _P), int(fmt), stream),
           "clbm_batch_create")
    return h


def _bcall(name, *args):
    _check(getattr(load(), name)(*args), name)


def clbm_batch_init(h, dom, rho=None, ux=None, uy=None):
    _, r = _host(rho)
    _, x = _host(ux)
    _, y = _host(uy)
    _bcall("clbm_batch_init", h, int(dom), r, x, y)


def clbm_batch_set_populations(h, dom, f, pre_collision=True):
    _, p = _host(f)
    _bcall("clbm_batch_set_populations", h, int(dom), p, int(bool(pre_collision)))


def clbm_batch_get_populations(h, dom, out, pre_collision=False):
    if not (isinstance(out, np.ndarray) and out.dtype == np.float64 and out.flags.c_contiguous):
        raise ValueError("out must be a C-contiguous float64 numpy array")
    _bcall("clbm_batch_get_populations", h, int(dom), out.ctypes.data_as(_P), int(bool(pre_collision)))
    return out


def clbm_batch_moments(h, dom, rho, ux, uy):
    ptrs = [None if a is None else a.ctypes.data_as(_P) for a in (rho, ux, uy)]
    _bcall("clbm_batch_moments", h, int(dom), *ptrs)


def clbm_batch_reduce(h, dom):
    out = (ctypes.c_double * 3)()
    _bcall("clbm_batch_reduce", h, int(dom), out)
    return out[0], out[1], out[2]


def clbm_batch_l2_error(h, dom, ua, va):
    a, pa = _host(ua)
    b, pb = _host(va)
    out = ctypes.c_double()
    _bcall("clbm_batch_l2_error", h, int(dom), pa, pb, ctypes.byref(out))
    return out.value


def clbm_batch_step(h, n):
    _bcall("clbm_batch_step", h, int(n))


def clbm_batch_set_tuning(h, vec_bytes, packed, stages=0, schedule=CLBM_SCHEDULE_INTERLEAVED):
    _bcall("clbm_batch_set_tuning", h, int(vec_bytes), int(packed), int(stages), int(schedule))


def clbm_batch_get_tuning(h):
    v, p, st, sc = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _bcall("clbm_batch_get_tuning", h, ctypes.byref(v), ctypes.byref(p), ctypes.byref(st),
           ctypes.byref(sc))
    return v.value, p.value, st.value, sc.value


def clbm_batch_autotune(h, steps, timed=True):
    ms = ctypes.c_double(0.0)
    _bcall("clbm_batch_autotune", h, int(steps), ctypes.byref(ms) if timed else None)
    return ms.value if timed else None


def clbm_batch_set_mode(h, persistent, resident=0, order=0):
    _bcall("clbm_batch_set_mode", h, int(persistent), int(resident), int(order))


def clbm_batch_get_mode(h):
    p, r, o = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _bcall("clbm_batch_get_mode", h, ctypes.byref(p), ctypes.byref(r), ctypes.byref(o))
    return p.value, r.value, o.value


def clbm_batch_resident_lattices(h) -> int:
    return load().clbm_batch_resident_lattices(h)


def clbm_batch_set_wait(h, spin_limit, delay_ns=0):
    _bcall("clbm_batch_set_wait", h, int(spin_limit), int(delay_ns))


def clbm_batch_synchronize(h):
    _bcall("clbm_batch_synchronize", h)


def clbm_batch_fluid_nodes(h) -> int:
    return load().clbm_batch_fluid_nodes(h)


def clbm_batch_bytes_per_step(h) -> float:
    return load().clbm_batch_bytes_per_step(h)


def clbm_batch_scale_exponent(h, dom) -> int:
    return load().clbm_batch_scale_exponent(h, int(dom))


def clbm_batch_destroy(h):
    return load().clbm_batch_destroy(h)


class Batch:
    """Owns one batch; methods are the clbm_batch_* entry points."""

    def __init__(self, domains, fmt=CLBM_FP32, stream=None):
        if isinstance(fmt, str):
            fmt = FORMATS[fmt]
        self.shapes = [(int(d["nx"]), int(d["ny"])) for d in domains]
        self.h = clbm_batch_create(domains, fmt, stream)

    def close(self):
        if self.h is not None and self.h.value:
            clbm_batch_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def init(self, dom, rho=None, ux=None, uy=None):
        clbm_batch_init(self.h, dom, rho, ux, uy)

    def set_populations(self, dom, f, pre_collision=True):
        nx, ny = self.shapes[dom]
        if np.asarray(f).size != 9 * nx * ny:
            raise ValueError("expected 9*nx*ny values")
        clbm_batch_set_populations(self.h, dom, f, pre_collision)

    def get_populations(self, dom, pre_collision=False):
        nx, ny = self.shapes[dom]
        return clbm_batch_get_populations(self.h, dom, np.empty((9, ny, nx)), pre_collision)

    def moments(self, dom):
        nx, ny = self.shapes[dom]
        rho, ux, uy = (np.empty((ny, nx)) for _ in range(3))
        clbm_batch_moments(self.h, dom, rho, ux, uy)
        return rho, ux, uy

    def reduce(self, dom):
        return clbm_batch_reduce(self.h, dom)

    def l2_error(self, dom, ua, va):
        return clbm_batch_l2_error(self.h, dom, ua, va)

    def step(self, n=1):
        clbm_batch_step(self.h, n)

    def autotune(self, steps=10, timed=True):
        return clbm_batch_autotune(self.h, steps, timed)

    def synchronize(self):
        clbm_batch_synchronize(self.h)

    @property
    def tuning(self):
        return clbm_batch_get_tuning(self.h)

    @tuning.setter
    def tuning(self, t):
        clbm_batch_set_tuning(self.h, *t)

    @property
    def fluid_nodes(self):
        return clbm_batch_fluid_nodes(self.h)

    @property
    def bytes_per_step(self):
        return clbm_batch_bytes_per_step(self.h)

    @property
    def mode(self):
        """(persistent, resident, order); see clbm_batch_set_mode."""
        return clbm_batch_get_mode(self.h)

    @mode.setter
    def mode(self, m):
        clbm_batch_set_mode(self.h, *m)

    @property
    def resident_lattices(self):
        return clbm_batch_resident_lattices(self.h)

    def set_wait(self, spin_limit, delay_ns=0):
        clbm_batch_set_wait(self.h, spin_limit, delay_ns)


class Lattice:
    """Owns one context; methods are the entry points above."""

    def __init__(self, nx, ny, rates, fmt=CLBM_FP32, fx=0.0, fy=0.0, force_kind=CLBM_FORCE_UNIFORM,
                 force=None, solid=None, stream=None, forcing=CLBM_FORCING_CONSISTENT):
        if isinstance(fmt, str):
            fmt = FORMATS[fmt]
        self.nx, self.ny, self.fmt = int(nx), int(ny), fmt
        self.h = clbm_create(nx, ny, rates, force_kind, force, fx, fy, solid, fmt, stream)
        if forcing != CLBM_FORCING_CONSISTENT:
            clbm_set_forcing_scheme(self.h, forcing)
            clbm_init(self.h)

    def close(self):
        if self.h is not None and self.h.value:
            clbm_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def init(self, rho=None, ux=None, uy=None):
        clbm_init(self.h, rho, ux, uy)

    def set_populations(self, f, pre_collision=True):
        clbm_set_populations(self.h, f, pre_collision)

    def get_populations(self, pre_collision=False):
        out = np.empty((9, self.ny, self.nx))
        return clbm_get_populations(self.h, out, pre_collision)

    def window(self, x0, y0, w, h):
        out = np.empty((9, h, w))
        return clbm_get_window(self.h, x0, y0, w, h, out)

    def window_async(self, x0, y0, out):
        """Enqueue a read of the window of out's shape [9][h][w] (see
        clbm_get_window_async)."""
        return clbm_get_window_async(self.h, x0, y0, out.shape[2], out.shape[1], out)

    def step(self, n=1):
        clbm_step(self.h, n)

    def moments(self):
        rho = np.empty((self.ny, self.nx))
        ux = np.empty_like(rho)
        uy = np.empty_like(rho)
        clbm_moments(self.h, rho, ux, uy)
        return rho, ux, uy

    def reduce(self):
        return clbm_reduce(self.h)

    def l2_error(self, ua, va):
        return clbm_l2_error(self.h, ua, va)

    def synchronize(self):
        clbm_synchronize(self.h)

    @property
    def tuning(self):
        """(vec_bytes, packed, prefetch, stages) of the step kernel."""
        return clbm_get_tuning(self.h)

    @tuning.setter
    def tuning(self, t):
        clbm_set_tuning(self.h, *t)

    def set_sparse(self, mode):
        clbm_set_sparse(self.h, mode)

    def set_rounding(self, mode):
        clbm_set_rounding(self.h, mode)

    @property
    def sparse_tasks(self):
        return clbm_sparse_tasks(self.h)

    @property
    def bytes_per_update(self):
        return clbm_bytes_per_update(self.h)

    @property
    def fluid_nodes(self):
        return clbm_fluid_nodes(self.h)

    @property
    def scale_exponent(self):
        return clbm_scale_exponent(self.h)
