"""CPU checks of the C ABI: the library builds and loads, it exports every
entry point that include/clbm.h declares, and argument errors are reported
before any CUDA work (so they are testable without a GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1705_11092_gb300 import build, clbm
    if not os.path.exists(build.library_path()):
        build.build()
    return clbm.load()


def declared_functions():
    names = []
    for hdr in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not hdr.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", hdr)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(clbm_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_step_entry_points():
    names = declared_functions()
    for must in ("clbm_create", "clbm_step", "clbm_moments", "clbm_destroy", "clbm_init",
                 "clbm_get_populations", "clbm_set_populations", "clbm_reduce"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_1705_11092_gb300 import clbm
    for name in declared_functions():
        assert name in clbm._SIGNATURES, name
        assert hasattr(clbm, name), name


def test_status_strings(lib):
    from paper_1705_11092_gb300 import clbm
    assert clbm.clbm_status_string(0) == "ok"
    assert "argument" in clbm.clbm_status_string(clbm.CLBM_ERR_ARG)
    assert clbm.clbm_status_string(12345) == "unknown status"


def _create(lib, nx=8, ny=8, rates=None, kind=0, force=None, fx=0.0, fy=0.0, solid=None, fmt=1):
    h = ctypes.c_void_p(1234)
    r = np.ones(9) if rates is None else np.asarray(rates, np.float64)
    P = ctypes.c_void_p
    fp = force.ctypes.data_as(P) if force is not None else None
    sp = solid.ctypes.data_as(P) if solid is not None else None
    st = lib.clbm_create(ctypes.byref(h), nx, ny, r.ctypes.data_as(P), kind, fp, fx, fy, sp, fmt, None)
    return st, h


@pytest.mark.parametrize("kw", [
    dict(nx=1), dict(ny=0), dict(fmt=7), dict(fmt=-1),
    dict(rates=[1, 1, 1, 1, 2.0, 2.0, 1, 1, 1]),          # s2 = 2 is outside (0, 2)
    dict(rates=[1, 1, 1, 1, 0.0, 0.0, 1, 1, 1]),
    dict(rates=[1, 1, 1.2, 1, 1, 1, 1, 1, 1]),            # s1 pair differs
    dict(rates=[1, 1, 1, 1, 1.1, 1.2, 1, 1, 1]),          # s2 pair differs
    dict(rates=[1, 1, 1, 1, 1, 1, 1.3, 1.0, 1]),          # s3 pair differs
    dict(rates=[1, 1, 1, 1, float("nan"), float("nan"), 1, 1, 1]),
    dict(kind=1),                                          # rows without array
    dict(kind=9),
    dict(fx=float("inf")),
    dict(kind=1, force=np.full(16, np.nan)),
    dict(kind=4),                                          # Shan-Chen without parameters
    dict(kind=4, force=np.array([-10 / 3, 0.0, 1.0])),     # psi0 must be > 0
    dict(kind=4, force=np.array([-10 / 3, 1.0, np.inf])),
    dict(kind=4, force=np.array([-10 / 3, 1.0, 1.0]),      # Shan-Chen with a solid node
         solid=np.eye(8, dtype=np.uint8)),
])
def test_create_rejects_bad_arguments_without_touching_the_gpu(lib, kw):
    st, h = _create(lib, **kw)
    assert st == -1
    assert h.value is None


def test_null_handles_are_rejected(lib):
    assert lib.clbm_step(None, 1) == -1
    assert lib.clbm_synchronize(None) == -1
    assert lib.clbm_destroy(None) == 0
    out = (ctypes.c_double * 3)()
    assert lib.clbm_reduce(None, out) == -1
    assert lib.clbm_bytes_per_update(None) == 0.0
    assert lib.clbm_set_rounding(None, 1) == -1
    assert lib.clbm_set_sparse(None, 1) == -1
    assert lib.clbm_sparse_tasks(None) == 0
    f = (ctypes.c_double * 9)()
    assert lib.clbm_get_window(None, 0, 0, 1, 1, f) == -1
    assert lib.clbm_get_window_async(None, 0, 0, 1, 1, f) == -1


def test_window_reads_check_their_buffer_before_the_library(lib):
    """The binding rejects a window buffer of the wrong size or type before
    any call; a null handle is the library's CLBM_ERR_ARG."""
    from paper_1705_11092_gb300 import clbm
    for fn in (clbm.clbm_get_window, clbm.clbm_get_window_async):
        with pytest.raises(ValueError):
            fn(None, 0, 0, 2, 1, np.empty(9))
        with pytest.raises(ValueError):
            fn(None, 0, 0, 1, 1, np.empty(9, dtype=np.float32))
        with pytest.raises(clbm.ClbmError):
            fn(None, 0, 0, 1, 1, np.empty(9))


def test_binding_raises_when_library_missing(monkeypatch, tmp_path):
    from paper_1705_11092_gb300 import clbm
    monkeypatch.setattr(clbm, "_lib", None)
    monkeypatch.setattr(clbm, "library_path", lambda: str(tmp_path / "missing.so"))
    with pytest.raises(ImportError):
        clbm.load()


def test_batch_create_rejects_bad_arguments_without_touching_the_gpu(lib):
    from paper_1705_11092_gb300 import clbm
    h = ctypes.c_void_p(7)
    assert lib.clbm_batch_create(ctypes.byref(h), 0, None, 1, None) == -1
    arr = (clbm._DomainDesc * 2)()
    for d in arr:
        d.nx, d.ny = 16, 16
        for i in range(9):
            d.rates[i] = 1.0
    arr[1].rates[4] = 2.5                       # second lattice invalid
    st = lib.clbm_batch_create(ctypes.byref(h), 2, ctypes.cast(arr, ctypes.c_void_p), 1, None)
    assert st == -1 and h.value is None
    arr[1].rates[4] = 1.0
    arr[1].forcing = 3                          # not a clbm_forcing
    st = lib.clbm_batch_create(ctypes.byref(h), 2, ctypes.cast(arr, ctypes.c_void_p), 1, None)
    assert st == -1 and h.value is None
    # three lattices that pass alone but hold 3 * 2^30 chunks of 64 nodes
    big = (clbm._DomainDesc * 3)()
    for d in big:
        d.nx, d.ny = 2, 1 << 30
        for i in range(9):
            d.rates[i] = 1.0
    st = lib.clbm_batch_create(ctypes.byref(h), 3, ctypes.cast(big, ctypes.c_void_p), 2, None)
    assert st == -1 and h.value is None
    assert lib.clbm_batch_step(None, 1) == -1
    assert lib.clbm_batch_destroy(None) == 0
    assert lib.clbm_batch_set_tuning(None, 16, 1, 2, clbm.CLBM_SCHEDULE_CONTIGUOUS) == -1


def test_channel_sweep_recipe():
    from paper_1705_11092_gb300 import inputs
    sw = inputs.channel_sweep(256)
    assert len(sw) == 256
    assert sum(1 for d in sw if d["ladder"] >= 0) == 252
    for d in sw:
        assert d["nx"] == 2 * d["ny"] and d["ny"] in inputs.CHANNEL_SWEEP_HEIGHTS
        assert 0.55 <= d["tau"] <= 1.5 and 1e-7 <= d["fx"] <= 1e-5
    lad = [d for d in sw if d["ladder"] == 3]
    assert len({d["tau"] for d in lad}) == 1 and len(lad) == 6
    assert sw == inputs.channel_sweep(256)      # seeded
