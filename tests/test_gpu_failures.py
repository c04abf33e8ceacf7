"""Failure paths of the C ABI, driven from the host by the test hook
clbm_debug_fail_next (no fault, trap or hang on the GPU: the failed call
sends nothing there).

* A failed device allocation returns CLBM_ERR_OOM and leaves the context
  usable; a failed clbm_create returns no handle.
* A failed step launch returns CLBM_ERR_CUDA and makes the error sticky:
  every later call on that context returns CLBM_ERR_STATE until
  clbm_destroy, which still succeeds.  Other contexts are unaffected.
"""
import ctypes

import numpy as np
import pytest

import oracle as O
from paper_1705_11092_gb300 import inputs

pytestmark = pytest.mark.gpu

S = O.rates(1.0, 1.0, 1.0, 1.5, 1.0, 1.0)


@pytest.fixture(scope="module")
def clbm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1705_11092_gb300 import clbm as mod
    mod.load()
    yield mod
    mod.clbm_debug_fail_next(mod.CLBM_FAIL_NONE)


def _status(call):
    from paper_1705_11092_gb300 import clbm
    try:
        call()
    except clbm.ClbmError as e:
        return e.status
    return clbm.CLBM_OK


def test_allocation_failure_in_create_returns_no_handle(clbm):
    clbm.clbm_debug_fail_next(clbm.CLBM_FAIL_ALLOC)
    lib = clbm.load()
    h = ctypes.c_void_p(1234)
    r = np.asarray(S, np.float64)
    st = lib.clbm_create(ctypes.byref(h), 32, 16, r.ctypes.data_as(ctypes.c_void_p), 0, None,
                         0.0, 0.0, None, clbm.CLBM_FP32, None)
    assert st == clbm.CLBM_ERR_OOM
    assert h.value is None
    # the hook fired once: the next create succeeds
    with clbm.Lattice(32, 16, S, fmt="fp32") as lat:
        lat.step(2)
        lat.synchronize()


def test_allocation_failure_leaves_the_context_usable(clbm):
    nx, ny = 48, 20
    f0 = inputs.random_populations(nx, ny, 0.05, seed=5)
    with clbm.Lattice(nx, ny, S, fmt="fp64", fx=1e-5) as lat:
        lat.step(3)
        clbm.clbm_debug_fail_next(clbm.CLBM_FAIL_ALLOC)
        # the first read-back allocates its staging buffer: that fails
        assert _status(lambda: lat.set_populations(f0)) == clbm.CLBM_ERR_OOM
        # nothing is sticky: the same calls work now
        lat.set_populations(f0)
        lat.step(4)
        a = lat.get_populations()
        assert np.isfinite(a).all()
        assert lat.reduce()[0] == pytest.approx(f0.sum(), rel=1e-13)


def test_launch_failure_is_sticky_until_destroy(clbm):
    nx, ny = 40, 24
    lat = clbm.Lattice(nx, ny, S, fmt="fp32", fx=1e-5)
    other = clbm.Lattice(nx, ny, S, fmt="fp32", fx=1e-5)
    try:
        lat.step(2)
        lat.synchronize()
        clbm.clbm_debug_fail_next(clbm.CLBM_FAIL_LAUNCH)
        assert _status(lambda: lat.step(1)) == clbm.CLBM_ERR_CUDA
        for call in (lambda: lat.step(1), lat.synchronize, lat.reduce, lat.get_populations,
                     lambda: lat.init(), lat.moments,
                     lambda: lat.set_populations(np.zeros((9, ny, nx)))):
            assert _status(call) == clbm.CLBM_ERR_STATE
        # another context is not affected
        other.step(3)
        other.synchronize()
        assert np.isfinite(other.reduce()[0])
    finally:
        assert clbm.clbm_destroy(lat.h) == clbm.CLBM_OK
        lat.h = None
        other.close()


def test_batch_launch_failure_is_sticky(clbm):
    doms = [{"nx": 34, "ny": 17, "rates": S, "fx": 1e-5, "solid": inputs.channel_mask(34, 17)},
            {"nx": 66, "ny": 33, "rates": S, "fx": 2e-6, "solid": inputs.channel_mask(66, 33)}]
    b = clbm.Batch(doms, fmt="fp32")
    try:
        b.step(1)
        b.synchronize()
        clbm.clbm_debug_fail_next(clbm.CLBM_FAIL_LAUNCH)
        assert _status(lambda: b.step(1)) == clbm.CLBM_ERR_CUDA
        assert _status(lambda: b.step(1)) == clbm.CLBM_ERR_STATE
        assert _status(b.synchronize) == clbm.CLBM_ERR_STATE
        assert _status(lambda: b.reduce(0)) == clbm.CLBM_ERR_STATE
    finally:
        assert clbm.clbm_batch_destroy(b.h) == clbm.CLBM_OK
        b.h = None


def test_hook_rejects_unknown_kinds(clbm):
    assert _status(lambda: clbm.clbm_debug_fail_next(7)) == clbm.CLBM_ERR_ARG
