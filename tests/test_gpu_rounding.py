"""Stochastic rounding of the 16-bit stores (clbm_set_rounding): the same
bits for every launch shape, run and graph replay; one rounding within one
storage step of the FP64 oracle; and small increments that nearest-even
rounding drops are kept on average (a body force below half a storage step
per step still accelerates the fluid)."""
import numpy as np
import pytest

import oracle as O
from paper_1705_11092_gb300 import inputs

pytestmark = pytest.mark.gpu

U_FMT = {"fp16": 2.0 ** -11, "bf16": 2.0 ** -8}


@pytest.fixture(scope="module")
def clbm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1705_11092_gb300 import clbm as mod
    mod.load()
    return mod


def _lattice():
    nx, ny = 301, 37
    rng = np.random.default_rng(12)
    solid = (rng.random((ny, nx)) < 0.1).astype(np.uint8)
    solid[0, :] = 1
    return nx, ny, solid


@pytest.mark.parametrize("fmt", ["fp16", "bf16"])
def test_same_bits_for_every_shape_run_and_graph_replay(clbm, fmt):
    nx, ny, solid = _lattice()
    S = O.rates(1.0, 1.0, 1.1, 1.5, 0.9, 1.0)
    f0 = inputs.random_populations(nx, ny, 0.05, seed=9) * (solid == 0)
    outs = []
    runs = [((16, 1, 0, 2), 64), ((16, 0, 0, 0), 64), ((8, 1, 0, 3), 64), ((16, 1, 0, 2), 64),
            ((16, 1, 0, 2), 1)]          # last: 64 single-step calls (no graphs)
    for shape, chunk in runs:
        with clbm.Lattice(nx, ny, S, fmt=fmt, fx=2e-5, solid=solid) as lat:
            lat.tuning = shape
            lat.set_rounding(clbm.CLBM_ROUND_STOCHASTIC)
            lat.set_populations(f0)
            for _ in range(64 // chunk):
                lat.step(chunk)
            outs.append(lat.get_populations())
    for o in outs[1:]:
        assert np.array_equal(outs[0], o)
    # and it differs from nearest rounding
    with clbm.Lattice(nx, ny, S, fmt=fmt, fx=2e-5, solid=solid) as lat:
        lat.set_populations(f0)
        lat.step(64)
        assert not np.array_equal(lat.get_populations(), outs[0])


@pytest.mark.parametrize("fmt", ["fp16", "bf16"])
def test_one_step_within_one_storage_step(clbm, fmt):
    """From an FP64-exact start (the stored values of a first nearest-rounded
    state), one stochastic step differs from the oracle's step by less than
    one storage step of each value plus the FP32 arithmetic."""
    nx, ny, solid = _lattice()
    S = O.rates(1.0, 1.0, 1.2, 1.4, 1.0, 1.1)
    f0 = inputs.random_populations(nx, ny, 0.05, seed=10) * (solid == 0)
    with clbm.Lattice(nx, ny, S, fmt=fmt, fx=1e-4, solid=solid) as lat:
        lat.set_rounding(clbm.CLBM_ROUND_STOCHASTIC)
        lat.set_populations(f0)
        start = lat.get_populations()        # decoded stored state (exact)
        lat.step(1)
        got = lat.get_populations()
    ref = O.Lattice(nx, ny, S, 1e-4, 0.0, solid=solid, mode=O.MODE_PRINTED)
    expect = ref.collide(ref.stream(start))
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)[:, None, None]
    g = np.abs(expect - w)
    bound = 2 * U_FMT[fmt] * g + 64 * 2.0 ** -24 * g.max()
    assert np.all(np.abs(got - expect) <= bound * (solid == 0) + 1e-300)


def test_small_force_increments_accumulate(clbm):
    """A 256 x 256 periodic FP16 lattice holding a uniform stream u = 0.05
    (every node alike) under Fx = 1e-7: each step adds about 3e-8 to a
    population, some 1/500 of the FP16 step of the stored values (~1.5e-5).
    Nearest rounding returns the same bits every step, so the fluid never
    accelerates; stochastic rounding keeps the increment on average, so the
    total momentum gained after n steps is n Fx N within a few per cent."""
    n_side, n, F = 256, 100, 1e-7
    S = O.rates(1.0, 1.0, 1.0, 1 / 0.6, 1.0, 1.0)
    ux = np.full((n_side, n_side), 0.05)
    expect = n * F * n_side * n_side
    got = {}
    for mode in ("nearest", "stochastic"):
        with clbm.Lattice(n_side, n_side, S, fmt="fp16", fx=F) as lat:
            if mode == "stochastic":
                lat.set_rounding(clbm.CLBM_ROUND_STOCHASTIC)
            lat.init(None, ux, None)
            _, p0, _ = lat.reduce()
            lat.step(n)
            _, p1, _ = lat.reduce()
            got[mode] = p1 - p0
    assert abs(got["stochastic"] - expect) < 0.05 * expect, got
    assert abs(got["nearest"]) < 0.01 * expect, got


def test_rounding_mode_checks(clbm):
    S = O.rates(1.0, 1.0, 1.0, 1.5, 1.0, 1.0)
    with clbm.Lattice(16, 16, S, fmt="fp32") as lat:
        with pytest.raises(Exception):
            lat.set_rounding(clbm.CLBM_ROUND_STOCHASTIC)
    with clbm.Lattice(16, 16, S, fmt="fp16") as lat:
        with pytest.raises(Exception):
            lat.set_rounding(7)
        lat.set_rounding(clbm.CLBM_ROUND_STOCHASTIC)
        lat.set_rounding(clbm.CLBM_ROUND_NEAREST)
