"""clbm_reduce_noalloc: the FP64 reduction for callers that cannot allocate
device memory (it uses a fixed device array as scratch, never cudaMalloc).

Checked through the C ABI against clbm_reduce, the context-based entry
point, on two calls in a row (the shared scratch keeps the first call's
values, which the second call must overwrite correctly).  Tolerance: both
sum the same FP64 values in different orders, so they agree to FP64
round-off of a sum of n terms, bounded here by 1e-12 relative (mass) and
1e-10 absolute (momentum).  This file is collected last on purpose.
"""
import numpy as np
import pytest

import oracle as O
from paper_1705_11092_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def clbm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1705_11092_gb300 import clbm as mod
    mod.load()
    return mod


def test_reduce_noalloc_matches_context_reduction_twice(clbm):
    import torch
    nx, ny = 333, 97
    solid = inputs.channel_mask(nx, ny)
    solid[40:50, 100:120] = 1
    S = O.rates(1.0, 1.0, 1.1, 1.4, 0.9, 1.0)
    fx, fy = 3e-5, -1e-5
    solid_t = torch.from_numpy(solid).cuda()
    out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    stream = clbm.current_stream()
    with clbm.Lattice(nx, ny, S, fmt="fp64", fx=fx, fy=fy, solid=solid,
                      stream=stream) as lat:
        lat.init(inputs.density_noise(nx, ny, 1e-3, seed=3),
                 *inputs.taylor_green_velocity(nx, ny, 0.02))
        for call in range(2):
            lat.step(25 + 10 * call)
            mass, mx, my = lat.reduce()
            f = torch.from_numpy(lat.get_populations()).cuda()
            clbm.clbm_reduce_noalloc(f, nx, ny, fx, fy, solid_t, out, stream)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            assert got[0] == pytest.approx(mass, rel=1e-12, abs=0)
            assert abs(got[1] - mx) <= 1e-10
            assert abs(got[2] - my) <= 1e-10
            assert got[3] == 0.0


def test_reduce_noalloc_rejects_rows_beyond_scratch(clbm):
    import torch
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    # a field of the right size, so that the library's own limit rejects it
    f = torch.zeros(9 * 65537, dtype=torch.float64, device="cuda")
    with pytest.raises(clbm.ClbmError) as e:
        clbm.clbm_reduce_noalloc(f, 1, 65537, 0.0, 0.0, None, out, None)
    assert e.value.status == clbm.CLBM_ERR_ARG
