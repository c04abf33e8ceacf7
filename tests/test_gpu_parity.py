"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances:
  * FP64 storage/compute: max |f*_gpu - f*_oracle| <= 1e-12 after up to 1000
    steps (the target the FP64 path is held to).
  * FP32 / FP16 / BF16 storage (FP32 compute): one collision from identical
    inputs errs by at most the storage rounding, u_fmt |g*|, plus FP32
    arithmetic, bounded by 64 * 2^-24 * max|g*| (about 100 dependent
    operations per node, each within 2^-24 relative of the largest moment);
    n steps are bounded by n times that (errors add at most linearly under
    the stable update).  u_fmt = 2^-24 (FP32), 2^-11 (FP16), 2^-8 (BF16);
    g* = f* - w rho0 is the stored deviation.
"""
import math

import numpy as np
import pytest

import oracle as O
from oracle import analytic as A
from paper_1705_11092_gb300 import inputs

pytestmark = pytest.mark.gpu

W = inputs.REST_WEIGHTS[:, None, None]
U_FMT = {"fp32": 2.0 ** -24, "fp16": 2.0 ** -11, "bf16": 2.0 ** -8,
         # stochastic rounding errs by less than one storage step
         "fp16_sr": 2.0 ** -10, "bf16_sr": 2.0 ** -7}
C_ALU = 64 * 2.0 ** -24


@pytest.fixture(scope="module")
def clbm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1705_11092_gb300 import clbm as mod
    mod.load()
    return mod


def bound(g_ref, fmt, nsteps=1):
    G = np.abs(g_ref).max()
    return nsteps * (U_FMT[fmt] * np.abs(g_ref) + C_ALU * G)


def run_pair(clbm, nx, ny, S, steps, fmt="fp64", f0=None, solid=None, fx=0.0, fy=0.0,
             force_kind=0, force=None, oracle_f=None):
    """Run GPU and oracle from the same pre-collision state; return both
    post-collision states after `steps` steps."""
    if f0 is None:
        f0 = inputs.random_populations(nx, ny, 0.05, seed=nx * 1000 + ny)
    if solid is not None:
        f0 = f0 * (solid == 0)
    if oracle_f is None:
        ofx, ofy = fx, fy
    else:
        ofx, ofy = oracle_f
    ref = O.Lattice(nx, ny, S, ofx, ofy, solid=solid, mode=O.MODE_PRINTED)
    expect = ref.collide(ref.run(f0, steps))
    with clbm.Lattice(nx, ny, S, fmt=fmt, fx=fx, fy=fy, force_kind=force_kind, force=force,
                      solid=solid) as lat:
        lat.set_populations(f0)
        lat.step(steps)
        got = lat.get_populations()
    return got, expect


# ---- FP64: <= 1e-12 --------------------------------------------------------

def test_fp64_periodic_ragged_1000_steps(clbm):
    # FP64 lanes hold 2 nodes: a warp covers 64, so nx = 150 spans three
    # chunks with a ragged tail of 22
    S = O.rates(0.8, 1.3, 1.1, 1.6, 0.9, 1.2)
    got, expect = run_pair(clbm, 150, 19, S, 1000, fx=1e-5, fy=-3e-6)
    assert np.abs(got - expect).max() <= 1e-12


def test_fp64_channel_row_force_1000_steps(clbm):
    nx, ny = 67, 24
    solid = inputs.channel_mask(nx, ny)
    F = inputs.modulated_force_rows(ny, 2e-5, 0.3)
    S = O.rates(1.0, 1.0, 1.2, 1.25, 0.95, 1.1)
    fx = F[:, 0][:, None] * np.ones((1, nx))
    got, expect = run_pair(clbm, nx, ny, S, 1000, solid=solid, force_kind=1, force=F,
                           oracle_f=(fx, 0.0))
    assert np.abs(got - expect).max() <= 1e-12


def test_fp64_obstacles_column_force(clbm):
    nx, ny = 45, 38
    rng = np.random.default_rng(7)
    solid = (rng.random((ny, nx)) < 0.2).astype(np.uint8)
    F = inputs.sinusoidal_force_columns(nx, 1e-4)
    F[:, 0] = 2e-5
    S = O.rates(1.0, 1.0, 1.0, 1.4, 1.3, 1.0)
    got, expect = run_pair(clbm, nx, ny, S, 300, solid=solid, force_kind=2, force=F,
                           oracle_f=(F[:, 0][None, :] * np.ones((ny, 1)),
                                     F[:, 1][None, :] * np.ones((ny, 1))))
    assert np.abs(got - expect).max() <= 1e-12


@pytest.mark.parametrize("nx,ny", [(2, 2), (3, 5), (5, 3), (3, 4), (65, 2), (2, 67)])
def test_fp64_degenerate_sizes_force_field(clbm, nx, ny):
    rng = np.random.default_rng(nx * 7 + ny)
    F = rng.uniform(-1e-4, 1e-4, (ny, nx, 2))
    S = O.rates(1.0, 1.0, 0.7, 1.5, 1.1, 0.9)
    got, expect = run_pair(clbm, nx, ny, S, 200, force_kind=3, force=F,
                           oracle_f=(F[..., 0], F[..., 1]))
    assert np.abs(got - expect).max() <= 1e-12


def test_fp64_channel_length_three(clbm):
    # the paper's channel of length 3 (Sec. 4A): nx smaller than a vector
    nx, ny = 3, 9
    solid = inputs.channel_mask(nx, ny)
    s2 = A.shear_rate(0.5)
    S = O.rates(s2, s2, s2, s2, 1.6, s2)
    got, expect = run_pair(clbm, nx, ny, S, 500, solid=solid, fx=0.01)
    assert np.abs(got - expect).max() <= 1e-12


# ---- reduced precision -------------------------------------------------------

@pytest.mark.parametrize("fmt", ["fp32", "fp16", "bf16"])
def test_reduced_single_collision(clbm, fmt):
    nx, ny = 300, 21      # FP32: 128 nodes per warp, FP16/BF16: 256
    S = O.rates(1.0, 1.0, 1.0, 1.0 / 0.6, 1.0, 1.0)
    got, expect = run_pair(clbm, nx, ny, S, 0, fmt=fmt, fx=1e-5)
    g_ref = expect - W
    assert np.all(np.abs(got - expect) <= bound(g_ref, fmt))


@pytest.mark.parametrize("fmt", ["fp32", "fp16", "bf16"])
def test_reduced_multi_step(clbm, fmt):
    nx, ny, n = 300, 21, 20
    solid = inputs.channel_mask(nx, ny)
    S = O.rates(1.0, 1.0, 1.0, 1.0 / 0.6, 1.0, 1.0)
    got, expect = run_pair(clbm, nx, ny, S, n, fmt=fmt, solid=solid, fx=1e-5)
    g_ref = expect - W
    assert np.all(np.abs(got - expect) <= bound(g_ref, fmt, n + 1))


# ---- initialisation, moments, reductions ------------------------------------

def test_init_equilibrium_then_steps(clbm):
    nx, ny = 96, 40
    rho = inputs.density_noise(nx, ny, 1e-3, seed=11)
    ux, uy = inputs.taylor_green_velocity(nx, ny, 0.02)
    S = O.rates(1.0, 1.0, 1.0, 1.0 / 0.55, 1.0, 1.0)
    ref = O.Lattice(nx, ny, S, 1e-6, 0.0, mode=O.MODE_PRINTED)
    f0 = ref.equilibrium(rho, ux, uy)
    expect = ref.collide(ref.run(f0, 50))
    with clbm.Lattice(nx, ny, S, fmt="fp64", fx=1e-6) as lat:
        lat.init(rho, ux, uy)
        lat.step(50)
        got = lat.get_populations()
    assert np.abs(got - expect).max() <= 1e-12


def test_moments_reduce_and_l2(clbm):
    nx, ny, n = 80, 30, 100
    solid = inputs.channel_mask(nx, ny)
    S = O.rates(1.0, 1.0, 1.1, 1.3, 1.2, 1.0)
    f0 = inputs.random_populations(nx, ny, 0.05, seed=21) * (solid == 0)
    ref = O.Lattice(nx, ny, S, 3e-5, 1e-5, solid=solid, mode=O.MODE_PRINTED)
    fn = ref.run(f0, n)
    rho_o, ux_o, uy_o = ref.moments(fn)
    with clbm.Lattice(nx, ny, S, fmt="fp64", fx=3e-5, fy=1e-5, solid=solid) as lat:
        lat.set_populations(f0)
        lat.step(n)
        rho, ux, uy = lat.moments()
        mass, mx, my = lat.reduce()
        ua = 0.01 * np.ones((ny, nx))
        va = 0.002 * np.ones((ny, nx))
        e2 = lat.l2_error(ua, va)
        assert lat.fluid_nodes == nx * (ny - 1)
        assert lat.bytes_per_update == 18 * 8 + 1.125
    assert np.abs(rho - rho_o).max() <= 1e-13
    assert np.abs(ux - ux_o).max() <= 1e-13
    assert np.abs(uy - uy_o).max() <= 1e-13
    fl = solid == 0
    assert abs(mass - rho_o[fl].sum()) <= 1e-11
    assert abs(mx - (rho_o * ux_o)[fl].sum()) <= 1e-11
    assert abs(my - (rho_o * uy_o)[fl].sum()) <= 1e-11
    assert e2 == pytest.approx(A.e2(ux_o, uy_o, ua, va, fl), rel=1e-12)


def test_mass_conservation_and_momentum_growth(clbm):
    nx, ny, n = 256, 64, 400
    S = O.rates(1.0, 1.0, 1.0, 1.0 / 0.55, 1.0, 1.0)
    with clbm.Lattice(nx, ny, S, fmt="fp64", fx=1e-6, fy=-2e-7) as lat:
        lat.init(inputs.density_noise(nx, ny, 1e-3), *inputs.taylor_green_velocity(nx, ny, 0.01))
        m0, px0, py0 = lat.reduce()
        lat.step(n)
        m1, px1, py1 = lat.reduce()
    assert abs(m1 - m0) <= 1e-12 * m0
    assert abs((px1 - px0) - n * 1e-6 * nx * ny) <= 1e-10
    assert abs((py1 - py0) + n * 2e-7 * nx * ny) <= 1e-10


# ---- launch machinery --------------------------------------------------------

def test_graph_replay_equals_single_launches(clbm):
    nx, ny = 200, 50
    S = O.rates(1.0, 1.0, 1.0, 1.5, 1.0, 1.0)
    f0 = inputs.random_populations(nx, ny, 0.05, seed=4)
    outs = []
    for chunked in (False, True):
        with clbm.Lattice(nx, ny, S, fmt="fp32", fx=1e-5) as lat:
            lat.set_populations(f0)
            if chunked:
                for _ in range(70):
                    lat.step(1)
            else:
                lat.step(70)          # two 32-step graph replays + 6 launches
            outs.append(lat.get_populations())
    assert np.array_equal(outs[0], outs[1])


def test_zero_steps_and_repeatability(clbm):
    nx, ny = 130, 17
    S = O.rates(1.0, 1.0, 1.0, 1.5, 1.0, 1.0)
    f0 = inputs.random_populations(nx, ny, 0.05, seed=9)
    res = []
    for _ in range(2):
        with clbm.Lattice(nx, ny, S, fmt="bf16", fx=1e-5) as lat:
            lat.set_populations(f0)
            a = lat.get_populations()
            lat.step(0)
            assert np.array_equal(a, lat.get_populations())
            lat.step(37)
            res.append(lat.get_populations())
    assert np.array_equal(res[0], res[1])


def test_torch_stream_and_device_outputs(clbm):
    import torch
    nx, ny = 64, 48
    S = O.rates(1.0, 1.0, 1.0, 1.6, 1.0, 1.0)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with clbm.Lattice(nx, ny, S, fmt="fp64", fx=1e-5, stream=clbm.current_stream()) as lat:
            rho_t = torch.full((ny, nx), 1.0, dtype=torch.float64, device="cuda")
            ux_t = torch.zeros((ny, nx), dtype=torch.float64, device="cuda")
            clbm.clbm_init_dev(lat.h, rho_t, ux_t, None)
            lat.step(10)
            out = torch.empty((3, ny, nx), dtype=torch.float64, device="cuda")
            clbm.clbm_moments_dev(lat.h, out[0], out[1], out[2])
            s.synchronize()
            rho, ux, uy = lat.moments()
    assert np.array_equal(out[0].cpu().numpy(), rho)
    assert np.array_equal(out[1].cpu().numpy(), ux)
    # uniform start + uniform force: momentum grows by F per step (Eq. 12, 15)
    # (rho u at time level t is t F + F/2: Eq. 15 adds F/2 to sum f_i e_i)
    assert np.allclose(ux, 10.5 * 1e-5, rtol=0, atol=1e-15)


# ---- canonical flows on the GPU ------------------------------------------------

def test_poiseuille_plain_fp64(clbm):
    """Force-driven channel nx=64, ny=33 (row 0 solid: H = 32), tau = 0.8,
    other rates 1, Fx = 1e-6, from rest.  The flow is x-invariant, so every
    column must equal the oracle's run on a 3-column channel."""
    nx, ny, n = 64, 33, 20000
    s2 = 1.0 / 0.8
    S = O.rates(1.0, 1.0, 1.0, s2, 1.0, 1.0)
    solid = inputs.channel_mask(nx, ny)
    ref = O.Lattice(3, ny, S, 1e-6, 0.0, solid=inputs.channel_mask(3, ny), mode=O.MODE_PRINTED)
    f_ref = ref.run(ref.equilibrium(1.0, 0.0, 0.0), n)
    _, ux_o, uy_o = ref.moments(f_ref)
    with clbm.Lattice(nx, ny, S, fmt="fp64", fx=1e-6, solid=solid) as lat:
        lat.init()
        lat.step(n)
        _, ux, uy = lat.moments()
    # FP64 round-off accumulated over 20000 steps (velocities ~1e-3)
    assert np.abs(ux - ux_o[:, :1]).max() <= 1e-13
    assert np.abs(uy).max() <= 1e-13
    # the profile is the start-up solution plus the bounce-back slip
    y = np.arange(ny) - 0.5
    nu = A.viscosity(s2)
    pred = A.poiseuille_startup(y, n, ny - 1, 1e-6, nu) + A.bounce_back_slip(1e-6, s2, 1.0)
    assert np.abs(ux[1:, 0] - pred[1:]).max() <= 1e-5 * np.abs(pred).max()


def test_poiseuille_nonslip_rule_converges_to_parabola(clbm):
    """Remark 4 on the GPU: s3 from the non-slip rule, run to steady state;
    E2 against the closed-form parabola at round-off level."""
    nx, ny = 64, 17
    s2 = 1.0 / 0.8
    s3 = A.nonslip_s3(s2)
    S = O.rates(1.0, 1.0, 1.0, s2, s3, 1.0)
    solid = inputs.channel_mask(nx, ny)
    y = np.arange(ny) - 0.5
    ua = A.poiseuille_steady(y, ny - 1, 1e-6, A.viscosity(s2))[:, None] * np.ones((1, nx))
    with clbm.Lattice(nx, ny, S, fmt="fp64", fx=1e-6, solid=solid) as lat:
        lat.init()
        lat.step(60000)
        e2 = lat.l2_error(ua, 0 * ua)
    assert e2 <= 1e-9


@pytest.mark.parametrize("fmt", ["fp64", "fp32"])
def test_isotropy_1024(clbm, fmt):
    """F = F0 sin(2 pi y/L) e_x and the same force turned by 90 degrees with
    the transposed initial density: the results are transposes.  The kernel
    shifts along x then y, so the two runs round differently: FP64 within
    1e-14; FP32 within the n-step bound n (u_fmt + 64 * 2^-24) max|u|."""
    n, steps = 1024, 200
    S = O.rates(1.0, 1.0, 1.0, 1.0 / 0.6, 1.0, 1.0)
    rho = inputs.density_noise(n, n, 1e-3, seed=1705)
    runs = []
    for kind, force, r in ((1, inputs.sinusoidal_force_rows(n, 1e-5), rho),
                           (2, inputs.sinusoidal_force_columns(n, 1e-5), rho.T.copy())):
        with clbm.Lattice(n, n, S, fmt=fmt, force_kind=kind, force=force) as lat:
            lat.init(r)
            lat.step(steps)
            runs.append(lat.moments())
    (ra, ua, va), (rb, ub, vb) = runs
    if fmt == "fp64":
        tol_r = tol_u = 1e-14
    else:
        tol_r = steps * (U_FMT[fmt] + C_ALU) * np.abs(ra - 1.0).max()
        tol_u = steps * (U_FMT[fmt] + C_ALU) * np.abs(ua).max()
    assert np.abs(rb.T - ra).max() <= tol_r
    assert np.abs(ub.T - va).max() <= tol_u
    assert np.abs(vb.T - ua).max() <= tol_u


def _config2_run(clbm, fmt, n, steps, transposed):
    """The isotropy workload: F = 1e-5 sin(2 pi y / n) e_x (or the same force
    turned by 90 degrees, with the transposed initial density), tau = 0.6,
    rho = 1 + 1e-3 U(-1, 1) from seed 1705, u = 0."""
    S = O.rates(1.0, 1.0, 1.0, 1.0 / 0.6, 1.0, 1.0)
    rho = inputs.density_noise(n, n, 1e-3, seed=1705)
    if transposed:
        kind, force, r = 2, inputs.sinusoidal_force_columns(n, 1e-5), rho.T.copy()
    else:
        kind, force, r = 1, inputs.sinusoidal_force_rows(n, 1e-5), rho
    with clbm.Lattice(n, n, S, fmt=fmt, force_kind=kind, force=force) as lat:
        lat.init(r)
        lat.step(steps)
        return lat.moments()


def test_config2_isotropy_5000_steps(clbm):
    """The isotropy workload at its stated length (1024 x 1024, 5000 steps),
    FP64 and FP32.  The x-forced and the transposed y-forced runs are
    transposes of each other: FP64 within 1e-13 (the two runs round in a
    different order); FP32 within its 5000-step bound
    n (u_fmt + 64 * 2^-24) max|u|, and FP32 against FP64 within the same
    bound."""
    n, steps = 1024, 5000
    res = {}
    for fmt in ("fp64", "fp32"):
        a = _config2_run(clbm, fmt, n, steps, False)
        b = _config2_run(clbm, fmt, n, steps, True)
        (ra, ua, va), (rb, ub, vb) = a, b
        if fmt == "fp64":
            tol_r = tol_u = 1e-13
        else:
            tol_r = steps * (U_FMT[fmt] + C_ALU) * np.abs(ra - 1.0).max()
            tol_u = steps * (U_FMT[fmt] + C_ALU) * np.abs(ua).max()
        assert np.abs(rb.T - ra).max() <= tol_r, fmt
        assert np.abs(ub.T - va).max() <= tol_u, fmt
        assert np.abs(vb.T - ua).max() <= tol_u, fmt
        res[fmt] = a
    # FP32 against FP64 within the same n-step bound (measured: relative L2
    # error 1.1e-4, the benchmark's config2 block reports it)
    _, u64, v64 = res["fp64"]
    _, u32, v32 = res["fp32"]
    tol = steps * (U_FMT["fp32"] + C_ALU) * max(np.abs(u64).max(), np.abs(v64).max())
    assert max(np.abs(u32 - u64).max(), np.abs(v32 - v64).max()) <= tol


def test_config2_fp64_matches_oracle_over_5000_steps(clbm):
    """The isotropy workload on a 96 x 96 lattice (the same force shape and
    noise recipe) over the full 5000 steps: FP64 populations against the
    oracle within 1e-12, for both force directions."""
    n, steps = 96, 5000
    S = O.rates(1.0, 1.0, 1.0, 1.0 / 0.6, 1.0, 1.0)
    rho = inputs.density_noise(n, n, 1e-3, seed=1705)
    Fr = inputs.sinusoidal_force_rows(n, 1e-5)
    Fc = inputs.sinusoidal_force_columns(n, 1e-5)
    cases = ((1, Fr, rho, Fr[:, 0][:, None] * np.ones((1, n)), 0.0),
             (2, Fc, rho.T.copy(), 0.0, Fc[:, 1][None, :] * np.ones((n, 1))))
    for kind, force, r, fx, fy in cases:
        ref = O.Lattice(n, n, S, fx, fy, mode=O.MODE_PRINTED)
        expect = ref.collide(ref.run(ref.equilibrium(r, 0.0, 0.0), steps))
        with clbm.Lattice(n, n, S, fmt="fp64", force_kind=kind, force=force) as lat:
            lat.init(r)
            lat.step(steps)
            got = lat.get_populations()
        assert np.abs(got - expect).max() <= 1e-12, kind


def test_1024_fp64_parity_with_oracle(clbm):
    n, steps = 1024, 10
    S = O.rates(1.0, 1.0, 1.0, 1.0 / 0.6, 1.0, 1.0)
    F = inputs.sinusoidal_force_rows(n, 1e-5)
    rho = inputs.density_noise(n, n, 1e-3, seed=1705)
    ref = O.Lattice(n, n, S, F[:, 0][:, None] * np.ones((1, n)), 0.0, mode=O.MODE_PRINTED)
    expect = ref.collide(ref.run(ref.equilibrium(rho, 0.0, 0.0), steps))
    with clbm.Lattice(n, n, S, fmt="fp64", force_kind=1, force=F) as lat:
        lat.init(rho)
        lat.step(steps)
        got = lat.get_populations()
    assert np.abs(got - expect).max() <= 1e-12


# ---- full-size sampled parity ----------------------------------------------------

def sampled_step_check(lat, S, points, force_at, solid=None, fmt="fp32"):
    """For each sample point: read the 3x3 neighbourhood at t, step once, and
    compare the node's new post-collision state with the oracle's pull +
    collision of the neighbourhood (a single step from identical inputs)."""
    nx, ny = lat.nx, lat.ny
    before = []
    for (x, y) in points:
        x0, y0 = (x - 1) % nx, (y - 1) % ny
        before.append(lat.window(x0, y0, 3, 3))
    lat.step(1)
    worst = 0.0
    for (x, y), win in zip(points, before):
        xs = [(x - 1 + k) % nx for k in range(3)]
        ys = [(y - 1 + k) % ny for k in range(3)]
        sw = None if solid is None else solid[np.ix_(ys, xs)]
        fx, fy = force_at(x, y)
        ref = O.Lattice(3, 3, S, fx, fy, solid=sw, mode=O.MODE_PRINTED)
        pre = ref.stream(win)
        got = lat.window(x, y, 1, 1)[:, 0, 0]
        if sw is not None and sw[1, 1]:
            assert np.all(got == 0.0)
            continue
        exp = O.collide_node(pre[:, 1, 1], fx, fy, S, O.MODE_PRINTED)
        g = exp - inputs.REST_WEIGHTS
        fluid = np.ones((3, 3), bool) if sw is None else sw == 0
        G = max(np.abs((win - W)[:, fluid]).max(), np.abs(g).max())
        tol = U_FMT[fmt] * np.abs(g) + C_ALU * G
        assert np.all(np.abs(got - exp) <= tol), ((x, y), got - exp, tol)
        worst = max(worst, float(np.abs(got - exp).max()))
    return worst


def edge_points(nx, ny, V):
    pts = [(0, 0), (nx - 1, ny - 1), (0, ny - 1), (nx - 1, 0)]
    for c in (32 * V - 1, 32 * V, 32 * V + 1, V - 1, V):
        pts.append((c % nx, ny // 2))
    rng = np.random.default_rng(17)
    pts += [(int(a), int(b)) for a, b in zip(rng.integers(0, nx, 8), rng.integers(0, ny, 8))]
    return pts


@pytest.mark.parametrize("fmt", ["fp32", "fp16", "bf16", "fp16_sr", "bf16_sr"])
def test_full_size_8192_sampled(clbm, fmt):
    """The benchmark's lattice: 8192 x 8192 periodic, Taylor-Green-like start
    u0 = 0.01, uniform Fx = 1e-7, tau = 0.55, in the launch configuration the
    benchmark times; sampled nodes checked against the oracle one by one.
    "_sr": stochastic rounding of the 16-bit stores."""
    n = 8192
    S = O.rates(1.0, 1.0, 1.0, 1.0 / 0.55, 1.0, 1.0)
    ux, uy = inputs.taylor_green_velocity(n, n, 0.01)
    V = {"fp32": 4, "fp16": 8, "bf16": 8}[fmt.split("_")[0]]
    with clbm.Lattice(n, n, S, fmt=fmt.split("_")[0], fx=1e-7) as lat:
        if fmt.endswith("_sr"):
            lat.set_rounding(clbm.CLBM_ROUND_STOCHASTIC)
        lat.init(None, ux, uy)
        del ux, uy
        m0, px0, _ = lat.reduce()
        lat.step(5)
        sampled_step_check(lat, S, edge_points(n, n, V), lambda x, y: (1e-7, 0.0), fmt=fmt)
        m1, px1, _ = lat.reduce()
    # 6 steps: mass is kept up to storage rounding; in FP32 the momentum
    # grows by F per node per step.  (With nearest rounding in FP16/BF16 the
    # per-step increments of F = 1e-7 lie below the storage spacing of the
    # deviations, so the growth is not resolved -- the precision limit these
    # formats report; stochastic rounding keeps it on average.)
    assert abs(m1 - m0) <= 64 * U_FMT[fmt] * 1e-2 * m0
    growth = 6 * 1e-7 * n * n
    if fmt == "fp32":
        assert abs((px1 - px0) - growth) <= 1e-3 * growth
    if fmt == "fp16_sr":
        assert abs((px1 - px0) - growth) <= 2e-2 * growth


def test_full_size_obstacles_sampled(clbm):
    """16384 x 8192 channel of 32 x 32 squares on a 64 pitch (25 % solid),
    Fx(y) = 1e-6 (1 + 0.1 sin(2 pi y / ny)), tau = 0.52, FP32."""
    nx, ny = 16384, 8192
    S = O.rates(1.0, 1.0, 1.0, 1.0 / 0.52, 1.0, 1.0)
    solid = inputs.obstacle_mask(nx, ny)
    F = inputs.modulated_force_rows(ny, 1e-6)
    rho = inputs.density_noise(nx, ny, 1e-4, seed=1705)
    with clbm.Lattice(nx, ny, S, fmt="fp32", force_kind=1, force=F, solid=solid) as lat:
        assert lat.fluid_nodes == nx * ny * 3 // 4
        lat.init(rho)
        lat.step(4)
        pts = [(31, 31), (32, 32), (32, 31), (31, 32), (63, 63), (64, 0), (0, 64), (33, 5),
               (5, 33), (nx - 1, ny - 1), (nx - 33, 40), (100, 200), (127, 32), (128, 32)]
        sampled_step_check(lat, S, pts, lambda x, y: (F[y, 0], F[y, 1]), solid=solid)


@pytest.mark.parametrize("fmt", ["fp64", "fp32", "fp16", "bf16"])
def test_launch_shape_does_not_change_results(clbm, fmt):
    """Every launch shape (8- or 16-byte lane vectors, scalar or packed FP32x2
    collision, any prefetch distance, direct or staged loads) runs the same
    operations per node with
    the same rounding: the results are bit-identical (ragged rows, walls,
    obstacles)."""
    nx, ny = 301, 37
    rng = np.random.default_rng(5)
    solid = (rng.random((ny, nx)) < 0.1).astype(np.uint8)
    solid[0, :] = 1
    S = O.rates(1.0, 1.0, 1.1, 1.5, 0.9, 1.0)
    f0 = inputs.random_populations(nx, ny, 0.05, seed=8) * (solid == 0)
    outs = []
    shapes = ((16, 0, 0, 0), (8, 0, 1, 0), (16, 1, 2, 0), (8, 1, 0, 3), (16, 0, 0, 2),
              (16, 1, 0, 3), (8, 0, 0, 2))
    if fmt == "fp64":
        shapes = ((16, 0, 0, 0), (16, 0, 2, 0), (16, 0, 0, 2), (16, 0, 0, 3))
    for shape in shapes:
        with clbm.Lattice(nx, ny, S, fmt=fmt, fx=2e-5, fy=1e-6, solid=solid) as lat:
            lat.tuning = shape
            assert lat.tuning == shape
            lat.set_populations(f0)
            lat.step(45)
            outs.append(lat.get_populations())
    for o in outs[1:]:
        assert np.array_equal(outs[0], o)


@pytest.mark.parametrize("scheme", ["M1", "M2"])
def test_comparison_forcing_schemes_fp64(clbm, scheme):
    """M1 (Eq. 17-19) and M2 (Eq. 21) against the oracle's literal steps."""
    nx, ny, n = 77, 21, 300
    solid = inputs.channel_mask(nx, ny)
    F = inputs.modulated_force_rows(ny, 3e-5, 0.5)
    F[:, 1] = -1e-5
    S = O.rates(1.0, 1.3, 1.1, 1.6, 0.9, 1.2)        # s1 != s2: exercises M2's momentum term
    c_mode = O.FORCING_M1 if scheme == "M1" else O.FORCING_M2
    forcing = clbm.CLBM_FORCING_M1 if scheme == "M1" else clbm.CLBM_FORCING_M2
    f0 = inputs.random_populations(nx, ny, 0.05, seed=31) * (solid == 0)
    ref = O.Lattice(nx, ny, S, F[:, 0][:, None] * np.ones((1, nx)), F[:, 1][:, None] * np.ones((1, nx)),
                    solid=solid, c_mode=c_mode)
    expect = ref.collide(ref.run(f0, n))
    with clbm.Lattice(nx, ny, S, fmt="fp64", force_kind=1, force=F, solid=solid,
                      forcing=forcing) as lat:
        lat.set_populations(f0)
        lat.step(n)
        got = lat.get_populations()
    assert np.abs(got - expect).max() <= 1e-12


@pytest.mark.parametrize("scheme", ["M1", "M2"])
def test_comparison_forcing_schemes_fp32_shapes(clbm, scheme):
    """FP32: within the one-collision bound, identical over launch shapes,
    also after 30 steps (the staged ring of the default shape against the
    direct-load kernels)."""
    nx, ny = 150, 19
    S = O.rates(1.0, 1.0, 1.1, 1.6, 0.9, 1.2)
    c_mode = O.FORCING_M1 if scheme == "M1" else O.FORCING_M2
    forcing = clbm.CLBM_FORCING_M1 if scheme == "M1" else clbm.CLBM_FORCING_M2
    f0 = inputs.random_populations(nx, ny, 0.05, seed=32)
    ref = O.Lattice(nx, ny, S, 2e-5, -1e-5, c_mode=c_mode)
    expect = ref.collide(f0)
    outs, stepped = [], []
    for shape in ((16, 1, 0, 2), (16, 0, 0, 0), (8, 1, 0, 3), (16, 1, 0, 0)):
        with clbm.Lattice(nx, ny, S, fmt="fp32", fx=2e-5, fy=-1e-5, forcing=forcing) as lat:
            lat.tuning = shape
            lat.set_populations(f0)
            outs.append(lat.get_populations())
            lat.step(30)
            stepped.append(lat.get_populations())
    assert np.all(np.abs(outs[0] - expect) <= bound(expect - W, "fp32"))
    for o in outs[1:]:
        assert np.array_equal(outs[0], o)
    for o in stepped[1:]:
        assert np.array_equal(stepped[0], o)


def test_m2_fp64_staged_shape_gives_the_same_bits(clbm):
    """M2 in FP64 on the staged ring (16, 0, 0, 2) and on direct loads: the
    same bits after 30 steps."""
    nx, ny = 150, 19
    S = O.rates(1.0, 1.3, 1.1, 1.3, 0.9, 1.2)
    f0 = inputs.random_populations(nx, ny, 0.05, seed=33)
    outs = []
    for shape in ((16, 0, 0, 0), (16, 0, 0, 2)):
        with clbm.Lattice(nx, ny, S, fmt="fp64", fx=2e-5, fy=-1e-5, forcing=clbm.CLBM_FORCING_M2) as lat:
            lat.tuning = shape
            lat.set_populations(f0)
            lat.step(30)
            outs.append(lat.get_populations())
    assert np.array_equal(outs[0], outs[1])


# ---- sparse tasks (clbm_set_sparse) ------------------------------------------

def _sparse_cases():
    rng = np.random.default_rng(21)
    blocky = (rng.random((37, 301)) < 0.6).astype(np.uint8)
    return [("obstacles", 200, 128, inputs.obstacle_mask(200, 128, 16, 32)),
            ("blocky", 301, 37, blocky)]


@pytest.mark.parametrize("fmt", ["fp64", "fp32", "fp16", "bf16", "fp16_sr", "bf16_sr"])
def test_sparse_tasks_give_the_same_bits(clbm, fmt):
    """The list of vectors holding a fluid node (one per lane) and the
    (row, chunk) tasks run the same per-node operations: same bits, for
    every launch shape (with stochastic rounding too: the random words
    depend on the node and the step only)."""
    S = O.rates(1.0, 1.0, 1.1, 1.4, 1.0, 1.0)
    stochastic = fmt.endswith("_sr")
    fmt = fmt.split("_")[0]
    shapes = ((16, 1, 0, 2), (16, 0, 0, 0), (8, 1, 0, 3)) if fmt != "fp64" else \
        ((16, 0, 0, 0), (16, 0, 0, 2))
    for name, nx, ny, solid in _sparse_cases():
        F = inputs.modulated_force_rows(ny, 3e-5, 0.2)
        f0 = inputs.random_populations(nx, ny, 0.05, seed=31) * (solid == 0)
        outs = []
        for shape in shapes:
            for mode in (clbm.CLBM_SPARSE_OFF, clbm.CLBM_SPARSE_ON):
                with clbm.Lattice(nx, ny, S, fmt=fmt, force_kind=1, force=F, solid=solid) as lat:
                    if stochastic:
                        lat.set_rounding(clbm.CLBM_ROUND_STOCHASTIC)
                    lat.tuning = shape
                    lat.set_sparse(mode)
                    assert (lat.sparse_tasks > 0) == (mode == clbm.CLBM_SPARSE_ON), name
                    lat.set_populations(f0)
                    lat.step(40)
                    outs.append(lat.get_populations())
        for o in outs[1:]:
            assert np.array_equal(outs[0], o), name


def test_sparse_auto_picks_the_list_for_obstacle_arrays(clbm):
    """AUTO: the list for obstacle arrays (a quarter of the vectors all
    solid) in every format; chunk tasks for channels."""
    S = O.rates(1.0, 1.0, 1.0, 1.3, 1.0, 1.0)
    for fmt, expect in (("fp64", True), ("fp16", True), ("bf16", True), ("fp32", True)):
        with clbm.Lattice(256, 128, S, fmt=fmt, solid=inputs.obstacle_mask(256, 128)) as lat:
            assert (lat.sparse_tasks > 0) == expect, fmt
    with clbm.Lattice(256, 129, S, fmt="fp64", solid=inputs.channel_mask(256, 129)) as lat:
        assert lat.sparse_tasks == 0


def test_fp64_sparse_matches_oracle(clbm):
    nx, ny, n = 96, 64, 300
    solid = inputs.obstacle_mask(nx, ny, 16, 32)
    F = inputs.sinusoidal_force_columns(nx, 1e-4)
    F[:, 0] = 3e-5
    S = O.rates(1.0, 1.0, 1.0, 1.4, 1.2, 1.0)
    f0 = inputs.random_populations(nx, ny, 0.05, seed=41) * (solid == 0)
    ref = O.Lattice(nx, ny, S, F[:, 0][None, :] * np.ones((ny, 1)), F[:, 1][None, :] * np.ones((ny, 1)),
                    solid=solid, mode=O.MODE_PRINTED)
    expect = ref.collide(ref.run(f0, n))
    with clbm.Lattice(nx, ny, S, fmt="fp64", force_kind=2, force=F, solid=solid) as lat:
        lat.set_sparse(clbm.CLBM_SPARSE_ON)
        assert lat.sparse_tasks > 0
        lat.set_populations(f0)
        lat.step(n)
        got = lat.get_populations()
    assert np.abs(got - expect).max() <= 1e-12


def _bounce_back_lattice():
    """A wall row, a dense random band (35 % solid) and a band of 8 x 8
    squares on a 16 pitch, over a ragged 203 x 41 lattice."""
    nx, ny = 203, 41
    rng = np.random.default_rng(17)
    solid = np.zeros((ny, nx), dtype=np.uint8)
    solid[0, :] = 1
    solid[13:27, :] = rng.random((14, nx)) < 0.35
    sq = inputs.obstacle_mask(nx, 14, 8, 16)
    solid[27:41, :] = sq
    return nx, ny, solid


@pytest.mark.parametrize("fmt", ["fp64", "fp32", "fp16", "bf16"])
def test_staged_bounce_back_reads(clbm, fmt):
    """Staged shapes fetch the own vectors that halfway bounce-back reads in
    three ways: into the slots of source rows that are all solid (along the
    wall and over the squares), into a per-warp pool (square sides), and,
    for lanes past the end of the pool, from global memory at collision
    time (the dense band gives every lane several links).  All give the
    bits of the direct-load kernel, with row-chunk and sparse tasks, and FP64
    matches the oracle."""
    nx, ny, solid = _bounce_back_lattice()
    S = O.rates(1.0, 1.0, 1.2, 1.4, 1.1, 1.0)
    F = inputs.modulated_force_rows(ny, 2e-5, 0.3)
    f0 = inputs.random_populations(nx, ny, 0.05, seed=19) * (solid == 0)
    shapes = ((16, 0, 0, 0), (16, 1, 0, 2), (8, 1, 0, 3), (16, 0, 0, 2), (8, 0, 0, 2)) \
        if fmt != "fp64" else ((16, 0, 0, 0), (16, 0, 0, 2), (16, 0, 0, 3))
    outs = []
    for shape in shapes:
        for mode in (clbm.CLBM_SPARSE_OFF, clbm.CLBM_SPARSE_ON):
            with clbm.Lattice(nx, ny, S, fmt=fmt, force_kind=1, force=F, solid=solid) as lat:
                lat.tuning = shape
                lat.set_sparse(mode)
                lat.set_populations(f0)
                lat.step(60)
                outs.append(lat.get_populations())
    for o in outs[1:]:
        assert np.array_equal(outs[0], o)
    if fmt == "fp64":
        ref = O.Lattice(nx, ny, S, F[:, 0][:, None] * np.ones((1, nx)), F[:, 1][:, None] * np.ones((1, nx)),
                        solid=solid, mode=O.MODE_PRINTED)
        expect = ref.collide(ref.run(f0, 60))
        assert np.abs(outs[0] - expect).max() <= 1e-12


def test_window_async_reads_each_step_while_the_next_runs(clbm):
    """Enqueued window reads into two page-locked buffers, each waited on by
    an event while the next step runs, give the bits of the synchronous
    read of the same step (a window that wraps in x and y); on the
    library's own stream clbm_synchronize completes them."""
    import torch
    nx, ny = 301, 37
    S = O.rates(1.0, 1.0, 1.1, 1.5, 0.9, 1.0)
    f0 = inputs.random_populations(nx, ny, 0.05, seed=23)
    bufs = [torch.empty((9, 2, 3), dtype=torch.float64).pin_memory().numpy() for _ in range(2)]
    got, expect = [], []
    with clbm.Lattice(nx, ny, S, fmt="fp32", fx=1e-5, stream=clbm.current_stream()) as lat:
        lat.set_populations(f0)
        evs = [torch.cuda.Event(), torch.cuda.Event()]
        for k in range(6):
            lat.step(1)
            lat.window_async(299, 36, bufs[k % 2])
            evs[k % 2].record()
            if k > 0:
                evs[(k - 1) % 2].synchronize()
                got.append(bufs[(k - 1) % 2].copy())
        evs[1].synchronize()
        got.append(bufs[1].copy())
    with clbm.Lattice(nx, ny, S, fmt="fp32", fx=1e-5) as lat:
        lat.set_populations(f0)
        for k in range(6):
            lat.step(1)
            expect.append(lat.window(299, 36, 3, 2))
        own = np.empty((9, 2, 3))
        lat.window_async(299, 36, own)
        lat.synchronize()
    for g, e in zip(got, expect):
        assert np.array_equal(g, e)
    assert np.array_equal(own, expect[-1])


def test_moments_into_page_locked_buffers(clbm):
    """Moments written by the readout kernel straight into mapped
    page-locked host buffers equal the staged copy into pageable ones, for
    any subset of the three outputs."""
    import torch
    nx, ny = 131, 47
    S = O.rates(1.0, 1.0, 1.1, 1.5, 0.9, 1.0)
    solid = inputs.channel_mask(nx, ny)
    f0 = inputs.random_populations(nx, ny, 0.05, seed=29) * (solid == 0)
    with clbm.Lattice(nx, ny, S, fmt="fp32", fx=1e-5, solid=solid) as lat:
        lat.set_populations(f0)
        lat.step(7)
        ref = [np.empty((ny, nx)) for _ in range(3)]
        clbm.clbm_moments(lat.h, *ref)
        pin = [torch.empty((ny, nx), dtype=torch.float64).pin_memory().numpy() for _ in range(3)]
        clbm.clbm_moments(lat.h, *pin)
        for a, b in zip(pin, ref):
            assert np.array_equal(a, b)
        only = torch.full((ny, nx), -1.0, dtype=torch.float64).pin_memory().numpy()
        clbm.clbm_moments(lat.h, None, only, None)
        assert np.array_equal(only, ref[1])


@pytest.mark.parametrize("fmt", ["fp64", "fp32", "fp16", "bf16"])
def test_checkpoint_and_resume(clbm, fmt):
    """A run saved after k steps (clbm_get_populations, post-collision) and
    restored into a fresh lattice as a post-collision state
    (clbm_set_populations with pre_collision = 0: stored, not collided)
    continues like the uninterrupted run, with no host-side streaming.
    FP32, FP16 and BF16 storage resume bit for bit: the decoded state
    re-encodes exactly (FP16 at the same scale exponent).  FP64 storage
    resumes to round-off: decoding adds w_i rho0 in FP64, which rounds the
    stored deviation's last bits (about 5e-17 per population)."""
    nx, ny = 97, 41
    solid = inputs.channel_mask(nx, ny)
    solid[15:19, 30:37] = 1
    S = O.rates(1.0, 1.0, 1.1, 1.4, 1.0, 1.0)
    F = inputs.modulated_force_rows(ny, 2e-5, 0.3)
    f0 = inputs.random_populations(nx, ny, 0.05, seed=37) * (solid == 0)
    with clbm.Lattice(nx, ny, S, fmt=fmt, force_kind=1, force=F, solid=solid) as lat:
        lat.set_populations(f0)
        lat.step(30)
        saved = lat.get_populations()
        k = lat.scale_exponent
        lat.step(20)
        full = lat.get_populations()
    with clbm.Lattice(nx, ny, S, fmt=fmt, force_kind=1, force=F, solid=solid) as lat:
        if fmt == "fp16":
            clbm.clbm_set_scale_exponent(lat.h, k)
        lat.set_populations(saved, pre_collision=False)
        assert np.array_equal(lat.get_populations(), saved) or fmt == "fp64"
        lat.step(20)
        resumed = lat.get_populations()
    if fmt == "fp64":
        assert np.abs(resumed - full).max() <= 1e-15
    else:
        assert np.array_equal(resumed, full)


@pytest.mark.parametrize("fmt", ["fp64", "fp32", "fp16", "bf16"])
def test_pre_collision_read_is_the_pull_of_the_stored_state(clbm, fmt):
    """clbm_get_populations with pre_collision = 1 is the pull-streaming of
    the stored post-collision state with halfway bounce-back (Eq. 10,
    Sec. 4A), without the collision: it equals the oracle's stream of the
    post-collision read, exactly (a permutation of the same decoded
    values), on a ragged lattice with walls, obstacles and a wrap."""
    nx, ny = 203, 41
    _, _, solid = _bounce_back_lattice()
    S = O.rates(1.0, 1.0, 1.2, 1.4, 1.1, 1.0)
    F = inputs.modulated_force_rows(ny, 2e-5, 0.3)
    f0 = inputs.random_populations(nx, ny, 0.05, seed=23) * (solid == 0)
    with clbm.Lattice(nx, ny, S, fmt=fmt, force_kind=1, force=F, solid=solid) as lat:
        lat.set_populations(f0)
        lat.step(7)
        post = lat.get_populations()
        pre = lat.get_populations(pre_collision=True)
    ref = O.Lattice(nx, ny, S, 0.0, 0.0, solid=solid, mode=O.MODE_PRINTED).stream(post)
    assert np.array_equal(pre, ref)


def test_fp64_pre_collision_state_matches_oracle(clbm):
    """The pre-collision state after n steps (the state Eq. 11 and 15 take
    rho and u of) against the oracle's f(t = n), FP64, within 1e-12."""
    nx, ny, n = 96, 64, 200
    solid = inputs.obstacle_mask(nx, ny, 16, 32)
    S = O.rates(1.0, 1.0, 1.0, 1.4, 1.2, 1.0)
    f0 = inputs.random_populations(nx, ny, 0.05, seed=43) * (solid == 0)
    ref = O.Lattice(nx, ny, S, 2e-5, -1e-5, solid=solid, mode=O.MODE_PRINTED)
    expect = ref.run(f0, n)
    with clbm.Lattice(nx, ny, S, fmt="fp64", fx=2e-5, fy=-1e-5, solid=solid) as lat:
        lat.set_populations(f0)
        lat.step(n - 1)
        got = lat.get_populations(pre_collision=True)
    assert np.abs(got - expect).max() <= 1e-12


def test_watchdog_reports_a_non_finite_state(clbm):
    """A NaN in the state makes the FP64 reduction return
    CLBM_ERR_DIVERGED; the error is not sticky, so a finite state set
    afterwards reduces again."""
    nx, ny = 64, 32
    S = O.rates(1.0, 1.0, 1.0, 1.5, 1.0, 1.0)
    f0 = inputs.random_populations(nx, ny, 0.05, seed=41)
    bad = f0.copy()
    bad[3, 5, 7] = np.nan
    with clbm.Lattice(nx, ny, S, fmt="fp32") as lat:
        lat.set_populations(bad)
        lat.step(3)
        with pytest.raises(clbm.ClbmError) as e:
            lat.reduce()
        assert e.value.status == clbm.CLBM_ERR_DIVERGED
        lat.set_populations(f0)
        m, px, py = lat.reduce()
        assert np.isfinite(m) and abs(m - f0.sum()) < 1e-9 * f0.sum()
