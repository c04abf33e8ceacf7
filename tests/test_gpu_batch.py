"""Batched lattices (clbm_batch_*): a lattice advanced inside a batch gives
exactly the result of the same lattice run alone (same kernel code, same
rounding, so bit for bit), FP64 batches match the oracle to 1e-12, and the
autotuner only changes the launch shape."""
import math

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


def mixed_domains():
    """Uneven sizes, rates, forces; walls, obstacles and fully periodic."""
    rng = np.random.default_rng(11)
    doms = []
    # channels of the sweep's smallest heights
    for ny in (17, 33, 65):
        s2 = 1.0 / (0.55 + 0.5 * rng.random())
        doms.append({"nx": 2 * ny, "ny": ny, "rates": O.rates(1, 1, 1, s2, 1, 1),
                     "fx": 1e-5 * rng.random(), "solid": inputs.channel_mask(2 * ny, ny)})
    # periodic with row force, ragged width
    F = inputs.sinusoidal_force_rows(23, 1e-5)
    doms.append({"nx": 301, "ny": 23, "rates": O.rates(1, 1, 1.2, 1.6, 0.9, 1.1),
                 "force_kind": 1, "force": F})
    # obstacles
    sol = (rng.random((40, 77)) < 0.15).astype(np.uint8)
    doms.append({"nx": 77, "ny": 40, "rates": O.rates(1, 1, 1, 1.8, 1.2, 1), "fx": 2e-5,
                 "fy": -1e-6, "solid": sol})
    # tiny
    doms.append({"nx": 3, "ny": 5, "rates": O.rates(1, 1, 1, 1.3, 1.0, 1), "fx": 1e-4})
    # per-column and per-node forces on widths whose ragged row ends are
    # packed several rows to a warp task (and one that is not)
    doms.append({"nx": 150, "ny": 37, "rates": O.rates(1, 1, 1, 1.4, 1.1, 1),
                 "force_kind": 2, "force": inputs.sinusoidal_force_columns(150, 1e-5)})
    Fxy = np.stack(inputs.taylor_green_velocity(40, 29, 1e-5), axis=-1)
    doms.append({"nx": 40, "ny": 29, "rates": O.rates(1, 1, 1, 1.5, 1.0, 1),
                 "force_kind": 3, "force": Fxy,
                 "solid": (rng.random((29, 40)) < 0.1).astype(np.uint8)})
    # the comparison forcing schemes M1 and M2 (Sec. 3)
    doms.append({"nx": 64, "ny": 33, "rates": O.rates(1, 1, 1, 1.25, 1.3, 1), "fx": 1e-5,
                 "solid": inputs.channel_mask(64, 33), "forcing": 1})
    doms.append({"nx": 64, "ny": 33, "rates": O.rates(1, 1.25, 1, 1.25, 1.3, 1), "fx": 1e-5,
                 "fy": 2e-6, "solid": inputs.channel_mask(64, 33), "forcing": 2})
    return doms


def init_fields(d, k):
    nx, ny = d["nx"], d["ny"]
    rho = inputs.density_noise(nx, ny, 1e-3, seed=100 + k)
    ux, uy = inputs.taylor_green_velocity(nx, ny, 0.01)
    return rho, ux, uy


@pytest.mark.parametrize("fmt", ["fp64", "fp32", "fp16", "bf16"])
def test_batch_equals_single_runs(clbm, fmt):
    doms = mixed_domains()
    n = 45
    with clbm.Batch(doms, fmt=fmt) as b:
        for k, d in enumerate(doms):
            b.init(k, *init_fields(d, k))
        b.step(n)
        got = [b.get_populations(k) for k in range(len(doms))]
        red = [b.reduce(k) for k in range(len(doms))]
    for k, d in enumerate(doms):
        with clbm.Lattice(d["nx"], d["ny"], d["rates"], fmt=fmt, fx=d.get("fx", 0.0),
                          fy=d.get("fy", 0.0), force_kind=d.get("force_kind", 0),
                          force=d.get("force"), solid=d.get("solid"),
                          forcing=d.get("forcing", 0)) as lat:
            lat.init(*init_fields(d, k))
            lat.step(n)
            ref = lat.get_populations()
            assert lat.reduce() == red[k]
        assert np.array_equal(got[k], ref), k


def test_fp64_batch_matches_oracle(clbm):
    doms = mixed_domains()
    n = 200
    with clbm.Batch(doms, fmt="fp64") as b:
        f0s = []
        for k, d in enumerate(doms):
            f0 = inputs.random_populations(d["nx"], d["ny"], 0.05, seed=k + 1)
            if d.get("solid") is not None:
                f0 = f0 * (d["solid"] == 0)
            f0s.append(f0)
            b.set_populations(k, f0)
        b.step(n)
        for k, d in enumerate(doms):
            kind = d.get("force_kind", 0)
            if kind == 1:      # per row [ny][2]
                fx = d["force"][:, 0][:, None] * np.ones((1, d["nx"]))
                fy = d["force"][:, 1][:, None] * np.ones((1, d["nx"]))
            elif kind == 2:    # per column [nx][2]
                fx = np.ones((d["ny"], 1)) * d["force"][:, 0][None, :]
                fy = np.ones((d["ny"], 1)) * d["force"][:, 1][None, :]
            elif kind == 3:    # per node [ny][nx][2]
                fx, fy = d["force"][..., 0], d["force"][..., 1]
            else:
                fx, fy = d.get("fx", 0.0), d.get("fy", 0.0)
            c_mode = {0: O.C_DERIVED, 1: O.FORCING_M1, 2: O.FORCING_M2}[d.get("forcing", 0)]
            ref = O.Lattice(d["nx"], d["ny"], d["rates"], fx, fy, solid=d.get("solid"),
                            mode=O.MODE_PRINTED, c_mode=c_mode)
            expect = ref.collide(ref.run(f0s[k], n))
            assert np.abs(b.get_populations(k) - expect).max() <= 1e-12, k


def test_autotune_changes_only_the_launch_shape(clbm):
    doms = mixed_domains()
    outs = []
    for tune in (False, True):
        with clbm.Batch(doms, fmt="fp32") as b:
            if tune:
                ms = b.autotune(5)
                assert ms > 0
                assert b.tuning in [(v, p, st, sc) for v in (16, 8) for p in (0, 1)
                                    for st in (0, 2, 3) for sc in (0, 1)]
            for k, d in enumerate(doms):
                b.init(k, *init_fields(d, k))
            b.step(70)        # two graph replays + 6 launches
            outs.append([b.get_populations(k) for k in range(len(doms))])
    for a, c in zip(*outs):
        assert np.array_equal(a, c)


def test_channel_sweep_batch_runs(clbm):
    """The 256-channel sweep recipe (FP32): every lattice stays finite and
    conserves mass; each moves by F per fluid node per step."""
    sweep = inputs.channel_sweep(256)
    doms = [{"nx": d["nx"], "ny": d["ny"], "rates": O.rates(1, 1, 1, 1 / d["tau"], 1, 1),
             "fx": d["fx"], "solid": inputs.channel_mask(d["nx"], d["ny"])} for d in sweep]
    with clbm.Batch(doms, fmt="fp32") as b:
        assert b.fluid_nodes == sum(d["nx"] * (d["ny"] - 1) for d in sweep)
        before = [b.reduce(k) for k in range(0, 256, 17)]
        b.step(100)
        after = [b.reduce(k) for k in range(0, 256, 17)]
    for j, k in enumerate(range(0, 256, 17)):
        d = sweep[k]
        nf = d["nx"] * (d["ny"] - 1)
        assert abs(after[j][0] - before[j][0]) <= 1e-5 * before[j][0]
        grow = 100 * d["fx"] * nf
        # walls take momentum out: growth is at most F per node per step
        assert -1e-6 * nf <= after[j][1] - before[j][1] <= grow * (1 + 1e-3) + 1e-6 * nf


@pytest.mark.parametrize("fmt", ["fp32", "fp16", "fp64"])
def test_batch_launch_shapes_bit_identical(clbm, fmt):
    doms = mixed_domains()
    shapes = [(16, 0, 0, 1), (16, 1, 2, 1), (8, 1, 3, 1), (8, 0, 2, 0), (16, 1, 0, 0),
              (16, 1, 2, 0), (16, 0, 0, 0)]
    if fmt == "fp64":
        shapes = [(16, 0, 0, 1), (16, 0, 2, 1), (16, 0, 3, 0), (16, 0, 0, 0)]
    outs = []
    for sh in shapes:
        with clbm.Batch(doms, fmt=fmt) as b:
            b.tuning = sh
            assert b.tuning == sh
            for k, d in enumerate(doms):
                b.init(k, *init_fields(d, k))
            b.step(37)
            outs.append([b.get_populations(k) for k in range(len(doms))])
    for o in outs[1:]:
        for a, c in zip(outs[0], o):
            assert np.array_equal(a, c)


def test_channel_sweep_errors_after_20000_steps(clbm):
    """The channels of four ladders of the sweep that reach steady state by
    step 20000 (H = 16, 32), in FP64.  Such a channel holds the parabola
    shifted by the two-rate halfway-bounce-back slip
    F (16 Lambda - 3) / (24 rho nu) (s3 = 1 here, off the non-slip rule), so
    its E_2 against the no-slip profile is that slip over the profile's norm,
    and the heights converge at second order.  (FP32 cannot hold slips of
    1e-8 to 1e-7 against its rounding over a relaxation time, so this check
    uses FP64.)"""
    from paper_1705_11092_gb300 import closed_forms as C
    sweep = [d for d in inputs.channel_sweep(256) if d["ladder"] in (0, 1, 2, 3) and d["ny"] <= 33]
    doms = [{"nx": d["nx"], "ny": d["ny"], "rates": O.rates(1, 1, 1, 1 / d["tau"], 1, 1),
             "fx": d["fx"], "solid": inputs.channel_mask(d["nx"], d["ny"])} for d in sweep]
    n = 20000
    t = n + 0.5
    with clbm.Batch(doms, fmt="fp64") as b:
        b.step(n)
        rows = []
        for k, d in enumerate(sweep):
            H, nu, s2 = d["ny"] - 1, C.viscosity(1 / d["tau"]), 1 / d["tau"]
            y = np.arange(d["ny"]) - 0.5
            ref = C.channel_startup(y, H, d["fx"], nu, t)
            ref[0] = 0.0
            ua = np.ascontiguousarray(np.repeat(ref[:, None], d["nx"], axis=1))
            e2 = b.l2_error(k, ua, np.zeros_like(ua))
            if math.exp(-(math.pi / H) ** 2 * nu * t) < 1e-6:
                slip = C.halfway_slip(d["fx"], nu, s2, 1.0)
                pred = abs(slip) * math.sqrt(H) / math.sqrt(np.sum(ref[1:] ** 2))
                assert e2 == pytest.approx(pred, rel=1e-3), (d["ny"], e2, pred)
                rows.append((d["ladder"], H, e2))
    for lad in (0, 1, 2, 3):
        st = [(H, e) for L, H, e in rows if L == lad]
        assert len(st) >= 2
        assert 1.9 < C.fitted_order([h for h, _ in st], [e for _, e in st]) < 2.1


# ---- persistent launches (clbm_batch_set_mode) -------------------------------

def _persistent_domains():
    """mixed_domains without the M2 lattice (persistent launches take the
    staged kernels, which M2 lattices do not run)."""
    return [d for d in mixed_domains() if d.get("forcing", 0) != 2]


@pytest.mark.parametrize("fmt", ["fp64", "fp32", "fp16", "bf16"])
def test_persistent_launches_give_the_same_bits(clbm, fmt):
    """A batch advanced by persistent launches (per-lattice waits between
    steps), with and without the smallest lattices held in shared memory,
    and with the largest-first order, equals the batch advanced one launch
    per step, bit for bit; 70 steps cover two graph replays of 32 steps and
    a persistent launch of the remaining 6."""
    doms = _persistent_domains()
    n = 70
    packed = 0 if fmt == "fp64" else 1
    runs = [((16, packed, 2, 0), (0, 0, 0)), ((16, packed, 2, 0), (1, 0, 0)),
            ((16, packed, 2, 0), (1, 1, 0)), ((16, packed, 3, 0), (1, 1, 1)),
            ((16, packed, 3, 0), (1, 0, 1))]
    outs = []
    for tuning, mode in runs:
        with clbm.Batch(doms, fmt=fmt) as b:
            b.tuning = tuning
            b.mode = mode
            assert b.mode == mode
            if mode[1]:
                assert b.resident_lattices >= 1
            for k, d in enumerate(doms):
                b.init(k, *init_fields(d, k))
            b.step(n)
            b.synchronize()
            outs.append([b.get_populations(k) for k in range(len(doms))])
    for o in outs[1:]:
        for k in range(len(doms)):
            assert np.array_equal(o[k], outs[0][k]), k


def _walled_domains():
    """Every lattice with solid nodes (the batch's all-masked form): channels
    of three heights, a lattice whose solids sit in two bands (plain rows
    between them and at the ends), and one with solids in every row (no
    rows of plain vectors)."""
    rng = np.random.default_rng(23)
    doms = []
    for ny in (17, 33, 65):
        doms.append({"nx": 2 * ny, "ny": ny, "rates": O.rates(1, 1, 1, 1.5, 1, 1),
                     "fx": 1e-5 * (1 + rng.random()), "solid": inputs.channel_mask(2 * ny, ny)})
    band = np.zeros((60, 90), dtype=np.uint8)
    band[20:24, :] = rng.random((4, 90)) < 0.3
    band[41:43, 10:30] = 1
    doms.append({"nx": 90, "ny": 60, "rates": O.rates(1, 1, 1.1, 1.4, 1.2, 1), "fx": 2e-5, "fy": 1e-6,
                 "solid": band})
    every = (rng.random((21, 47)) < 0.2).astype(np.uint8)
    every[:, 5] = 1
    doms.append({"nx": 47, "ny": 21, "rates": O.rates(1, 1, 1, 1.6, 1, 1), "fx": 1e-5, "solid": every})
    return doms


@pytest.mark.parametrize("fmt", ["fp32", "fp16"])
def test_persistent_rows_of_plain_vectors_give_the_same_bits(clbm, fmt):
    """With every lattice walled, persistent launches step the tasks inside
    each lattice's rows of plain vectors without masks and the rest with
    them; the result equals one launch per step (masked path for all
    tasks), bit for bit, with and without lattices held in shared memory."""
    doms = _walled_domains()
    runs = [((16, 1, 2, 0), (0, 0, 0)), ((16, 1, 2, 0), (1, 0, 0)), ((16, 1, 2, 0), (1, 1, 0))]
    outs = []
    for tuning, mode in runs:
        with clbm.Batch(doms, fmt=fmt) as b:
            b.tuning = tuning
            b.mode = mode
            for k, d in enumerate(doms):
                b.init(k, *init_fields(d, k))
            b.step(45)
            b.synchronize()
            outs.append([b.get_populations(k) for k in range(len(doms))])
    for o in outs[1:]:
        for k in range(len(doms)):
            assert np.array_equal(o[k], outs[0][k]), k


def test_persistent_mode_checks(clbm):
    doms = _persistent_domains()
    with clbm.Batch(doms, fmt="fp32") as b:
        b.tuning = (16, 1, 0, 0)
        with pytest.raises(clbm.ClbmError):
            b.mode = (1, 0, 0)                      # persistent needs a staged shape
        b.tuning = (16, 1, 2, 0)
        with pytest.raises(clbm.ClbmError):
            b.mode = (0, 1, 0)                      # resident needs persistent
        b.mode = (1, 0, 0)
        with pytest.raises(clbm.ClbmError):
            b.tuning = (16, 1, 0, 0)                # and keeps it staged
    with clbm.Batch(mixed_domains(), fmt="fp32") as b:
        b.tuning = (16, 1, 2, 0)
        with pytest.raises(clbm.ClbmError):
            b.mode = (1, 0, 0)                      # an M2 lattice


def test_persistent_wait_gives_up_with_a_status(clbm):
    """A persistent launch whose first warp starts 2 ms late, with waits
    that poll once: the warps that share its lattice give up, the launch
    ends, and the next synchronising call returns CLBM_ERR_TIMEOUT; the
    batch is then sticky.  Nothing hangs or faults: every wait is bounded
    and a warp that gives up returns.  A new batch runs normally after."""
    big = {"nx": 512, "ny": 257, "rates": O.rates(1, 1, 1, 1.6, 1, 1), "fx": 1e-5,
           "solid": inputs.channel_mask(512, 257)}
    small = {"nx": 66, "ny": 33, "rates": O.rates(1, 1, 1, 1.2, 1, 1), "fx": 2e-6,
             "solid": inputs.channel_mask(66, 33)}
    b = clbm.Batch([big, small], fmt="fp32")
    try:
        b.tuning = (16, 1, 2, 0)
        b.mode = (1, 0, 0)
        b.step(3)
        b.synchronize()                             # the normal bound: no timeout
        b.set_wait(1, 2_000_000)
        b.step(4)
        with pytest.raises(clbm.ClbmError) as e:
            b.synchronize()
        assert e.value.status == clbm.CLBM_ERR_TIMEOUT
        with pytest.raises(clbm.ClbmError) as e:
            b.step(1)
        assert e.value.status == clbm.CLBM_ERR_STATE
    finally:
        assert clbm.clbm_batch_destroy(b.h) == clbm.CLBM_OK
        b.h = None
    with clbm.Batch([big, small], fmt="fp32") as b2:
        b2.tuning = (16, 1, 2, 0)
        b2.mode = (1, 0, 0)
        b2.step(40)
        b2.synchronize()
        assert np.isfinite(b2.reduce(0)[0])


def test_autotune_remembers_across_processes(clbm, tmp_path):
    """The autotuner writes its pick to the cache file; another process
    with the same GPU, format and lattice shapes applies it without timing."""
    import json
    import os
    import subprocess
    import sys
    path = tmp_path / "tune.txt"
    os.environ["CLBM_TUNE_CACHE"] = str(path)
    try:
        doms = _persistent_domains()[:4]
        with clbm.Batch(doms, fmt="fp32") as b:
            b.autotune(4)
            picked = list(b.tuning) + list(b.mode)
        lines = path.read_text().splitlines()
        assert len(lines) == 1 and len(lines[0].split()) == 8
        assert [int(v) for v in lines[0].split()[1:]] == picked[:4] + picked[4:]
        code = (
            "import sys, json; sys.path.insert(0, %r)\n"
            "from tests.test_gpu_batch import _persistent_domains\n"
            "from paper_1705_11092_gb300 import clbm\n"
            "clbm.load()\n"
            "b = clbm.Batch(_persistent_domains()[:4], fmt='fp32')\n"
            "b.autotune(4, timed=False)\n"
            "print(json.dumps(list(b.tuning) + list(b.mode)))\n" % os.getcwd())
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                           env=dict(os.environ), timeout=300)
        assert r.returncode == 0, r.stderr
        assert json.loads(r.stdout.strip().splitlines()[-1]) == picked
    finally:
        del os.environ["CLBM_TUNE_CACHE"]
