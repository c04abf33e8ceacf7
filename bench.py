"""Benchmark: one D2Q9 cascaded-LBM time step with consistent forcing
(Fei & Luo, arXiv:1705.11092) on an 8192 x 8192 periodic lattice.

Workload (one "step" = one fused pull-stream + collide + force launch over
every node): Taylor-Green-like start u = u0 [sin sin, cos cos] with u0 = 0.01
and phi = 2 pi / 8192, rho = 1, uniform force Fx = 1e-7, tau = 0.55 (s2 = 1/tau,
all other rates 1).  Headline: FP32 storage (FP32 compute); the "formats"
block reports FP64, FP32, FP16 and BF16 storage with their velocity error
against the FP64 path after the same number of steps.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Prints one JSON line on rank 0.  For N > 1 (torchrun) every rank runs its own
replica (the step has no cross-replica exchange); value = all ranks' node
updates / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "D2Q9 CLBM MLUPS & % of HBM roofline; low-precision vs FP64 at equal error"
NX = NY = 8192          # overridden by --nx/--ny (profiling captures only)
TAU = 0.55
FX = 1e-7
U0 = 0.01
WORKLOAD = ("8192x8192 periodic D2Q9 CLBM, Taylor-Green-like start u0=0.01, "
            "uniform Fx=1e-7, tau=0.55, other rates 1")
FALLBACK_HBM_GBS = 6800.0
KERNEL_SOURCES = ["paper_1705_11092_gb300/csrc/clbm_step.cuh",
                  "paper_1705_11092_gb300/csrc/clbm_device.cuh"]
TRAFFIC_PROFILE = os.path.join(ROOT, "profiles", "step_kernel_8192.md")
FP64_PROFILE = os.path.join(ROOT, "profiles", "step_kernel_fp64_alu_4096.md")
ALU_PROFILE = os.path.join(ROOT, "profiles", "alu_peaks.md")
# FP64 arithmetic roof derived from unit counts and clocks, used only when no
# measured figure is committed: 152 SMs x 2 FP64 operations per clock per SM
# x 2.07 GHz
FP64_DERIVED_GOPS = 152 * 2 * 2.07


def fp64_peak():
    """FP64 operations per second (G/s) the GPU sustains: the FMA chains
    measured by `bench.py --alu` (profiles/alu_peaks.md; DADD and DMUL run on
    the same FP64 pipe at the same rate), else the derived figure."""
    try:
        t = re.search(r"fp64_fma_gops:\s*([0-9.eE+]+)", open(ALU_PROFILE).read())
        if t:
            return float(t.group(1)), "measured (FP64 FMA chains, profiles/alu_peaks.md)"
    except OSError:
        pass
    return FP64_DERIVED_GOPS, "derived: 152 SMs x 2 FP64 op/clk x 2.07 GHz"


def rates():
    s2 = 1.0 / TAU
    return [1.0, 1.0, 1.0, 1.0, s2, s2, 1.0, 1.0, 1.0]


def kernel_hash() -> str:
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(os.path.join(ROOT, p), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured (copy bandwidth, MEASURED_PEAKS.json)"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def profiled_fp64_ops():
    """FP64 operations (DFMA + DADD + DMUL) per node update of the FP64 step
    kernel, counted by ncu on the current kernel source; else None."""
    try:
        text = open(FP64_PROFILE).read()
    except OSError:
        return None
    m = re.search(r"source_hash:\s*([0-9a-f]+)", text)
    if not m or m.group(1) != kernel_hash():
        return None
    t = re.search(r"fp64_ops_per_node:\s*([0-9.eE+]+)", text)
    return float(t.group(1)) if t else None


def profiled_traffic(fmt: str):
    """DRAM bytes per launch of the step kernel from the committed ncu
    summary, if it was taken on the current kernel source; else None."""
    try:
        text = open(TRAFFIC_PROFILE).read()
    except OSError:
        return None
    m = re.search(r"source_hash:\s*([0-9a-f]+)", text)
    if not m or m.group(1) != kernel_hash():
        return None
    t = re.search(r"traffic_bytes_per_launch_%s:\s*([0-9.eE+]+)" % fmt, text)
    return float(t.group(1)) if t else None


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except OSError:
            pass
        finally:
            try:
                os.unlink(self.path)
            except OSError:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}

        def num(s):
            try:
                return float(s)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        smax = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max((num(r[3]) or 0.0) for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# distributed plumbing (replicas only)
# ---------------------------------------------------------------------------
def dist_setup(n_gpus, backend="nccl"):
    """Rank, world size and local rank from the launcher's environment; one
    process group per job (NCCL on GPUs; gloo carries the same host logic on
    CPU).  Replicas only: the group is used for the barrier and the timing
    maximum, never on the data path."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_mlups(world, nodes_per_rank, steps, seconds):
    """Whole-job throughput of independent replicas: every rank's node
    updates over the slowest rank's time."""
    return world * nodes_per_rank * steps / seconds / 1e6


# ---------------------------------------------------------------------------
# the CPU oracle as a baseline (bounded sample of the same workload)
# ---------------------------------------------------------------------------
def oracle_sample_lattice(side):
    """A side x side window of the workload's initial field (periodic inside
    the window) for the oracle."""
    import numpy as np
    import oracle as O
    from paper_1705_11092_gb300 import inputs
    x = np.arange(side, dtype=np.float64)
    phi = 2 * math.pi / NX
    X, Y = np.meshgrid(x, x)
    ux = U0 * np.sin(phi * X) * np.sin(phi * Y)
    uy = U0 * np.cos(phi * X) * np.cos(phi * Y)
    lat = O.Lattice(side, side, O.rates(1, 1, 1, 1 / TAU, 1, 1), FX, 0.0, mode=O.MODE_PRINTED)
    return lat, lat.equilibrium(1.0, ux, uy)


def oracle_cores():
    import oracle as O
    if not O.has_openmp():
        return 1
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def cpu_baseline(min_seconds=10.0, max_seconds=30.0, side=1024):
    lat, f = oracle_sample_lattice(side)
    lat.run(f, 1)   # warm (and build) once
    t0 = time.perf_counter()
    steps = 0
    while True:
        f = lat.run(f, 1)
        steps += 1
        el = time.perf_counter() - t0
        if el >= min_seconds or el >= max_seconds:
            break
    mlups = side * side * steps / el / 1e6
    return {"value": mlups, "unit": "MLUPS", "cores": oracle_cores(), "kind": "oracle",
            "sample": "%dx%d window of the workload's initial field, %d time steps, FP64 oracle "
                      "(printed-matrix mode), %.1f s" % (side, side, steps, el)}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    total = max(1, args.steps + args.warmup)
    side = int(math.sqrt(2.0e8 / total))
    side = max(32, min(1024, side // 32 * 32))
    lat, f = oracle_sample_lattice(side)
    for _ in range(args.warmup):
        f = lat.run(f, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        f = lat.run(f, 1)
    el = time.perf_counter() - t0
    mlups = side * side * args.steps / el / 1e6
    sample = ("%dx%d window of the workload's initial field per step, FP64 oracle "
              "(printed-matrix mode) on host cores" % (side, side))
    line = {"impl": "reference", "metric": METRIC, "value": mlups, "unit": "MLUPS",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": el / max(1, args.steps) * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": mlups, "unit": "MLUPS", "kind": "oracle",
                             "cores": oracle_cores(), "sample": sample},
            "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def workload_fields():
    import numpy as np
    from paper_1705_11092_gb300 import inputs
    return inputs.taylor_green_velocity(NX, NY, U0)


def make_lattice(clbm, fmt):
    return clbm.Lattice(NX, NY, rates(), fmt=fmt, fx=FX, stream=clbm.current_stream())


def time_steps(lat, clbm, steps, warmup, world):
    import torch
    lat.step(warmup)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    start.record()                     # torch's current stream = the lattice's stream
    lat.step(steps)
    stop.record()
    torch.cuda.synchronize()
    ms = start.elapsed_time(stop)
    barrier(world)
    torch.cuda.synchronize()
    return ms


def velocity_error(u, v, u64, v64):
    import numpy as np
    num = float(np.sum((u - u64) ** 2 + (v - v64) ** 2))
    den = float(np.sum(u64 ** 2 + v64 ** 2))
    return {"rel_l2_u": math.sqrt(num / den), "max_abs_u": float(max(np.abs(u - u64).max(),
                                                                          np.abs(v - v64).max()))}


def format_sweep(clbm, ux, uy, steps, warmup, err_steps, peak):
    """Throughput and roofline of each storage format, and its velocity error
    against the FP64 path after err_steps steps from the same start.  The
    16-bit formats run with nearest and with stochastic rounding ("_sr")."""
    import numpy as np
    out = {}
    ref_u = None
    for key in FORMAT_KEYS:
        fmt = key.split("_")[0]
        with make_lattice(clbm, fmt) as lat:
            if key.endswith("_sr"):
                lat.set_rounding(clbm.CLBM_ROUND_STOCHASTIC)
            lat.init(None, ux, uy)
            ms = time_steps(lat, clbm, steps, warmup, 1)
            per = ms / steps
            b = lat.bytes_per_update
            nodes = lat.fluid_nodes
            gbs = b * nodes / (per * 1e-3) / 1e9
            rec = {"mlups": nodes / (per * 1e-3) / 1e6, "ms_per_step": per,
                   "bytes_per_update": b, "achieved_gbs": gbs, "frac_of_measured_hbm": gbs / peak,
                   "scale_exponent": lat.scale_exponent}
            lat.init(None, ux, uy)
            lat.step(err_steps)
            _, u, v = lat.moments()
            if fmt == "fp64":
                ref_u = (u, v)
                rec.update({"rel_l2_u": 0.0, "max_abs_u": 0.0})
                ops = profiled_fp64_ops()
                if ops is not None:          # bound by the FP64 pipe, not HBM
                    gops = ops * nodes / (per * 1e-3) / 1e9
                    fpk, fkind = fp64_peak()
                    rec["roofline"] = {"bound": "alu", "achieved": gops, "peak": fpk,
                                       "unit": "G FP64 op/s", "frac": gops / fpk,
                                       "ops_per_node": ops, "peak_kind": fkind}
            else:
                rec.update(velocity_error(u, v, *ref_u))
            rec["error_steps"] = err_steps
            rec["error_reference"] = ERROR_REFERENCE
            out[key] = rec
    return out


# storage formats of the format and obstacle blocks ("_sr": stochastic
# rounding of the 16-bit stores, clbm_set_rounding)
FORMAT_KEYS = ("fp64", "fp32", "fp16", "bf16", "fp16_sr", "bf16_sr")

OBSTACLE_NX, OBSTACLE_NY = 16384, 8192
OBSTACLE_TAU = 0.52
OBSTACLE_BOUND = 1e-3          # relative L2 velocity error against the FP64 run


def obstacle_sweep(clbm, time_steps_n, err_steps, peak, nx=OBSTACLE_NX, ny=OBSTACLE_NY,
                   keys=FORMAT_KEYS):
    """The large obstacle flow at fixed accuracy: a 16384 x 8192 periodic
    lattice with 32 x 32 solid squares on a 64 pitch (25 % solid), per-row
    force Fx = 1e-6 (1 + 0.1 sin(2 pi y / ny)), tau = 0.52, rho = 1 + 1e-4
    noise, u = 0.  Each storage format is timed, then run err_steps steps from
    the same start; its velocity error is taken against the FP64 run on the
    fluid nodes, and the fastest format within the error bound is named.
    (Profiling captures pick other sizes and a subset of the formats; without
    FP64 among them no errors are taken.)"""
    import numpy as np
    from paper_1705_11092_gb300 import inputs
    with_errors = "fp64" in keys and err_steps > 0
    keys = sorted(keys, key=lambda k: k != "fp64")       # the FP64 reference first
    solid = inputs.obstacle_mask(nx, ny)
    force = inputs.modulated_force_rows(ny, 1e-6, 0.1)
    rho0 = inputs.density_noise(nx, ny, 1e-4, seed=1705)
    s2 = 1.0 / OBSTACLE_TAU
    r = [1.0, 1.0, 1.0, 1.0, s2, s2, 1.0, 1.0, 1.0]
    fluid = solid == 0
    out = {}
    ref = None
    for key in keys:
        fmt = key.split("_")[0]
        with clbm.Lattice(nx, ny, r, fmt=fmt, force_kind=clbm.CLBM_FORCE_ROWS, force=force,
                          solid=solid, stream=clbm.current_stream()) as lat:
            if key.endswith("_sr"):
                lat.set_rounding(clbm.CLBM_ROUND_STOCHASTIC)
            lat.init(rho0, None, None)
            n = time_steps_n if fmt != "fp64" else max(20, time_steps_n // 10)
            ms = time_steps(lat, clbm, n, 3, 1)
            per = ms / n
            nodes = lat.fluid_nodes
            gbs = lat.bytes_per_update * nodes / (per * 1e-3) / 1e9
            rec = {"mlups": nodes / (per * 1e-3) / 1e6, "ms_per_step": per,
                   "achieved_gbs": gbs, "frac_of_measured_hbm": gbs / peak,
                   "scale_exponent": lat.scale_exponent, "sparse_tasks": lat.sparse_tasks}
            out[key] = rec
            if not with_errors:
                continue
            lat.init(rho0, None, None)
            lat.step(err_steps)
            _, u, v = lat.moments()
            u, v = u[fluid], v[fluid]
            if ref is None:
                ref = (u, v)
                rec.update({"rel_l2_u": 0.0, "max_abs_u": 0.0,
                            "max_speed": float(np.sqrt(u * u + v * v).max())})
            else:
                rec.update(velocity_error(u, v, *ref))
    workload = ("%dx%d periodic, 32x32 squares on a 64 pitch (25%% solid), "
                "Fx = 1e-6 (1 + 0.1 sin(2 pi y/ny)), tau = 0.52, rho = 1 + 1e-4 noise" % (nx, ny))
    if not with_errors:
        return {"workload": workload, "fluid_nodes": int(fluid.sum()), "formats": out}
    ok = [f for f in out if out[f]["rel_l2_u"] <= OBSTACLE_BOUND]
    best = max(ok, key=lambda f: out[f]["mlups"])
    return {"workload": workload,
            "fluid_nodes": int(fluid.sum()), "error_steps": err_steps,
            "error_reference": ERROR_REFERENCE,
            "error_bound_rel_l2_u": OBSTACLE_BOUND, "formats": out,
            "within_bound": ok, "fastest_within_bound": best,
            "speedup_vs_fp64_at_bound": out[best]["mlups"] / out["fp64"]["mlups"]}


ERROR_REFERENCE = "the GPU FP64 path (equal to the FP64 oracle to 1e-12)"


def config2_sweep(clbm, time_steps=500, err_steps=5000, n=1024):
    """The isotropy workload: 1024 x 1024 periodic, F = 1e-5 sin(2 pi y/n) e_x
    and the same force turned by 90 degrees (Fy = 1e-5 sin(2 pi x/n), with
    the transposed initial density), tau = 0.6, rho = 1 + 1e-3 U(-1, 1)
    (seed 1705), u = 0.  FP64 and FP32: MLUPS (the state fits in L2: no HBM
    claim), the transposition residual of the two runs after err_steps steps,
    and the FP32 velocity error against FP64."""
    import numpy as np
    from paper_1705_11092_gb300 import inputs
    s2 = 1.0 / 0.6
    r = [1.0, 1.0, 1.0, 1.0, s2, s2, 1.0, 1.0, 1.0]
    rho = inputs.density_noise(n, n, 1e-3, seed=1705)
    runs = (("x", 1, inputs.sinusoidal_force_rows(n, 1e-5), rho),
            ("y", 2, inputs.sinusoidal_force_columns(n, 1e-5), np.ascontiguousarray(rho.T)))
    out, fields = {}, {}
    for fmt in ("fp64", "fp32"):
        rec = {}
        for name, kind, force, r0 in runs:
            with clbm.Lattice(n, n, r, fmt=fmt, force_kind=kind, force=force,
                              stream=clbm.current_stream()) as lat:
                if name == "x":
                    lat.init(r0)
                    ms = time_steps_on(lat, time_steps, 3)
                    rec["mlups"] = lat.fluid_nodes / (ms * 1e-3) / 1e6
                    rec["ms_per_step"] = ms
                lat.init(r0)
                lat.step(err_steps)
                fields[(fmt, name)] = lat.moments()
        (ra, ua, va), (rb, ub, vb) = fields[(fmt, "x")], fields[(fmt, "y")]
        rec["transpose_residual_u"] = float(max(np.abs(ub.T - va).max(), np.abs(vb.T - ua).max()))
        rec["transpose_residual_rho"] = float(np.abs(rb.T - ra).max())
        rec["max_speed"] = float(np.sqrt(ua * ua + va * va).max())
        out[fmt] = rec
    _, u64, v64 = fields[("fp64", "x")]
    _, u32, v32 = fields[("fp32", "x")]
    out["fp32"].update(velocity_error(u32, v32, u64, v64))
    return {"workload": "1024x1024 periodic, F = 1e-5 sin(2 pi y/1024) e_x and the transposed "
                        "force along y, tau = 0.6, rho = 1 + 1e-3 noise",
            "l2": "state 38 MB (FP32) / 75 MB (FP64) per copy: L2-resident, no HBM claim",
            "time_steps": time_steps, "error_steps": err_steps,
            "error_reference": ERROR_REFERENCE, "formats": out}


# Shan-Chen parameters of Sec. 4C: G, psi0, rho0 of the pseudopotential
# psi = psi0 exp(-rho0 / rho), and the coexistence densities it quotes
SC_G, SC_PSI0, SC_RHO0 = -10.0 / 3.0, 1.0, 1.0
SC_RHO_L, SC_RHO_V = 2.783, 0.3675


def extras_sweep(clbm, peak, n_sc=4096, n_forcing=8192):
    """Throughput of the paper's other forms of the step: Shan-Chen lattices
    (Sec. 4C; a liquid disc of radius n/4 in vapour, two launches per step:
    the psi pass and the step reading psi at the node's neighbours; 27
    population transfers plus a psi write and read per node update) in FP32
    and FP64, and the comparison forcing schemes M1 and M2 (Sec. 3) on the
    8192^2 periodic workload in FP32."""
    import numpy as np
    x = np.arange(n_sc)[None, :]
    y = np.arange(n_sc)[:, None]
    rho0 = np.where((x - n_sc / 2) ** 2 + (y - n_sc / 2) ** 2 <= (n_sc / 4) ** 2, SC_RHO_L, SC_RHO_V)
    out = {}
    for fmt, steps in (("fp32", 200), ("fp64", 20)):
        S = [1.0, 1.0, 1.0, 1.4, 1.4, 1.4, 1.2, 1.2, 1.0]
        with clbm.Lattice(n_sc, n_sc, S, fmt=fmt, force_kind=clbm.CLBM_FORCE_SHAN_CHEN,
                          force=[SC_G, SC_PSI0, SC_RHO0], stream=clbm.current_stream()) as lat:
            lat.init(rho0, None, None)
            ms = time_steps_on(lat, steps, 5)
            out["shan_chen_%s_%d" % (fmt, n_sc)] = {
                "mlups": lat.fluid_nodes / (ms * 1e-3) / 1e6, "ms_per_step": ms,
                "bytes_per_update": lat.bytes_per_update,
                "frac_of_measured_hbm": lat.bytes_per_update * lat.fluid_nodes / (ms * 1e-3) / 1e9 / peak}
    for name, scheme in (("m1", clbm.CLBM_FORCING_M1), ("m2", clbm.CLBM_FORCING_M2)):
        s1 = 1.0 / TAU if scheme == clbm.CLBM_FORCING_M2 else 1.0    # M2 takes s1 = s2
        S = [1.0, s1, s1, 1.0, 1.0 / TAU, 1.0 / TAU, 1.0, 1.0, 1.0]
        with clbm.Lattice(n_forcing, n_forcing, S, fmt="fp32", fx=FX, forcing=scheme,
                          stream=clbm.current_stream()) as lat:
            lat.init()
            ms = time_steps_on(lat, 200, 10)
            out["forcing_%s_fp32_%d" % (name, n_forcing)] = {
                "mlups": lat.fluid_nodes / (ms * 1e-3) / 1e6, "ms_per_step": ms,
                "bytes_per_update": lat.bytes_per_update,
                "frac_of_measured_hbm": lat.bytes_per_update * lat.fluid_nodes / (ms * 1e-3) / 1e9 / peak}
    return out


def time_steps_on(lat, steps, warmup):
    """ms per step of `steps` steps after `warmup`, by CUDA events on torch's
    current stream (the lattice's stream)."""
    import torch
    lat.step(warmup)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    lat.step(steps)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def _sig(x, digits=3):
    """x to `digits` significant digits (None stays None)."""
    if x is None:
        return None
    return float("%.*g" % (digits, x))


def summary(formats, obstacles, batch, config2, extras=None):
    """The measured numbers in a compact form, printed as the JSON line's
    last key so that a reader keeping only the end of the line has them."""
    s = {"key": "[MLUPS, fraction of measured HBM (fp64: of its FP64 ALU roof), relative L2 "
                "u error vs " + ERROR_REFERENCE + "]"}
    if formats:
        f = {}
        for k, v in formats.items():
            frac = v["roofline"]["frac"] if k == "fp64" and "roofline" in v else v["frac_of_measured_hbm"]
            f[k] = [round(v["mlups"]), _sig(frac), _sig(v["rel_l2_u"], 2)]
        s["formats_8192"] = f
    if obstacles:
        o = {}
        for k, v in obstacles["formats"].items():
            o[k] = [round(v["mlups"]), _sig(v["frac_of_measured_hbm"]), _sig(v.get("rel_l2_u"), 2)]
        s["obstacles_16384x8192"] = o
        if "fastest_within_bound" in obstacles:
            s["obstacles_fastest_within_1e-3"] = [obstacles["fastest_within_bound"],
                                                  _sig(obstacles["speedup_vs_fp64_at_bound"])]
    if batch:
        e = batch.get("errors") or {}
        s["batch_256"] = {"mlups": round(batch["mlups"]), "frac": _sig(batch["frac_of_measured_hbm"]),
                          "mode": batch["tuning"] + [batch["mode"]["persistent"], batch["mode"]["resident"],
                                                     batch["mode"]["order"]],
                          "speedup_vs_sequential": _sig(batch["speedup_vs_sequential"]),
                          "e2_median": _sig(e.get("e2_median"), 2),
                          "order_steady": _sig(e.get("order_steady_heights_median"))}
    if config2:
        c = config2["formats"]
        s["config2_1024_l2_resident"] = {
            k: [round(v["mlups"]), _sig(v["transpose_residual_u"], 2), _sig(v.get("rel_l2_u"), 2)]
            for k, v in c.items()}
        s["config2_key"] = "[MLUPS, transpose residual of u after 5000 steps, rel L2 u error]"
    if extras:
        s["extras"] = {k: [round(v["mlups"]), _sig(v["frac_of_measured_hbm"])] for k, v in extras.items()}
    return s


def run_alu(args):
    """The ALU roofs: chains of FP64 FMA, add and multiply, FP32 and packed
    FP32x2 FMA on every SM, each for 2 s, with the SM clock sampled
    meanwhile (operations per second; an FMA is two flops)."""
    import torch
    from paper_1705_11092_gb300 import clbm
    torch.cuda.set_device(0)
    clbm.load()
    out = {}
    for name, kind in (("fp64", clbm.ALU_FP64), ("fp64_add", clbm.ALU_FP64_ADD),
                       ("fp64_mul", clbm.ALU_FP64_MUL), ("fp32", clbm.ALU_FP32),
                       ("fp32x2", clbm.ALU_FP32X2)):
        clbm.clbm_alu_throughput(kind, 0.2)                     # warm
        with ClockSampler(0) as clk:
            ops = clbm.clbm_alu_throughput(kind, 2.0)
        c = clk.summary()
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        per_clk = ops / (sms * c["sm_mhz"] * 1e6) if c.get("sm_mhz") else None
        out[name] = {"gops": ops / 1e9, "sm_mhz": c.get("sm_mhz"),
                     "reasons": c.get("reasons"), "per_clock_per_sm": per_clk}
    print(json.dumps({"alu": out, "sms": torch.cuda.get_device_properties(0).multi_processor_count}),
          flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch
    from paper_1705_11092_gb300 import clbm

    rank, world, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    clbm.load()
    # a dedicated stream: the lattices run on it and the CUDA events that
    # time them are recorded on it
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        return _run_ours(args, clbm, rank, world, local)


def batch_errors(b, sweep, steps):
    """E_2 (Eq. 24) of every channel after `steps` steps from rest against
    the start-up series of the channel (FP64 reduction on the GPU), and the
    convergence order fitted per ladder of heights.  The pre-collision
    velocity after n steps has taken n + 1/2 force impulses, so the series
    is taken at t = n + 1/2.  Heights whose slowest mode has decayed below
    1e-6 by then are 'steady'; for them the error is the halfway-bounce-back
    slip of the two-rate collision, second order in H."""
    import numpy as np
    from paper_1705_11092_gb300 import closed_forms as cf
    for k in range(len(sweep)):
        b.init(k)
    b.step(steps)
    t = steps + 0.5
    e2, steady = [], []
    for k, d in enumerate(sweep):
        nx, ny, H = d["nx"], d["ny"], d["ny"] - 1
        nu = cf.viscosity(1.0 / d["tau"])
        y = np.arange(ny) - 0.5
        row = cf.channel_startup(y, H, d["fx"], nu, t)
        row[0] = 0.0
        ua = np.ascontiguousarray(np.repeat(row[:, None], nx, axis=1))
        e2.append(b.l2_error(k, ua, np.zeros_like(ua)))
        steady.append(math.exp(-(math.pi / H) ** 2 * nu * t) < 1e-6)
    ladders = {}
    for k, d in enumerate(sweep):
        if d["ladder"] >= 0:
            ladders.setdefault(d["ladder"], []).append((d["ny"] - 1, e2[k], steady[k]))
    orders_all, orders_steady = [], []
    for rows in ladders.values():
        orders_all.append(cf.fitted_order([r[0] for r in rows], [r[1] for r in rows]))
        st = [r for r in rows if r[2]]
        if len(st) >= 2:
            orders_steady.append(cf.fitted_order([r[0] for r in st], [r[1] for r in st]))
    return {"steps": steps, "reference": "start-up series of the channel (no slip), t = n + 1/2",
            "e2_min": min(e2), "e2_median": float(np.median(e2)), "e2_max": max(e2),
            "ladders": len(ladders),
            "order_all_heights_median": float(np.median(orders_all)),
            "order_steady_heights_median": float(np.median(orders_steady)) if orders_steady else None,
            "ladders_with_two_steady_heights": len(orders_steady)}


def sequential_runs(clbm, doms, steps=64):
    """The same channels advanced one after another, each as its own
    lattice (clbm_create, CUDA-graph replay of its steps): the baseline the
    batch replaces.  Returns ms per step of all of them."""
    import torch
    lats = [clbm.Lattice(d["nx"], d["ny"], d["rates"], fmt="fp32", fx=d["fx"], solid=d["solid"],
                         stream=clbm.current_stream()) for d in doms]
    try:
        for lat in lats:
            lat.step(steps)               # warm-up and graph capture
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for lat in lats:
            lat.step(steps)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps
    finally:
        for lat in lats:
            lat.close()


def batch_sweep(clbm, steps, peak, fmt="fp32", error_steps=20000, mode=None):
    """The batched resolution/parameter sweep: 256 force-driven channels,
    ny in {17, 33, 65, 129, 257, 513}, nx = 2 ny, tau ~ U[0.55, 1.5],
    Fx ~ log-U[1e-7, 1e-5] (42 ladders + 4 extra), all advanced together; the
    launch shape and mode (one launch per step or persistent launches,
    small lattices in shared memory, lattice order) are picked by the
    library's autotuner."""
    import torch
    from paper_1705_11092_gb300 import inputs
    sweep = inputs.channel_sweep(256)
    doms = [{"nx": d["nx"], "ny": d["ny"],
             "rates": [1.0, 1.0, 1.0, 1.0, 1 / d["tau"], 1 / d["tau"], 1.0, 1.0, 1.0],
             "fx": d["fx"], "solid": inputs.channel_mask(d["nx"], d["ny"])} for d in sweep]
    with clbm.Batch(doms, fmt=fmt, stream=clbm.current_stream()) as b:
        if mode is None:
            tune_ms = b.autotune(32)
        else:                              # a fixed shape and mode (profiling captures)
            tune_ms = None
            b.tuning = (16, 1, 2, 0)
            b.mode = mode
        for k in range(len(doms)):
            b.init(k)
        b.step(4)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        b.step(steps)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        tuning = list(b.tuning)
        used = list(b.mode)
        resident = b.resident_lattices
        gbs = b.bytes_per_step / (ms * 1e-3) / 1e9
        errors = batch_errors(b, sweep, error_steps) if error_steps > 0 else None
        nodes = b.fluid_nodes
    seq_ms = sequential_runs(clbm, doms) if mode is None else None
    return {"workload": "256 channels (ny 17..513, nx = 2 ny), one launch per step over all",
            "storage": fmt, "domains": len(doms), "fluid_nodes": nodes,
            "steps": steps, "ms_per_step": ms,
            "mlups": nodes / (ms * 1e-3) / 1e6, "achieved_gbs": gbs,
            "frac_of_measured_hbm": gbs / peak, "tuning": tuning,
            "mode": {"persistent": used[0], "resident": used[1], "order": used[2],
                     "resident_lattices": resident},
            "bytes": "algorithmic bytes of every lattice every step (HBM-equivalent: lattices held "
                     "in shared memory count as if streamed)",
            "autotune_ms_per_step": tune_ms, "errors": errors,
            "sequential_ms_per_step": seq_ms, "speedup_vs_sequential": seq_ms / ms if seq_ms else None,
            "sequential": "the 256 channels as 256 lattices stepped one after another "
                          "(each with its CUDA-graph replay)"}


def _run_ours(args, clbm, rank, world, local):
    import numpy as np
    import torch
    peak, peak_kind = measured_peak()
    ux, uy = workload_fields()
    fmt = args.format

    with make_lattice(clbm, fmt) as lat:
        lat.init(None, ux, uy)
        nodes = lat.fluid_nodes
        bpu = lat.bytes_per_update
        with ClockSampler(local) as clk:
            ms = time_steps(lat, clbm, args.steps, args.warmup, world)
        clocks = clk.summary()
        ms = max_over_ranks(ms, world)
        mass, px, py = lat.reduce()          # watchdog: raises on NaN/Inf

    per = ms / args.steps
    value = replica_mlups(world, nodes, args.steps, ms * 1e-3)
    achieved = bpu * nodes / (per * 1e-3) / 1e9
    traffic = profiled_traffic(fmt)

    # end to end through the C ABI with pinned host buffers: clbm_init from
    # the host u fields (H2D), then every step clbm_step(1) and a read of the
    # step's result at a monitoring node (clbm_get_window of one node: its 9
    # populations, D2H, synchronising), and clbm_moments of the final field
    # (D2H of rho, u)
    e2e = None
    if not args.no_e2e:
        hux = torch.from_numpy(ux).pin_memory().numpy()
        huy = torch.from_numpy(uy).pin_memory().numpy()
        outs = [torch.empty((NY, NX), dtype=torch.float64).pin_memory().numpy() for _ in range(3)]
        probes = [torch.empty(9, dtype=torch.float64).pin_memory().numpy() for _ in range(2)]
        px, py = NX // 3, NY // 3
        with make_lattice(clbm, fmt) as lat:
            lat.init(None, hux, huy)
            lat.step(args.warmup)
            # warm-up of the host side too: the first GPU write into freshly
            # page-locked memory costs its page mappings (26.6 ms for these
            # 1.6 GB against 8.4 ms afterwards), so each output buffer is
            # written once before the timed region, as the steps are run
            clbm.clbm_moments(lat.h, *outs)
            for pr in probes:
                clbm.clbm_get_window(lat.h, px, py, 1, 1, pr)
            lat.synchronize()
            barrier(world)
            evs = [torch.cuda.Event(), torch.cuda.Event()]   # on the lattice's (torch's) stream
            bad = 0
            t0 = time.perf_counter()
            clbm.clbm_init(lat.h, None, hux, huy)
            t_init = time.perf_counter()
            for k in range(args.steps):
                clbm.clbm_step(lat.h, 1)
                clbm.clbm_get_window_async(lat.h, px, py, 1, 1, probes[k & 1])
                evs[k & 1].record()
                if k:                  # the previous step's read, while this step runs
                    evs[(k - 1) & 1].synchronize()
                    bad += not np.isfinite(probes[(k - 1) & 1]).all()
            evs[(args.steps - 1) & 1].synchronize()
            bad += not np.isfinite(probes[(args.steps - 1) & 1]).all()
            t_steps = time.perf_counter()
            clbm.clbm_moments(lat.h, *outs)
            el = time.perf_counter() - t0
            phases = {"init_ms": (t_init - t0) * 1e3, "steps_ms": (t_steps - t_init) * 1e3,
                      "moments_ms": (t0 + el - t_steps) * 1e3}
            if bad:
                raise FloatingPointError("non-finite populations at the monitoring node")
        el = max_over_ranks(el, world)
        h2d = 2 * 8 * NX * NY
        d2h = 3 * 8 * NX * NY + 9 * 8 * args.steps
        e2e = {"value": replica_mlups(world, nodes, args.steps, el), "unit": "MLUPS",
               "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
               "phases": {k: round(v, 2) for k, v in phases.items()},
               "job": "clbm_init(host u fields) + %d x [clbm_step(1) + clbm_get_window_async(1 node, "
                      "page-locked host); the previous step's read waited on and checked while this "
                      "step runs] + clbm_moments(host)" % args.steps}

    formats = None
    if rank == 0 and world == 1 and not args.no_formats:
        formats = format_sweep(clbm, ux, uy, args.format_steps, 3, args.error_steps, peak)

    batch = None
    if rank == 0 and world == 1 and not args.no_batch:
        mode = tuple(int(v) for v in args.batch_mode.split(",")) if args.batch_mode else None
        batch = batch_sweep(clbm, args.batch_steps, peak, error_steps=args.batch_error_steps, mode=mode)

    config2 = None
    if rank == 0 and world == 1 and not args.no_config2:
        config2 = config2_sweep(clbm)

    extras = None
    if rank == 0 and world == 1 and not args.no_extras:
        extras = extras_sweep(clbm, peak)

    obstacles = None
    if rank == 0 and world == 1 and not args.no_obstacles:
        obstacles = obstacle_sweep(clbm, args.format_steps, args.obstacle_steps, peak,
                                   args.obstacle_nx, args.obstacle_ny, args.obstacle_formats.split(","))

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if fmt == "fp64" else "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "nx": NX, "ny": NY, "storage": fmt,
                       "compute": "f64" if fmt == "fp64" else "f32",
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": "state %.1f GB per buffer >> 129 MB L2 (no flush needed)"
                             % (9 * NX * NY * {"fp64": 8, "fp32": 4}.get(fmt, 2) / 1e9)},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "bytes_per_update": bpu, "peak_kind": peak_kind,
                         "kernel": "step_kernel (fused pull-stream + collide + force)"},
            "e2e": e2e,
            "gpu_launches": args.steps,
            "clocks": clocks,
            "cpu_baseline": cpu,
            "mass": mass,
            "formats": formats,
            "batch": batch,
            "obstacles": obstacles,
            "config2": config2,
            "extras": extras,
            "summary": summary(formats, obstacles, batch, config2, extras),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def make_parser():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--format", default="fp32", choices=["fp64", "fp32", "fp16", "bf16"])
    ap.add_argument("--format-steps", type=int, default=200)
    ap.add_argument("--error-steps", type=int, default=1000)
    ap.add_argument("--no-formats", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-obstacles", action="store_true")
    ap.add_argument("--no-config2", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the Shan-Chen and M1/M2 throughput block")
    ap.add_argument("--alu", action="store_true", help="measure the FP64/FP32 FMA roofs and exit")
    ap.add_argument("--obstacle-steps", type=int, default=2000)
    ap.add_argument("--obstacle-nx", type=int, default=OBSTACLE_NX, help="(profiling captures)")
    ap.add_argument("--obstacle-ny", type=int, default=OBSTACLE_NY)
    ap.add_argument("--obstacle-formats", default=",".join(FORMAT_KEYS),
                    help="comma-separated subset of " + ",".join(FORMAT_KEYS))
    ap.add_argument("--batch-steps", type=int, default=400)
    ap.add_argument("--batch-error-steps", type=int, default=20000)
    ap.add_argument("--batch-mode", default="", help="persistent,resident,order instead of the autotuner "
                                                     "(profiling captures)")
    ap.add_argument("--nx", type=int, default=8192, help="lattice size (profiling captures)")
    ap.add_argument("--ny", type=int, default=8192)
    return ap


def main():
    ap = make_parser()
    args = ap.parse_args()
    global NX, NY
    NX, NY = args.nx, args.ny
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.alu:
        return run_alu(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
