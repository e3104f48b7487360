#!/usr/bin/env python3
"""Benchmark of the fractional-step IB solver at 512 x 256 x 256.

One "step" is one full time step of the method (Sec. II.B order: RHS, three
implicit factors, IB interpolation/spreading, flag sub-steps, mass fix,
Poisson solve, projection) of the production workload: 512 x 256 x 256
cells, domain 8 x 4 x 4, Re = 200, bar grid (mesh 0.5, width 0.1) at x = 0.5,
65 x 65 flag hinged at x = 3, CFL 0.3, seeded synthetic initial noise.

Output: one JSON line (rank 0). `value` is steps/s of the mixed-precision
path (FP32 fields; Poisson transforms as split-TF32 tensor-core GEMMs with a
refinement sweep on a double-single residual; FP64 flag and global sums)
summed over all ranks; each rank runs an independent replica (the path is
not sharded). Beside it: the FP64 path (the other half of the metric's
pair) and the FP32 path, each with its own clock record; the roofline of
every kernel of the step and of the dominant one; the end-to-end rate
through the C ABI with host buffers; the CPU oracle on one core and on all
host cores (bounded samples).

--impl reference times the CPU oracle (the reference arm of this repository)
on the same metric, on all host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "fractional steps/s & Gcell-updates/s at 512x256x256, mixed vs FP64, % HBM peak"
FALLBACK_HBM_GBS = 6800.0
FALLBACK_BF16_TFLOPS = 1900.0

# Algorithmic bytes per launch of each kernel of the step, in units of one
# scalar field (one read or one write of every cell): the inputs it must read
# and the outputs it must write, with perfect on-chip reuse inside the kernel.
# Velocity-grid kernels count (nx + 1) ny nz cells, pressure-grid kernels
# (transforms, x solves, residual) nx ny nz.
# Bfloat16 stages count half a pass per bfloat16 field: the mixed solve's
# correction transform (tc_bf16, read and write) and Thomas solve
# (poisson_x16), and the residual's bfloat16 output.
FIELD_PASSES = {
    "rhs": 13, "af_x": 6, "af_yz": 9, "mass_div": 4,
    "dht2d": 2, "poisson_x": 3, "project": 9, "tc_pass": 2, "tc_pass1": 2, "residual": 2.5,
    "tc_bf16": 1, "poisson_x16": 1.5,
}
PRESSURE_GRID = ("dht2d", "poisson_x", "tc_pass", "tc_pass1", "residual", "tc_bf16", "poisson_x16")
# launches of each stage per step
PER_STEP = {
    "fp32": {"rhs": 1, "outflow": 1, "af_x": 1, "af_yz": 1, "ib": 1, "flag": 1, "mass_div": 1,
             "dht2d": 2, "poisson_x": 1, "project": 1},
    "mixed": {"rhs": 1, "outflow": 1, "af_x": 1, "af_yz": 1, "ib": 1, "flag": 1, "mass_div": 1,
              "dht2d": 2, "poisson_x": 1, "residual": 1, "tc_bf16": 4, "poisson_x16": 1, "project": 1},
}
# The method's unfused field passes per step (explicit stage 13, three
# implicit factors 21, mass fix and divergence 4, pressure solve 10,
# projection 9): the step's roofline counts these bytes whatever the fusion.
# The mixed path adds its refinement at the storage it uses: the residual
# (two FP32 reads, a bfloat16 write: 2.5), the bfloat16 correction solve (10
# bfloat16 passes: 5) and the projection's read of the correction (0.5).
METHOD_PASSES = {"fp32": 57, "mixed": 65}
# DRAM bytes per launch of a stage (dram__bytes_read.sum +
# dram__bytes_write.sum, both launches for "ib") from single-pass ncu
# captures of every launch of the production FP32 and mixed steps
# (profiles/launches_production_fp32.md, launches_production_mixed.md);
# valid for the kernels of those captures and to be refreshed whenever one
# of them changes.
_TRAFFIC_COMMON = {"rhs": 1743.1e6, "af_yz": 1156.6e6, "af_x": 752.3e6, "mass_div": 519.2e6,
                   "poisson_x": 218.4e6, "ib": 57.9e6}
TRAFFIC_BYTES = {
    "fp32": dict(_TRAFFIC_COMMON, dht2d=209.9e6, project=1181.3e6),
    "mixed": dict(_TRAFFIC_COMMON, dht2d=212.3e6, tc_bf16=84.6e6, residual=317.6e6, poisson_x16=78.2e6,
                  project=1258.4e6),
}
# the mixed path's projection reads the solve's two parts (FP32 predictor,
# bfloat16 correction): half a pass more than FIELD_PASSES["project"]
MIXED_PASSES = {"project": 9.5}
# FP64 path: the explicit stage's FP64 instructions per cell (DFMA + DMUL +
# DADD, from an ncu count of k_rhs_vec<double>) and the FP64 issue rate of
# GB300 (2 per clock per SM): the FP64 step is bound by that pipe.
FP64_RHS_INST_PER_CELL = 86.2
# DRAM bytes of one residual-block convolution of the generator (8 x 256 x 256
# pixels, 128 -> 128 channels) from an ncu capture of the current kernel
GEN_CONV_TRAFFIC_BYTES = 757.4e6
FP64_INST_PER_CLK_SM = 2
N_SMS = 152
CLOCK_WINDOW_S = 0.6   # each leg's clock record spans at least this long
SAMPLE_NX = 64   # x planes of the CPU sample (the inflow end of the workload)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true",
                    help="skip the FP64, FP32, ensemble and generator legs")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--profile-steps", type=int, default=0,
                    help="only run this many FP32 production steps (for ncu) and exit")
    ap.add_argument("--profile-precision", choices=["fp32", "fp64", "mixed"], default="fp32")
    ap.add_argument("--profile-small", action="store_true",
                    help="profile the 256x256x256 half-length case (flag at x = 2)")
    ap.add_argument("--profile-generator", type=int, default=0,
                    help="only run this many launches of each generator kernel timing "
                         "(residual-block convolution, input gradient, weight gradient; "
                         "256x256 planes, batch 8) for ncu and exit")
    ap.add_argument("--profile-generator-train", type=int, default=0,
                    help="only run this many generator training steps (256x256 planes, "
                         "batch 8, 13 blocks) after one warm step, for ncu, and exit")
    ap.add_argument("--profile-slabs", type=int, default=0,
                    help="only run this many FP64 steps of the 256x256x256 half-length case in four "
                         "x slabs (all on this GPU, after the initial projection), for ncu, and exit")
    return ap.parse_args()


def run_profile(args):
    """Plain run for profilers: create the production state and step it."""
    import torch
    from paper_2103_08246_gb300 import binding, build, inputs
    build.build()
    wl = inputs.PRODUCTION
    if args.profile_small:
        wl = wl.replace(name="half-256x256x256", nx=256, lx=4.0, flag_x_le=2.0)
    prec = {"fp32": binding.IBM_FP32, "fp64": binding.IBM_FP64,
            "mixed": binding.IBM_MIXED}[args.profile_precision]
    s = binding.Solver(wl, prec, noise=inputs.initial_noise(wl))
    s.step(args.profile_steps)
    torch.cuda.synchronize()
    s.close()


def run_profile_slabs(args):
    """Plain run for profilers: the half-length production case (256 x-planes,
    bars and flag, fixed dt 2e-3) decomposed into four x slabs on this GPU."""
    import torch
    from paper_2103_08246_gb300 import build, inputs
    from paper_2103_08246_gb300 import slab as S
    build.build()
    wl = inputs.PRODUCTION.replace(name="half-256x256x256", nx=256, lx=4.0, flag_x_le=2.0, dt=2e-3)
    ranks = S.make_ranks(wl, 4, wl.dt, inputs.initial_noise(wl))
    comm = S.LoopbackComm()
    S.run_phases(ranks, comm, S.INIT_SEQUENCE)
    for _ in range(args.profile_slabs):
        S.run_phases(ranks, comm, S.STEP_SEQUENCE, wl.dt)
    torch.cuda.synchronize()
    for r in ranks:
        r.close()


def run_profile_generator(args):
    """Plain run for profilers: one residual block of the inflow generator at
    the production plane; each kernel timed once warm plus n times."""
    from paper_2103_08246_gb300 import binding, build, inputs
    build.build()
    g = binding.Generator(256, 256, blocks=1, in_channels=6, batch=8)
    g.set_params(inputs.generator_params(0, 128, 1, 6))
    for what in ("conv_fwd", "conv_dgrad", "conv_wgrad"):
        print(what, "ms", g.time(what, args.profile_generator))
    g.close()


def run_profile_generator_train(args):
    """Plain run for profilers: training steps of the production-size generator."""
    from paper_2103_08246_gb300 import binding, build, inputs
    build.build()
    g = binding.Generator(256, 256, blocks=13, in_channels=6, batch=8)
    g.set_params(inputs.generator_params(0, 128, 13, 6))
    print("train_step ms", g.time("train_step", args.profile_generator_train))
    g.close()


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            if d.get("hbm_gbs"):
                return float(d["hbm_gbs"]), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


def measured_bf16_peak():
    """Dense bf16 TFLOP/s: the measured burst figure (a kernel timed alone)."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            if d.get("bf16_tflops"):
                return float(d["bf16_tflops"]), "measured bf16 burst"
        except Exception:
            pass
    return FALLBACK_BF16_TFLOPS, "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ distributed
def dist_setup(n):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if _cuda_ok() else "gloo"
        dist.init_process_group(backend)
        pg = dist
    return rank, world, local, pg


def _cuda_ok():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def barrier(pg):
    if pg is not None:
        pg.barrier()


def max_over_ranks(pg, x):
    if pg is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if _cuda_ok() else "cpu")
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ CPU oracle
def cpu_model():
    """The host CPU's model name (lscpu / /proc/cpuinfo), or 'unknown'."""
    try:
        out = subprocess.run(["lscpu"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                             timeout=10).stdout.decode()
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def _sample_code(steps, warmup, nx):
    from paper_2103_08246_gb300 import inputs
    h = inputs.PRODUCTION.lx / inputs.PRODUCTION.nx
    lx = nx * h
    wp = inputs.PRODUCTION
    bars = lx >= wp.bar_x + 0.5 * wp.bar_width + 3 * h
    code = f"""
import json, sys, time
sys.path.insert(0, {ROOT!r})
from paper_2103_08246_gb300 import inputs
wl = inputs.PRODUCTION.replace(nx={nx}, lx={lx!r}, flag_on=False, bars_on={bars!r})
from oracle.solver import OracleSolver
s = OracleSolver(wl, inputs.initial_noise(wl))
for _ in range({warmup}):
    s.step()
t0 = time.perf_counter()
for _ in range({steps}):
    s.step()
dt = (time.perf_counter() - t0) / {steps}
print(json.dumps({{"sec_per_step": dt, "cells": wl.cells}}))
"""
    desc = (f"oracle (numpy/scipy FP64, 1 thread per process) on the first {nx} of 512 x-planes "
            f"({nx}x256x256, {'bars' if bars else 'inflow region only'}, no flag), "
            f"{steps} step(s) after {warmup} warm-up; scaled to the full workload by cell count")
    return code, desc


def oracle_sample_rate(steps: int, warmup: int, nx: int = SAMPLE_NX, procs: int = 1):
    """Time the CPU oracle on the first `nx` x-planes of the production
    workload (same spacing and transverse size; the bar grid when the sample
    reaches it; the flag lies further downstream and is left out), in `procs`
    independent single-threaded processes at once (one per host core for the
    all-cores figure). Returns (aggregate cell-updates/s, mean seconds per
    sample step, description)."""
    code, desc = _sample_code(steps, warmup, nx)
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    env["CUDA_VISIBLE_DEVICES"] = ""
    ps = [subprocess.Popen([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE,
                           stderr=subprocess.PIPE) for _ in range(procs)]
    rate, secs = 0.0, []
    for p in ps:
        out, err = p.communicate(timeout=3600)
        if p.returncode != 0:
            raise RuntimeError(err.decode()[-2000:])
        r = json.loads(out.decode().strip().splitlines()[-1])
        rate += r["cells"] / r["sec_per_step"]
        secs.append(r["sec_per_step"])
    if procs > 1:
        desc += f"; {procs} such processes at once (one per host core), rates summed"
    return rate, sum(secs) / len(secs), desc


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def run_reference(args):
    from paper_2103_08246_gb300 import inputs
    wl = inputs.PRODUCTION
    cores = host_cores()
    # size each process's sample so that warm-up + timed steps take about two minutes
    _, sec16, _ = oracle_sample_rate(1, 0, 16)
    per_plane = sec16 / 16
    budget = 120.0 / max(1, args.steps + args.warmup)
    nx = int(max(8, min(SAMPLE_NX, budget / per_plane / 2)))
    rate, sec, desc = oracle_sample_rate(max(1, args.steps), max(0, args.warmup), nx, procs=cores)
    steps_per_s = rate / wl.cells
    line = {
        "impl": "reference", "metric": METRIC, "value": steps_per_s, "unit": "steps/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 / steps_per_s, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "gcell_updates_per_s": rate / 1e9,
        "config": {"workload": wl.name, "cells": wl.cells, "precision": "fp64",
                   "cache": "inputs larger than L2"},
        "cpu_baseline": {"value": steps_per_s, "unit": "steps/s", "cores": cores, "kind": "oracle",
                         "sample": desc, "cpu_model": cpu_model()},
        "e2e": {"value": steps_per_s, "unit": "steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm
def time_steps(solver, steps, stream):
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    solver.step(steps)
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / steps


def timed_leg(solver, steps, gpu_index, pg=None):
    """ms per step of `steps` steps (CUDA events on the solver's stream,
    bracketed by a barrier and a synchronize), with the SM clocks sampled
    from just before the timed region until at least CLOCK_WINDOW_S later: a
    short timed region is followed by more identical (untimed) steps inside
    the sampling window, so that the record holds several samples."""
    import torch
    barrier(pg)
    torch.cuda.synchronize()
    clocks = ClockSampler(gpu_index)
    clocks.start()
    t0 = time.perf_counter()
    ms = time_steps(solver, steps, solver.stream)
    while time.perf_counter() - t0 < CLOCK_WINDOW_S:
        solver.step(max(1, steps))
        torch.cuda.synchronize()
    clk = clocks.stop()
    clk["window_s"] = time.perf_counter() - t0
    barrier(pg)
    return ms, clk


def ib_algorithmic_bytes(solver, elem):
    """Bytes the IB stage must move per step: every velocity node in the
    support of any marker read once for the interpolation and read and
    written once by the spreading (per component), plus the marker data
    (positions read by both passes, the FP64 forcing amplitude written and
    read, the flag's target velocity and force)."""
    import numpy as np
    wl = solver.wl
    h = wl.lx / wl.nx
    X = solver.markers()
    nodes = 0
    for comp in range(3):
        off = [0.0 if d == comp else 0.5 for d in range(3)]
        base = [np.floor(X[:, d] / h - off[d] - 0.5).astype(np.int64) for d in range(3)]
        lo = 1 if comp == 0 else 0
        keys = []
        for a in range(3):
            i = base[0] + a
            ok = (i >= lo) & (i <= wl.nx - 1)
            for b in range(3):
                j = np.mod(base[1] + b, wl.ny)
                for e in range(3):
                    k = np.mod(base[2] + e, wl.nz)
                    keys.append(((i * wl.ny + j) * wl.nz + k)[ok])
        nodes += np.unique(np.concatenate(keys)).size
    nm = X.shape[0]
    return nodes * 3 * elem + nm * (2 * 24 + 2 * 24) + solver.nf * 48, nodes


def stage_roofline(wl, precision, peak_gbs, peak_kind):
    """Per-kernel device times on a timing-only state; roofline of every
    streamed kernel and of the IB stage, and the dominant kernel (the most
    time per step)."""
    from paper_2103_08246_gb300 import binding, inputs
    key = "mixed" if precision == binding.IBM_MIXED else "fp32"
    t = binding.Solver(wl, precision, noise=inputs.initial_noise(wl))
    t.step(5)
    n_sub = t.stats()["n_sub"]
    elem = 4
    cells = {"velocity": (wl.nx + 1) * wl.ny * wl.nz, "pressure": wl.nx * wl.ny * wl.nz}
    stages = {}
    for name in PER_STEP[key]:
        t.time_stage(name, 2)
        stages[name] = t.time_stage(name, 10)
    t.time_stage("poisson", 2)
    stages["poisson"] = t.time_stage("poisson", 10)
    ib_bytes, ib_nodes = ib_algorithmic_bytes(t, elem)
    t.close()
    per_step = {k: stages[k] * PER_STEP[key][k] for k in PER_STEP[key]}
    kernels = {}
    for k in PER_STEP[key]:
        if k in FIELD_PASSES:
            n = cells["pressure" if k in PRESSURE_GRID else "velocity"]
            passes = MIXED_PASSES.get(k, FIELD_PASSES[k]) if key == "mixed" else FIELD_PASSES[k]
            nbytes = passes * n * elem
        elif k == "ib":
            nbytes = ib_bytes
        else:
            continue
        gbs = nbytes / (stages[k] * 1e-3) / 1e9
        kernels[k] = {"ms_per_launch": stages[k], "launches_per_step": PER_STEP[key][k],
                      "alg_bytes_per_launch": nbytes, "achieved_gbs": gbs, "frac": gbs / peak_gbs,
                      "traffic": TRAFFIC_BYTES[key].get(k)}
    kernels["ib"]["nodes_touched"] = ib_nodes
    # the FP64 flag update (side stream, overlapped with the pressure solve);
    # its cost scales with the sub-step count of this state's time step
    kernels["flag"] = {"ms_per_launch": stages["flag"], "launches_per_step": 1, "sub_steps": n_sub,
                       "bound": "fp64 pipe and cluster barriers", "overlapped": True}
    dom = max((k for k in kernels if k not in ("ib", "flag")), key=lambda k: per_step[k])
    d = kernels[dom]
    roof = {"kernel": dom, "bound": "hbm", "achieved": d["achieved_gbs"], "peak": peak_gbs,
            "peak_kind": peak_kind, "unit": "GB/s", "frac": d["frac"], "traffic": d["traffic"],
            "alg_bytes_per_launch": d["alg_bytes_per_launch"], "ms_per_launch": d["ms_per_launch"]}
    return roof, stages, kernels


def host_link_gbs(nbytes=256 << 20, reps=5):
    """Pinned host <-> device copy bandwidth (GB/s) of this box, H2D and D2H,
    by CUDA events around cudaMemcpyAsync on a side stream."""
    import torch
    h = torch.empty(nbytes // 8, dtype=torch.float64, pin_memory=True)
    h.fill_(1.0)
    d = torch.empty_like(h, device="cuda")
    st = torch.cuda.Stream()
    out = []
    for direction in ("h2d", "d2h"):
        with torch.cuda.stream(st):
            for r in range(2):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(st)
                for _ in range(reps):
                    if direction == "h2d":
                        d.copy_(h, non_blocking=True)
                    else:
                        h.copy_(d, non_blocking=True)
                e1.record(st)
                e1.synchronize()
        out.append(nbytes * reps / (e0.elapsed_time(e1) * 1e6))
    return out


def e2e_rate(wl, precision, steps):
    """Steps/s through the C ABI with host buffers: upload the state (FP64
    host arrays, converted on the device) from pinned host memory, K x
    (ibm_step + flag state read-back), read the fields back. One untimed pass
    of the same sequence first (module loading, first graph uploads), then the
    median of three timed passes. Also
    reports the host link's copy bandwidth and the state transfer time it
    implies; the caller adds the rate these allow, K / (K x device step time +
    transfer time)."""
    import torch
    from paper_2103_08246_gb300 import binding, inputs
    s = binding.Solver(wl, precision, noise=inputs.initial_noise(wl))
    s.step(2)
    fields = [s.field(q) for q in (binding.IBM_FIELD_U, binding.IBM_FIELD_V, binding.IBM_FIELD_W,
                                   binding.IBM_FIELD_P)]
    host = []
    for a in fields:
        t = torch.empty(a.shape, dtype=torch.float64, pin_memory=True)
        t.numpy()[...] = a
        host.append(t.numpy())
    nf = s.nf
    X = torch.empty((nf, 3), dtype=torch.float64, pin_memory=True).numpy()
    V = torch.empty((nf, 3), dtype=torch.float64, pin_memory=True).numpy()
    F = torch.empty((nf, 3), dtype=torch.float64, pin_memory=True).numpy()
    qs = (binding.IBM_FIELD_U, binding.IBM_FIELD_V, binding.IBM_FIELD_W, binding.IBM_FIELD_P)

    def run(k):
        for q, a in zip(qs, host):
            binding.ibm_set_field(s.state, q, a)
        for _ in range(k):
            s.step(1)
            binding.ibm_flag_state(s.state, X, V, F)
        for q, a in zip(qs, host):
            binding.ibm_get_field(s.state, q, a)
    run(1)
    # three timed repetitions, the median reported: the host's own scheduling
    # between the per-step synchronisations moves single runs by up to ~20%
    els = []
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        run(steps)
        els.append(time.perf_counter() - t0)
    el = statistics.median(els)
    s.close()
    field_bytes = sum(a.nbytes for a in host)          # FP64 host arrays: the bytes that cross the link
    h2d = field_bytes / steps + 16                     # + the time-step mode (two doubles) per step
    d2h = field_bytes / steps + 3 * X.nbytes + 8 * 64  # + flag X, V, F and the step parameters
    link_h2d, link_d2h = host_link_gbs()
    return {"value": steps / el, "unit": "steps/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "repeats_steps_per_s": [steps / e for e in els],
            "link_gbs": {"h2d": link_h2d, "d2h": link_d2h}, "state_transfer_ms":
            (field_bytes / (link_h2d * 1e6) + field_bytes / (link_d2h * 1e6))}


def _ensemble_ms(ens, steps):
    import torch
    ens.step(3)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(ens.stream)
    ens.step(steps)
    e1.record(ens.stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / steps


def ensemble_rate(steps):
    """The 16-case ensemble (uneven grids, mixed precision, tuned tiles):
    aggregate cell updates per second stepped together (one graph launch per
    step with every member a branch; and with the members' explicit stages
    batched into one persistent case-table launch) and one by one."""
    import torch
    from paper_2103_08246_gb300 import binding, ensemble
    solvers, ens = ensemble.build()
    ms_together = _ensemble_ms(ens, steps)
    ens.close()
    bat = binding.Ensemble(solvers, batched=True)
    ms_batched = _ensemble_ms(bat, steps)
    bat.close()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s in solvers:
        s.step(steps)
    torch.cuda.synchronize()
    ms_alone = (time.perf_counter() - t0) * 1e3 / steps
    cells = sum(s.wl.cells for s in solvers)
    shapes = [f"{s.wl.nx}x{s.wl.ny}x{s.wl.nz}" for s in solvers]
    for s in solvers:
        s.close()
    return {"cases": len(shapes), "cells": cells, "ms_per_ensemble_step": ms_together,
            "gcell_updates_per_s": cells / ms_together / 1e6,
            "batched_explicit_stage": {"ms_per_ensemble_step": ms_batched,
                                       "gcell_updates_per_s": cells / ms_batched / 1e6},
            "ms_per_step_one_by_one": ms_alone, "speedup_over_one_by_one": ms_alone / ms_together,
            "precision": "mixed", "shapes": shapes}


def slab_rate(steps, nranks=4):
    """The production workload (fixed dt = 2e-3, FP64) decomposed into
    `nranks` x slabs, the paper's own split of one case over four GPUs,
    with every rank emulated on this one GPU: each phase runs on every rank
    in turn and the exchanges are device copies (no collective, no kernel
    waiting on another rank). Wall time per step with a synchronize on both
    sides, against the single-domain FP64 step at the same dt; plus the bytes
    each rank would exchange per step on several GPUs."""
    import torch
    from paper_2103_08246_gb300 import binding, inputs
    from paper_2103_08246_gb300 import slab as S
    wl = inputs.PRODUCTION.replace(dt=2e-3)
    noise = inputs.initial_noise(wl)
    ranks = S.make_ranks(wl, nranks, wl.dt, noise)
    comm = S.LoopbackComm()
    S.run_phases(ranks, comm, S.INIT_SEQUENCE)
    for _ in range(2):
        S.run_phases(ranks, comm, S.STEP_SEQUENCE, wl.dt)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        S.run_phases(ranks, comm, S.STEP_SEQUENCE, wl.dt)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3 / steps
    # each rank's own phases, timed one at a time with a synchronize after
    # each (what that rank's GPU would spend per step), and the device-copy
    # exchanges between them
    per_rank = [0.0] * nranks
    xch = 0.0
    for _ in range(steps):
        recv = [None] * nranks
        for ph in S.STEP_SEQUENCE:
            sends = []
            for i, r in enumerate(ranks):
                t1 = time.perf_counter()
                sends.append(r.phase(ph, wl.dt, recv[i]))
                torch.cuda.synchronize()
                per_rank[i] += time.perf_counter() - t1
            t1 = time.perf_counter()
            kind, _, recv_count = ranks[0].plan(ph)
            recv = comm.exchange(kind, sends, recv_count)
            torch.cuda.synchronize()
            xch += time.perf_counter() - t1
    xbytes = max(8 * sum(r.plan(ph)[1] for ph in S.STEP_SEQUENCE) for r in ranks)
    ghosts = ranks[0].slab.ghosts
    for r in ranks:
        r.close()
    one = binding.Solver(wl, binding.IBM_FP64, noise=noise)
    one.step(3)
    ms1 = time_steps(one, steps, one.stream)
    one.close()
    return {"ranks": nranks, "precision": "fp64", "dt": wl.dt, "ghost_planes": ghosts,
            "ms_per_step": ms, "steps_per_s": 1000.0 / ms, "single_domain_ms_per_step": ms1,
            "rank_phases_ms_per_step": [1e3 * t / steps for t in per_rank],
            "loopback_exchange_ms_per_step": 1e3 * xch / steps,
            "exchange_mb_per_rank_per_step": xbytes / 1e6,
            "emulated": "all ranks on one GPU in turn, exchanges as device copies"}


def generator_flops(P, blocks, cin=6, width=128, cout=3):
    """Algorithmic FLOPs of the inflow generator per sample: forward, input
    gradients (every layer but the first) and weight gradients; 2 per
    multiply-add of each 3 x 3 periodic convolution over P pixels."""
    conv = lambda ci, co: 2.0 * P * 9 * ci * co
    fwd = conv(cin, width) + blocks * conv(width, width) + conv(width, cout)
    dgrad = blocks * conv(width, width) + conv(cout, width)
    return fwd, fwd + dgrad + fwd


def generator_rate(bf16_peak, peak_kind, nrep=10):
    """The learned inflow generator at the production plane (256 x 256,
    13 residual blocks of width 128, batch 8): training step, rollout and
    its dominant kernel (the residual-block convolution) on the tensor
    cores."""
    from paper_2103_08246_gb300 import binding, inputs
    ny = nz = 256
    blocks, batch = 13, 8
    gen = binding.Generator(ny, nz, blocks=blocks, in_channels=6, batch=batch)
    gen.set_params(inputs.generator_params(0, 128, blocks, 6))
    fwd, train = generator_flops(ny * nz, blocks)
    ms_train = gen.time("train_step", nrep)
    ms_fwd = gen.time("forward", nrep)
    ms_conv = gen.time("conv_fwd", 3 * nrep)
    ms_dgrad = gen.time("conv_dgrad", 3 * nrep)
    ms_wgrad = gen.time("conv_wgrad", 3 * nrep)
    gen.close()
    g1 = binding.Generator(ny, nz, blocks=blocks, in_channels=6, batch=1)
    g1.set_params(inputs.generator_params(0, 128, blocks, 6))
    ms_roll = g1.time("forward", nrep)
    g1.close()
    conv_flops = 2.0 * batch * ny * nz * 9 * 128 * 128
    # algorithmic bytes of the residual-block convolution: read the bf16
    # activation and the FP32 residual, write the FP32 sum and its bf16
    # activation (the weights and the halo rows come from L2)
    conv_bytes = batch * ny * nz * 128 * (2 + 4 + 4 + 2)
    tf = lambda fl, ms: fl / (ms * 1e-3) / 1e12
    hbm_peak, hbm_kind = measured_peaks()
    gbs = conv_bytes / (ms_conv * 1e-3) / 1e9
    # the binding roof: HBM (0.119 ms at the measured copy bandwidth) above
    # the tensor pipe (0.082 ms at the measured bf16 burst)
    return {"plane": f"{ny}x{nz}", "blocks": blocks, "width": 128, "batch": batch,
            "params": inputs.generator_param_count(128, blocks, 6),
            "train_step_ms": ms_train, "train_samples_per_s": batch / ms_train * 1e3,
            "train_tflops": tf(batch * train, ms_train),
            "forward_ms": ms_fwd, "forward_tflops": tf(batch * fwd, ms_fwd),
            "rollout_forward_ms": ms_roll,
            "conv_ms": {"fwd": ms_conv, "dgrad": ms_dgrad, "wgrad": ms_wgrad},
            "roofline": {"kernel": "k_conv<128,128,256> (residual block, forward)", "bound": "hbm",
                         "achieved": gbs, "peak": hbm_peak, "peak_kind": hbm_kind, "unit": "GB/s",
                         "frac": gbs / hbm_peak, "traffic": GEN_CONV_TRAFFIC_BYTES, "bytes_per_launch": conv_bytes,
                         "ms_per_launch": ms_conv},
            "tensor": {"achieved": tf(conv_flops, ms_conv), "peak": bf16_peak, "peak_kind": peak_kind,
                       "unit": "TFLOP/s", "frac": tf(conv_flops, ms_conv) / bf16_peak,
                       "flops_per_launch": conv_flops},
            "wgrad_tflops": tf(conv_flops, ms_wgrad), "dgrad_tflops": tf(conv_flops, ms_dgrad)}


def _with_clocks(gpu_index, fn, *a, **kw):
    clocks = ClockSampler(gpu_index)
    clocks.start()
    out = fn(*a, **kw)
    clk = clocks.stop()
    if isinstance(out, dict):
        out["clocks"] = clk
    return out


def run_ours(args):
    import torch
    from paper_2103_08246_gb300 import binding, build, inputs
    rank, world, local, pg = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    if local == 0:
        build.build()
    barrier(pg)
    build.build()
    binding.load()
    wl = inputs.PRODUCTION
    prec = binding.IBM_MIXED
    solver = binding.Solver(wl, prec, noise=inputs.initial_noise(wl))
    solver.step(max(3, args.warmup))
    torch.cuda.synchronize()
    kernels_per_step = solver.stats()["kernels_per_step"]
    ms, clk = timed_leg(solver, args.steps, local, pg)
    ms = max_over_ranks(pg, ms)
    st = solver.stats()
    solver.close()
    peak, peak_kind = measured_peaks()
    if rank == 0:
        cells = wl.cells
        roof, stages, kernels = stage_roofline(wl, prec, peak, peak_kind)
        step_bytes = METHOD_PASSES["mixed"] * (wl.nx + 1) * wl.ny * wl.nz * 4
        fp32 = fp64 = ens = gen = slab = None
        if not args.no_fp64:
            s32 = binding.Solver(wl, binding.IBM_FP32, noise=inputs.initial_noise(wl))
            s32.step(3)
            ms32, clk32 = timed_leg(s32, args.steps, local)
            s32.close()
            roof32, stages32, kernels32 = stage_roofline(wl, binding.IBM_FP32, peak, peak_kind)
            fp32 = {"steps_per_s": 1000.0 / ms32, "ms_per_step": ms32,
                    "gcell_updates_per_s": cells / ms32 / 1e6, "dtype": "f32",
                    "step_hbm_frac": (METHOD_PASSES["fp32"] * (wl.nx + 1) * wl.ny * wl.nz * 4
                                      / (ms32 * 1e-3) / 1e9) / peak,
                    "roofline": roof32, "stages_ms": stages32, "kernels": kernels32, "clocks": clk32}
            s64 = binding.Solver(wl, binding.IBM_FP64, noise=inputs.initial_noise(wl))
            s64.step(3)
            ms64, clk64 = timed_leg(s64, max(5, args.steps // 4), local)
            s64.time_stage("rhs", 1)
            rhs64 = s64.time_stage("rhs", 3)
            s64.close()
            mhz = clk64.get("sm_mhz") or 2070.0
            peak_inst = FP64_INST_PER_CLK_SM * N_SMS * mhz * 1e6 / 1e9
            ach_inst = FP64_RHS_INST_PER_CELL * (wl.nx + 1) * wl.ny * wl.nz / (rhs64 * 1e-3) / 1e9
            fp64 = {"steps_per_s": 1000.0 / ms64, "ms_per_step": ms64,
                    "gcell_updates_per_s": cells / ms64 / 1e6, "dtype": "f64",
                    "roofline": {"kernel": "rhs", "bound": "alu", "unit": "G FP64 inst/s",
                                 "achieved": ach_inst, "peak": peak_inst,
                                 "peak_kind": "derived: 2 FP64 inst/clk/SM x 152 SMs x sampled clock",
                                 "frac": ach_inst / peak_inst, "ms_per_launch": rhs64},
                    "clocks": clk64}
            ens = _with_clocks(local, ensemble_rate, max(5, args.steps // 5))
            slab = _with_clocks(local, slab_rate, 3)
            gen = _with_clocks(local, generator_rate, *measured_bf16_peak())
        e2e = None if args.no_e2e else e2e_rate(wl, prec, args.steps)
        if e2e is not None:
            e2e["value"] *= world
            e2e["link_bound"] = world * args.steps / (args.steps * ms + e2e["state_transfer_ms"]) * 1000.0
        cpu = None
        if not args.no_cpu_baseline:
            rate1, _, desc1 = oracle_sample_rate(2, 1)
            cores = host_cores()
            rate_n, _, desc_n = oracle_sample_rate(1, 1, procs=cores)
            cpu = {"value": rate1 / cells, "unit": "steps/s", "cores": 1, "kind": "oracle",
                   "sample": desc1, "gcell_updates_per_s": rate1 / 1e9, "cpu_model": cpu_model(),
                   "all_cores": {"value": rate_n / cells, "unit": "steps/s", "cores": cores,
                                 "sample": desc_n, "gcell_updates_per_s": rate_n / 1e9}}
        value = world * 1000.0 / ms
        out = {
            "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "mixed: f32 fields, f32 fft predictor, double-single residual, bf16 tensor-core correction, f64 flag",
            "data": "synthetic",
            "config": {"workload": wl.name, "cells": cells,
                       "precision": "mixed (fp32 fields, fp32 fft predictor, double-single residual, bf16 tcgen05 correction, fp64 flag)",
                       "cfl": wl.cfl, "re": wl.re, "markers": st["n_markers"],
                       "cache": "inputs larger than L2 (each field 134 MB)",
                       "parallelism": f"replicas x{world}"},
            "gcell_updates_per_s": world * cells / ms / 1e6,
            "speedup_over_fp64": (fp64["ms_per_step"] / ms) if fp64 else None,
            "step_hbm_frac": (step_bytes / (ms * 1e-3) / 1e9) / peak,
            "roofline": roof, "stages_ms": stages, "kernels": kernels,
            "fp64": fp64, "fp32": fp32, "ensemble": ens, "inflow_generator": gen, "e2e": e2e,
            "x_slabs": slab,
            "cpu_baseline": cpu, "clocks": clk,
            "gpu_launches": kernels_per_step * args.steps,
            "dt_last": st["dt"], "cfl_last": st["cfl"], "n_sub": st["n_sub"],
            "max_div": st["max_div"],
        }
        print(json.dumps(out), flush=True)
    barrier(pg)
    if pg is not None:
        pg.destroy_process_group()


def main():
    args = parse()
    if args.profile_steps > 0:
        run_profile(args)
        return
    if args.profile_generator > 0:
        run_profile_generator(args)
        return
    if args.profile_slabs > 0:
        run_profile_slabs(args)
        return
    if args.profile_generator_train > 0:
        run_profile_generator_train(args)
        return
    if args.impl == "reference":
        rank = int(os.environ.get("RANK", "0"))
        if rank == 0:
            run_reference(args)
        return
    run_ours(args)


if __name__ == "__main__":
    main()
