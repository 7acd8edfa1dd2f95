#!/usr/bin/env python
"""Benchmark of the GB300 over-decomposed Jacobi library.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload poisson2d_8192|poisson3d_512|laplace2d_256|...]

Other workloads (separate JSON lines, see --help): the profiling sizes
poisson2d_4096 and poisson3d_256, time to 1e-8 (tts2d_512, tts3d_128,
tts3d_512), the 256-solve batch (batched), Poisson arrivals into the server
(serving) and the paper's 1024x1024x768 shape at four over-decomposition
levels (paper3d_od).

Workload (default): 2D 5-point Poisson, 8192x8192 FP64, over-decomposed into
16x16 blocks of 512x512 with device-side halo exchange, seeded uniform[0,1)
boundary and initial field, source normal(0,1).  One step is the workload's
whole run: 1000 Jacobi sweeps with the residual tested every 50 sweeps
(jacobi_solve with an unreachable tolerance and max_sweeps = 1000).  It is
timed for the plain FP64 path (the headline `value`) and for the FP32-inner
and BF16-stored-inner iterative refinement with 50 inner sweeps per FP64
outer step.  Inputs are 1.6 GB per sweep, far larger than the 129 MB L2.

Under torchrun (N > 1) every rank solves its own copy of the problem (the
solves are independent: weak scaling, no collective on the data path); the
barrier and the max-over-ranks time only bracket the timed region.

The default line also carries the metric's other legs, each measured in the
same run: `tts`, time to relative residual 1e-8 of plain FP64 against the
FP32- and BF16-inner refinement (real solves on a 512^2 2D and a 128^3 3D
Poisson grid, with each mixed form's error against the FP64 solution), and
`serving`, a short Poisson-arrival stream into the continuous-batching server
(fixed window, sizes capped, p50/p99 latency, completed and censored counts).
The headline region runs without per-kernel timing; the kernel split and the
roofline come from a second, profiled pass of the same steps.  The FP64
sweep's roofline peak is the FP64 pipe's rate measured by the library's probe
in the same process.

--impl reference times the CPU oracle (plain C, all host cores) on a bounded
sample of the same workload (100 of the 1000 sweeps per step at 8192^2): the
paper's code is not available, so the oracle is the reference arm.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SWEEPS_PER_STEP = 1000
CHECK_EVERY = 50


def refine_period_of(p):
    """Inner sweeps per refinement step: 20 for the 3D workloads (the 512^3
    configuration's), one residual interval (50) in 2D."""
    return 20 if p.ndim == 3 else CHECK_EVERY
HBM_PEAK_FALLBACK = 6800.0
# FP64 pipe, nominal: 1.25 TFLOP/s counts an FMA as 2 flops, i.e. 0.625e12
# FP64 instructions/s.  Used only if the library's FP64 probe cannot run.
FP64_ADD_PEAK_NOMINAL_G = 625.0
# FP64 additions one update needs in the canonical order with pair sharing
FP64_ADDS_PER_LUP = {2: 3.0, 3: 5.0}
BYTES_PER_LUP = {"f64": 24.0, "f32_refine": 12.0, "bf16_refine": 8.0}
METRIC = "Jacobi GLUP/s & % HBM roofline, mixed vs FP64 at 1e-8 resid; p99 solve ms"
# DRAM bytes (read + write) per lattice update of the 2D FP64 sweep kernel
# (k_f64_march4, lines staged in shared memory), from an ncu capture of one
# 8192^2 launch (1160.5 MB read + 506.9 MB written for 67.1 M updates).  None
# once that kernel has changed since the capture.
F64_SWEEP_DRAM_BYTES_PER_LUP = (1160.466e6 + 506.8544e6) / (8192 * 8192)

def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="poisson2d_8192",
                    choices=["poisson2d_8192", "poisson2d_4096", "laplace2d_256", "poisson3d_512", "poisson3d_256",
                             "tts2d_512", "tts3d_128", "tts3d_512", "batched", "serving", "paper3d_od"])
    ap.add_argument("--scale", type=float, default=0.25, help="batched: side scale (1.0 = the full 64..2048 recipe)")
    ap.add_argument("--rate", type=float, default=10.0, help="serving: arrivals per second")
    ap.add_argument("--window", type=float, default=20.0, help="serving: arrival window, seconds")
    ap.add_argument("--cap2d", type=int, default=512, help="serving: largest 2D side admitted to the stream")
    ap.add_argument("--cap3d", type=int, default=128, help="serving: largest 3D side admitted to the stream")
    ap.add_argument("--no-seq", action="store_true", help="batched: skip the one-by-one comparison")
    ap.add_argument("--sweeps", type=int, default=0, help="override the sweeps per step (profiling runs)")
    ap.add_argument("--forms", default="f64,f32_refine,bf16_refine")
    ap.add_argument("--emu", type=int, default=-1, help="FP64 additions per warp step on the integer pipe (0, 2, 3)")
    ap.add_argument("--tma", type=int, default=-1, help="2D inner sweeps staged by bulk async copies (0/1)")
    ap.add_argument("--march", type=int, default=-1, help="2D FP64 sweeps over march items (0..3; -1: the library default, 3)")
    ap.add_argument("--outer-split", type=int, default=-1, help="3D outer step in two passes (0/1)")
    ap.add_argument("--rows-low", type=int, default=0, help="lines per low-precision work item (0: library default)")
    ap.add_argument("--l2pf", type=int, default=-1, help="FP64 sweeps: lines prefetched into L2 ahead (0: none)")
    ap.add_argument("--tb", type=int, default=-1, help="2D inner sweeps two per launch (2) or one (0)")
    ap.add_argument("--rows-f64", type=int, default=0, help="lines per FP64 work item (0: library default)")
    ap.add_argument("--server-opts", default="", help="serving: server options as key=value,key=value")
    ap.add_argument("--budget-gib", type=float, default=64.0, help="serving: HBM budget of the server arena (GiB)")
    ap.add_argument("--grace", type=float, default=60.0, help="serving: seconds after the window before censoring")
    ap.add_argument("--block", default="", help="override the workload's block shape, e.g. 512,64,64")
    ap.add_argument("--full-f64", action="store_true",
                    help="tts3d_512: run the plain FP64 solve to 1e-8 (~11 min) instead of extrapolating it, "
                         "which also gives the mixed forms' error against it")
    ap.add_argument("--ref-sweeps", type=int, default=0,
                    help="tts3d_512: sweep count of a refinement solve measured earlier, for the FP64 extrapolation "
                         "when only f64 runs")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-legs", action="store_true", help="skip the time-to-tolerance and serving legs")
    ap.add_argument("--leg-rate", type=float, default=30.0, help="serving leg: arrivals per second")
    ap.add_argument("--leg-window", type=float, default=5.0, help="serving leg: arrival window, seconds")
    ap.add_argument("--leg-cap2d", type=int, default=256, help="serving leg: largest 2D side")
    ap.add_argument("--leg-cap3d", type=int, default=64, help="serving leg: largest 3D side")
    return ap.parse_args()


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return HBM_PEAK_FALLBACK, "fallback"


def fp64_peak(stream):
    """Measured FP64 pipe rate (G lane operations/s) of fma.rn.f64 with the
    multiplier 1.0 in a register -- the form of every FP64 addition in the
    sweeps, and the fastest FP64 instruction form on GB300 -- in 8 independent
    chains per thread on a full device: best of three."""
    from paper_2303_02543_gb300 import jacobi as J
    try:
        best = max(J.jacobi_probe_fp64_rate(1, 8, 8, 8192, stream) for _ in range(3))
        return best / 1e9, "measured: fma.rn.f64 probe, register multiplier (8 chains/thread, 8 CTAs/SM), best of 3"
    except J.JacobiError as e:
        return FP64_ADD_PEAK_NOMINAL_G, f"nominal (probe failed: {e})"


def make_workload(name):
    from paper_2303_02543_gb300 import inputs
    if name == "poisson2d_8192":
        p = inputs.poisson_2d_large()
        desc = "2D 5-point Poisson 8192x8192 FP64, 16x16 blocks of 512x512, 1000 sweeps, residual every 50"
    elif name == "poisson2d_4096":
        p = inputs.poisson_2d_large(n=4096)
        desc = "2D 5-point Poisson 4096x4096 FP64, 8x8 blocks of 512x512 (profiling size, > L2)"
    elif name == "poisson3d_256":
        p = inputs.poisson_3d(n=256)
        desc = "3D 7-point Poisson 256^3 FP64, blocks of 64^3 (profiling size, > L2)"
    elif name == "laplace2d_256":
        p = inputs.laplace_2d_small()
        desc = "2D 5-point Laplace 256x256 FP64, 4x4 blocks of 64x64, 100 sweeps"
    else:
        p = inputs.poisson_3d()
        desc = "3D 7-point Poisson 512^3 FP64, blocks of 64^3, sweeps with residual every 50"
    sweeps = 100 if name == "laplace2d_256" else SWEEPS_PER_STEP
    return p, desc, sweeps


class ClockSampler:
    """nvidia-smi clock / throttle samples every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import datetime

        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        # a rank that fails or never arrives ends the others' next collective
        # with an error after this long instead of leaving them waiting
        timeout = datetime.timedelta(seconds=float(os.environ.get("JACOBI_PG_TIMEOUT_S", "900")))
        dist.init_process_group(backend=backend, timeout=timeout)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, world):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---- CPU oracle timing ------------------------------------------------------

def oracle_sample(p, sweeps, threads=0):
    """Time the oracle on `sweeps` sweeps of the workload with residual tests
    at both ends, on all host cores (threads=0) or on `threads`; returns
    (GLUP/s, seconds, threads used)."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    oracle.solve(p.dims, p.faces, p.source, p.x0, 1e-300, sweeps, CHECK_EVERY, threads=threads)
    dt = time.perf_counter() - t0
    return p.points * sweeps / dt / 1e9, dt, threads or oracle.max_threads()


def cpu_baseline(p, name):
    # on 8192^2 the whole 1000-sweep step: about 7 s on 16 cores
    sweeps = {"poisson2d_8192": 1000, "poisson2d_4096": 2000, "laplace2d_256": 100000, "poisson3d_512": 300,
              "poisson3d_256": 2000}[name]
    glups, dt, cores = oracle_sample(p, sweeps)
    # one core, on a twentieth of the sweeps (a few seconds); taken last,
    # because the oracle keeps the thread count it was last given
    one, dt1, _ = oracle_sample(p, max(1, sweeps // 20), threads=1)
    return {"value": glups, "unit": "GLUP/s", "cores": cores, "kind": "oracle",
            "sample": f"{sweeps} sweeps of the full {'x'.join(map(str, p.dims))} grid with residual tests "
                      f"before and after ({dt:.1f} s, OpenMP on {cores} threads)",
            "single_thread": {"value": one, "unit": "GLUP/s", "cores": 1,
                              "sample": f"{max(1, sweeps // 20)} sweeps of the same grid on one thread ({dt1:.1f} s)"}}


def run_reference(args, rank, world):
    if rank != 0:
        return
    if args.workload not in ("poisson2d_8192", "poisson2d_4096", "laplace2d_256", "poisson3d_512", "poisson3d_256"):
        args.workload = "poisson2d_8192"
    p, desc, _ = make_workload(args.workload)
    # about a second per step on 16 cores, so that the oracle's per-call setup
    # (ghosted copies of the inputs, two residual tests) is a small part of it
    sweeps = {"poisson2d_8192": 100, "poisson2d_4096": 400, "laplace2d_256": 20000, "poisson3d_512": 20,
              "poisson3d_256": 150}[args.workload]
    for _ in range(args.warmup):
        oracle_sample(p, sweeps)
    t0 = time.perf_counter()
    cores = 1
    for _ in range(args.steps):
        _, _, cores = oracle_sample(p, sweeps)
    dt = time.perf_counter() - t0
    glups = p.points * sweeps * args.steps / dt / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": glups, "unit": "GLUP/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "description": desc,
                       "sample": f"{sweeps} sweeps per step (bounded sample of the {SWEEPS_PER_STEP}-sweep run)",
                       "setup_note": "each step is one oracle solve call: its set-up (ghosted copies of the "
                                     "inputs, ||b||^2 and three residual tests, partly single-threaded) is "
                                     "inside the timed step, about 30% of it at 100 sweeps"},
            "cpu_baseline": {"value": glups, "unit": "GLUP/s", "cores": cores, "kind": "oracle",
                             "sample": f"{sweeps} sweeps per step x {args.steps} steps"},
            "e2e": {"value": glups, "unit": "GLUP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---- GPU arm ----------------------------------------------------------------

def time_form(p, form, sweeps, args, world, stream, sampler=None):
    import torch
    from paper_2303_02543_gb300 import jacobi as J
    opts = {}
    if form == "f64" and args.emu >= 0:
        opts["emu_adds"] = args.emu
    if form == "f64" and args.march >= 0:
        opts["march"] = args.march
    if form == "f64" and args.l2pf >= 0:
        opts["l2pf"] = args.l2pf
    if form != "f64" and args.tma >= 0:
        opts["tma"] = args.tma
    if form != "f64" and args.outer_split >= 0:
        opts["outer_split"] = args.outer_split
    if form != "f64" and args.tb >= 0:
        opts["tb"] = args.tb
    if form != "f64" and args.rows_low > 0:
        opts["rows_low"] = args.rows_low
    if args.rows_f64 > 0:
        opts["rows_f64"] = args.rows_f64
    s = J.Solver(p.dims, p.block, dtype=form, faces=p.faces, source=p.source, x0=p.x0,
                 check_every=CHECK_EVERY, refine_period=refine_period_of(p), profile=0, **opts)

    def step():
        st, sw, rel = s.solve(1e-300, sweeps)
        if st not in (J.OK, J.ERR_NOT_CONVERGED) or sw != sweeps:
            raise RuntimeError(f"step failed: status {st}, sweeps {sw}")
        return rel

    def timed(nsteps):
        barrier(world)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        rel = None
        for _ in range(nsteps):
            rel = step()
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        return max_over_ranks(ev0.elapsed_time(ev1), world), rel

    for _ in range(args.warmup):
        step()
    kern = "sweep_f64" if form == "f64" else "sweep_low"
    # the headline region: no per-kernel events inside it
    launches0 = s.profile("all")[1]
    if sampler:
        sampler.start()
    ms, rel = timed(args.steps)
    clocks = sampler.stop() if sampler else None
    launches = s.profile("all")[1] - launches0
    # a second pass of the same steps with CUDA events around every launch on
    # the launching stream: the kernel split and the roofline's kernel time
    s.set_option("profile", 1)
    step()
    for k in ("sweep_f64", "sweep_low", "refine_outer", "reduce", "halo"):
        s.profile(k, reset=True)
    ms_prof, _ = timed(args.steps)
    kms, kn = s.profile(kern)
    other = {k: s.profile(k) for k in ("refine_outer", "reduce", "halo")}
    s.set_option("profile", 0)
    out = {"ms": ms, "ms_profiled_pass": ms_prof, "kernel": kern, "kernel_ms": kms, "kernel_launches": kn,
           "launches": launches, "rel": rel, "clocks": clocks, "other": other, "solver": s}
    return out


def e2e_form(s, p, sweeps, args, world, stream):
    """Same step through the C ABI with host buffers: upload x from pinned host
    memory, run the step, read the field back into pinned host memory."""
    import torch
    x0 = p.x0 if p.x0 is not None else np.zeros(p.shape)
    x_host = torch.from_numpy(x0.copy()).pin_memory()
    out = torch.empty(p.shape, dtype=torch.float64).pin_memory()
    for _ in range(max(1, args.warmup - 2)):
        s.set_field(x_host)
        s.solve(1e-300, sweeps)
        s.field(out)
    barrier(world)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        s.set_field(x_host)
        st, sw, rel = s.solve(1e-300, sweeps)
        s.field(out)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    ms = max_over_ranks(ev0.elapsed_time(ev1), world)
    nbytes = p.points * 8
    return ms, nbytes, nbytes + 16


def run_ours(args, rank, world, local):
    import torch
    from paper_2303_02543_gb300 import build as B
    if rank == 0 and not B.up_to_date():
        B.build()
    barrier(world)
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    p, desc, sweeps = make_workload(args.workload)
    if args.block:
        p.block = tuple(int(v) for v in args.block.split(","))
        desc += f" (blocks overridden to {'x'.join(map(str, p.block))})"
    if args.sweeps > 0:
        sweeps = args.sweeps
    hbm_peak, peak_kind = measured_peaks()
    f64_peak, f64_peak_kind = fp64_peak(stream.cuda_stream)
    forms = [f for f in args.forms.split(",") if f]
    results = {}
    clocks = None
    head = forms[0]
    for form in forms:
        sampler = ClockSampler(torch.cuda.current_device()) if form == head and rank == 0 else None
        results[form] = time_form(p, form, sweeps, args, world, stream, sampler)
        if sampler:
            clocks = results[form]["clocks"]
    h = results[head]
    lups = p.points * sweeps * args.steps * world
    value = lups / (h["ms"] / 1e3) / 1e9
    e2e = None
    if not args.no_e2e:
        ms_e2e, h2d, d2h = e2e_form(h["solver"], p, sweeps, args, world, stream)
        e2e = {"value": lups / (ms_e2e / 1e3) / 1e9, "unit": "GLUP/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}
    # roofline of the dominant kernel of the headline form
    nd = p.ndim
    per_launch_ms = h["kernel_ms"] / max(1, h["kernel_launches"])
    lup_rate = p.points / (per_launch_ms / 1e3)
    if head == "f64":
        achieved = FP64_ADDS_PER_LUP[nd] * lup_rate / 1e9
        traffic = (F64_SWEEP_DRAM_BYTES_PER_LUP * p.points
                   if (nd == 2 and args.emu <= 0 and args.march in (-1, 3) and F64_SWEEP_DRAM_BYTES_PER_LUP)
                   else None)
        roof = {"bound": "alu", "kernel": "sweep_f64", "achieved": achieved, "peak": f64_peak,
                "unit": "G FP64 adds/s", "frac": achieved / f64_peak, "traffic": traffic,
                "traffic_note": "ncu dram read+write of one 8192^2 launch, per update times the points" if traffic else None,
                "peak_kind": f64_peak_kind, "adds_per_lup": FP64_ADDS_PER_LUP[nd],
                "nominal_frac": achieved / FP64_ADD_PEAK_NOMINAL_G,
                "hbm": {"achieved": BYTES_PER_LUP[head] * lup_rate / 1e9, "peak": hbm_peak, "unit": "GB/s",
                        "frac": BYTES_PER_LUP[head] * lup_rate / 1e9 / hbm_peak, "peak_kind": peak_kind,
                        "bytes_per_lup": BYTES_PER_LUP[head]}}
    else:
        per_sweep_ms = h["kernel_ms"] / (sweeps * args.steps)
        achieved = BYTES_PER_LUP[head] * p.points / (per_sweep_ms / 1e3) / 1e9
        roof = {"bound": "hbm", "kernel": "sweep_low", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": None, "peak_kind": peak_kind,
                "note": "effective: one sweep's bytes per point over the time per sweep"}
    forms_out = {}
    for form, r in results.items():
        kl = r["kernel_ms"] / max(1, r["kernel_launches"])
        # the inner sweeps may run two per launch: their time per sweep is the
        # class's total over the profiled pass divided by the sweeps it ran
        ks = kl if form == "f64" else r["kernel_ms"] / (sweeps * args.steps)
        lr = p.points / (ks / 1e3)
        forms_out[form] = {
            "glups": p.points * sweeps * args.steps * world / (r["ms"] / 1e3) / 1e9,
            "ms_per_step": r["ms"] / args.steps,
            "ms_per_step_profiled_pass": r["ms_profiled_pass"] / args.steps,
            "kernel": r["kernel"], "kernel_us": kl * 1e3, "kernel_launches_per_step": r["kernel_launches"] / args.steps,
            "kernel_us_per_sweep": ks * 1e3,
            "kernel_hbm_gbs": BYTES_PER_LUP[form] * lr / 1e9,
            "kernel_hbm_frac": BYTES_PER_LUP[form] * lr / 1e9 / hbm_peak,
            "kernel_hbm_note": (None if form == "f64" else
                                "bytes of one sweep per point / time per sweep: with two sweeps per launch "
                                "(temporal blocking) this is an effective figure and can exceed 1"),
            "rel_residual_after": r["rel"],
            "launches_per_step": r["launches"] / args.steps,
            "other_kernels_ms": {k: v[0] / args.steps for k, v in r["other"].items()},
        }
        r["solver"].close()
    line = {
        "metric": METRIC,
        "value": value, "unit": "GLUP/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": h["ms"] / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if head == "f64" else head, "data": "synthetic",
        "config": {"workload": args.workload, "description": desc, "grid": list(p.dims),
                   "block": list(p.block), "sweeps_per_step": sweeps, "check_every": CHECK_EVERY,
                   "refine_period": refine_period_of(p),
                   "l2": "inputs larger than L2 (no flush)" if p.points * 24 > 129e6 else "L2-resident",
                   "parallelism": f"replicas x{world}"},
        "roofline": roof, "forms": forms_out, "clocks": clocks, "e2e": e2e,
        "gpu_launches": int(h["launches"]),
    }
    if not args.no_legs:
        # the metric's other legs, on the same GPU in the same run
        line["tts"] = {w: tts_leg(w, args, local) for w in ("tts2d_512", "tts3d_128")}
        line["serving"] = serving_leg(args.leg_rate, args.leg_window, args.leg_cap2d, args.leg_cap3d, local)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(p, args.workload)
    if rank == 0:
        print(json.dumps(line), flush=True)


# ---- time to tolerance, batches, serving (separate lines, not the default) ---

def run_paper3d_od(args, rank, world, local):
    """The shape of the paper's Jacobi3D runs (section 4.3: a 1024x1024x768
    domain, a fixed number of iterations; section 4.4: over-decomposition
    levels): FP64, 100 sweeps with the residual tested every 50, the same
    grid cut into 1, 2, 8 and 64 blocks.  With block widths multiples of 64
    along x and 8 along z the residual does not depend on the decomposition,
    so every level must report the same bits."""
    import torch

    from paper_2303_02543_gb300 import inputs
    from paper_2303_02543_gb300 import jacobi as J
    torch.cuda.set_device(local)
    dims = (1024, 1024, 768)
    levels = {1: (1024, 1024, 768), 2: (1024, 1024, 384), 8: (512, 512, 384), 64: (256, 256, 192)}
    p = inputs.make_problem(dims, levels[1], 2310, boundary="zero", source="normal", x0="zero")
    sweeps = 100
    out, rels = {}, {}
    for od, blk in levels.items():
        with J.Solver(p.dims, blk, dtype="f64", faces=p.faces, source=p.source, check_every=CHECK_EVERY) as s:
            s.solve(1e-300, 10)  # warm-up
            s.set_field(np.zeros(p.shape))
            torch.cuda.synchronize()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record()
            st, sw, rel = s.solve(1e-300, sweeps)
            ev1.record()
            torch.cuda.synchronize()
            ms = ev0.elapsed_time(ev1)
            out[od] = {"blocks": int(np.prod([-(-dims[a] // blk[a]) for a in range(3)])), "block": list(blk),
                       "ms": ms, "glups": p.points * sweeps / (ms / 1e3) / 1e9, "rel_after": rel}
            rels[od] = rel
    if rank == 0:
        print(json.dumps({"metric": "Jacobi3D (paper shape) FP64 GLUP/s by over-decomposition level",
                          "workload": "paper3d_od", "grid": list(dims), "sweeps": sweeps,
                          "check_every": CHECK_EVERY, "od": out,
                          "residual_identical_across_levels": len(set(rels.values())) == 1,
                          "higher_is_better": True, "data": "synthetic"}), flush=True)


def tts_problem(workload):
    from paper_2303_02543_gb300 import inputs
    n = {"tts2d_512": 512, "tts3d_128": 128, "tts3d_512": 512}[workload]
    if workload == "tts2d_512":
        return inputs.make_problem((n, n), (128, 128), 2309, boundary="uniform", source="normal", x0="zero")
    return inputs.poisson_3d(n=n, block=64 if n >= 256 else 32)


def tts_leg(workload, args, local, forms=("f64", "f32_refine", "bf16_refine"), full_f64=True, ref_sweeps=0):
    """Time to relative residual 1e-8 of each form on the same grid and GPU.
    Each form is a real solve (jacobi_solve with tol 1e-8) unless full_f64 is
    False, when plain FP64 is timed over 500 sweeps with residual tests and
    multiplied by the refinement's sweep count (labelled `extrapolated`).
    rel is the library's FP64 residual of the returned field (an explicit
    b - A x pass); rel_error_vs_f64 = ||x_form - x_f64|| / ||x_f64|| where the
    FP64 solve really ran."""
    import torch

    from paper_2303_02543_gb300 import jacobi as J
    torch.cuda.set_device(local)
    p = tts_problem(workload)
    forms = list(forms)
    if not full_f64 and "f64" in forms:
        forms = [f for f in forms if f != "f64"] + ["f64"]
    out, fields = {}, {}
    for form in forms:
        opts = dict(check_every=CHECK_EVERY, refine_period=20 if p.ndim == 3 else 50, schedule=1, graph=1,
                    autotune=1)
        s = J.Solver(p.dims, p.block, dtype=form, faces=p.faces, source=p.source, **opts)
        if not full_f64 and form == "f64":
            # the warm-up goes through solve() so the autotuner picks the work
            # shape as in a real solve; the timed 500 sweeps include the
            # residual tests every check_every sweeps, as a real solve does
            s.solve(1e-300, 50)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s.solve(1e-300, 500)
            torch.cuda.synchronize()
            per = (time.perf_counter() - t0) / 500
            s.close()
            sw = ref_sweeps if ref_sweeps > 0 else (out.get("f32_refine") or next(iter(out.values())))["sweeps"]
            out[form] = {"status": None, "sweeps": sw, "seconds": per * sw, "extrapolated": True,
                         "seconds_per_sweep": per, "glups": p.points / per / 1e9}
            continue
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, sw, rel = s.solve(1e-8, 10 ** 9)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        fields[form] = s.field()
        s.close()
        out[form] = {"status": J.STATUS.get(st, st), "sweeps": sw, "seconds": dt, "rel": rel,
                     "glups": p.points * sw / dt / 1e9}
    base = out.get("f64", {}).get("seconds")
    for f, r in out.items():
        r["speedup_vs_f64"] = (base / r["seconds"]) if base else None
        if f != "f64" and "f64" in fields and f in fields:
            r["rel_error_vs_f64"] = float(np.linalg.norm(fields[f] - fields["f64"]) / np.linalg.norm(fields["f64"]))
    return {"grid": list(p.dims), "block": list(p.block), "tol": 1e-8, "unit": "s", "forms": out}


def run_tts(args, rank, world, local):
    """Time to relative residual 1e-8: plain FP64 against FP32- and
    BF16-inner refinement on the same grid and GPU (each a real solve; on
    512^3 plain FP64 takes ~11 minutes and is extrapolated unless --full-f64)."""
    forms = [f for f in args.forms.split(",") if f]
    full = not (args.workload == "tts3d_512" and not args.full_f64)
    leg = tts_leg(args.workload, args, local, forms=forms, full_f64=full, ref_sweeps=args.ref_sweeps)
    if rank == 0:
        print(json.dumps({"metric": "time to relative residual 1e-8 (s)", "workload": args.workload,
                          "grid": leg["grid"], "block": leg["block"], "higher_is_better": False,
                          "forms": leg["forms"], "data": "synthetic"}), flush=True)


def run_batched(args, rank, world, local):
    """The batched recipe (256 uneven 2D solves, sides log-uniform per axis,
    128^2 blocks) at side scale args.scale, FP32-inner refinement to 1e-8 in
    one persistent launch per step replayed from a CUDA graph, tiles from the
    autotuner; compared with solving the same grids one after another."""
    import torch

    from paper_2303_02543_gb300 import inputs
    from paper_2303_02543_gb300 import jacobi as J
    torch.cuda.set_device(local)
    probs = inputs.batched_2d(count=256, size_scale=args.scale)
    pts = sum(p.points for p in probs)
    opts = dict(refine_period=20, schedule=1, graph=1, autotune=1)
    b = J.Batch(probs, dtype="f32_refine", **opts)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st, res = b.solve(1e-8, 20 * 10 ** 7)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    launches = b.profile("all")[1]
    b.close()
    lups = sum(p.points * r[1] for p, r in zip(probs, res))
    # the same grids one context at a time (no batching), same options
    dt_seq = None
    if not args.no_seq:
        t1 = time.perf_counter()
        for p in probs:
            with J.Solver(p.dims, p.block, dtype="f32_refine", faces=p.faces, source=p.source,
                          refine_period=20, schedule=1, graph=1) as s:
                s.solve(1e-8, 20 * 10 ** 7)
        torch.cuda.synchronize()
        dt_seq = time.perf_counter() - t1
    if rank == 0:
        print(json.dumps({"metric": "batched solve to 1e-8: aggregate GLUP/s", "workload": "batched",
                          "value": lups / dt / 1e9, "unit": "GLUP/s", "seconds": dt,
                          "seconds_one_by_one": dt_seq, "speedup_vs_one_by_one": dt_seq / dt if dt_seq else None,
                          "solves": len(probs), "points": pts, "all_ok": st == J.OK,
                          "max_sweeps": max(r[1] for r in res), "launches": launches,
                          "max_rel": max(r[2] for r in res),
                          "config": {"scale": args.scale, "sides": [64 * args.scale, 2048 * args.scale],
                                     "block": 128, "refine_period": 20, "schedule": "persistent+graph",
                                     "autotune": True}, "data": "synthetic"}), flush=True)


def serving_leg(rate, window, cap2d, cap3d, local, server_opts=None, budget=16 << 30, grace=60.0):
    """Poisson arrivals at `rate` per second over `window` seconds into the
    continuous-batching server (FP32-inner refinement, each request to 1e-8):
    2D squares of side log-uniform in [128, cap2d] and 3D cubes of side
    log-uniform in [32, cap3d].  Requests not done `grace` seconds after the
    window closes are counted as censored; p50/p99 are over completed ones, and
    p50/p99_all_lower_bound over all requests, a censored one counted with the
    time from its arrival to the poll (a lower bound of its latency)."""
    import torch

    from paper_2303_02543_gb300 import inputs
    from paper_2303_02543_gb300 import jacobi as J
    torch.cuda.set_device(local)
    stream = inputs.serving_stream(rate=rate, window_s=window, lo2=128, hi2=cap2d, lo3=32, hi3=cap3d)
    sopts = dict(refine_period=20)
    sopts.update(server_opts or {})
    srv = J.Server("f32_refine", budget_bytes=budget, max_slots=256, **sopts)
    t0 = time.perf_counter()
    tickets = []
    for a in stream:
        now = time.perf_counter() - t0
        if a.t > now:
            time.sleep(a.t - now)
        tickets.append((srv.submit(a.problem, 1e-8, 20 * 10 ** 7), a.problem, a.t))
    # every request is done, or the deadline has passed; then each ticket is
    # polled once without blocking (a long solve early in the stream must not
    # hide the later ones that finished)
    deadline = t0 + window + grace
    while time.perf_counter() < deadline:
        s_ = srv.stats()
        if s_["completed"] + s_["rejected"] >= len(tickets):
            break
        time.sleep(0.05)
    lat, lups, censored, failed = [], 0.0, 0, 0
    waited = []  # censored requests: arrival to poll, seconds
    for t, p, t_arr in tickets:
        r = srv.poll(t, want_field=False)
        if r is None:
            censored += 1
            waited.append(time.perf_counter() - t0 - t_arr)
            continue
        st, sw, rel, secs, _ = r
        if st != J.OK:
            failed += 1
        lat.append(secs)
        lups += p.points * sw
    wall = time.perf_counter() - t0
    stats = srv.stats()
    srv.close()
    lat.sort()
    every = sorted(lat + waited)

    def pct(q, xs=lat):
        return xs[min(len(xs) - 1, int(q * len(xs)))] * 1e3 if xs else None
    return {"offered_rate": rate, "window_s": window, "requests": len(tickets), "completed": len(lat),
            "censored": censored, "not_ok": failed, "completed_per_s": len(lat) / wall, "p50_ms": pct(0.5),
            "p99_ms": pct(0.99), "p50_ms_all_lower_bound": pct(0.5, every),
            "p99_ms_all_lower_bound": pct(0.99, every), "glups": lups / wall / 1e9, "steps": stats["steps"],
            "evictions": stats["evictions"], "resumed": stats["resumed"],
            "config": {"cap2d": cap2d, "cap3d": cap3d, "dtype": "f32_refine", "tol": 1e-8,
                       "grace_s": grace, "budget_gib": budget / (1 << 30), "server_options": sopts}}


def run_serving(args, rank, world, local):
    """Poisson arrivals over a bounded window into the continuous-batching
    server; 2D and 3D solves (sizes capped, labelled), each to 1e-8."""
    sopts = {}
    for kv in filter(None, args.server_opts.split(",")):
        k, v = kv.split("=")
        sopts[k.strip()] = int(v)
    leg = serving_leg(args.rate, args.window, args.cap2d, args.cap3d, local, sopts,
                      budget=int(args.budget_gib * (1 << 30)), grace=args.grace)
    if rank == 0:
        full = args.cap2d >= 4096 and args.cap3d >= 256
        leg["config"]["note"] = ("configured sizes (2D 128^2-4096^2, 3D 32^3-256^3)" if full
                                 else "sizes capped (full 4096^2 solves take ~1 h each)")
        print(json.dumps({"metric": "serving: p50/p99 solve latency (ms) and aggregate GLUP/s",
                          "workload": "serving", "higher_is_better": False, "data": "synthetic", **leg}),
              flush=True)


def main():
    args = parse()
    rank, world, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload.startswith("tts"):
        run_tts(args, rank, world, local)
    elif args.workload == "batched":
        run_batched(args, rank, world, local)
    elif args.workload == "paper3d_od":
        run_paper3d_od(args, rank, world, local)
    elif args.workload == "serving":
        run_serving(args, rank, world, local)
    else:
        run_ours(args, rank, world, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
