#!/usr/bin/env python
"""Throughput of the N-phase phase-field LB time step on one GB300.

Workload: N = 5 phases on a 2048 x 2048 periodic D2Q9 grid (two horizontal
tanh interfaces stacking phases 1-3 plus 16 seeded drops of phases 4-5,
seeded sigma in [5e-4, 2e-3], M = 0.05, tau = 0.7), FP32 storage. A step is
one time step of the whole grid (one fused kernel launch). Metric: MLUPS =
node updates per second, each update advancing all N LB equations.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0). Multi-GPU runs are independent replicas (the
method's grid is not sharded here): value = sum over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS (node updates per second, all N LB equations)"
WORKLOAD = ("N=5 droplets and interfaces, D2Q9 2048x2048 periodic, "
            "FP32 storage")
SEED = 4
BYTES_PER_VALUE = {"fp64": (8, 8), "fp32": (4, 4), "bf16": (2, 4),
                   "fp16": (2, 4)}


def alg_bytes_per_node(N: int, prec: str) -> int:
    """Algorithmic bytes per node-step: read + write of 9(N-1) h + 8 g +
    (N-1) phi_prev + 2 u_prev; the 8N moving populations in the storage
    type, the N-1 rest slots and the N+1 state values in the arithmetic
    type. The 16-bit forms also carry p(t-1), which their g storage is
    relative to."""
    s_mov, s_rest = BYTES_PER_VALUE[prec]
    extra = 1 if s_mov == 2 else 0
    return 2 * (8 * N * s_mov + (N - 1) * s_rest + (N + 1 + extra) * s_rest)


# FP64 operations one node-step executes in the FP64 form at N=5 (ncu
# instruction counts of the step kernel on the 1024x1024 droplets and
# interfaces case, per node: 187 DFMA counted twice, 180.5 DADD, 125 DMUL;
# profiles/tile_kernel_fp64_n5_1024.md).
FP64_FLOP_PER_NODE_N5 = 679.5
# FP64 ALU peak derived from the GB300's unit counts and clock: 152 SMs x
# 2 FP64 FMA lanes per SM per clock x 2 FLOP x 2070 MHz = 1.2586 TFLOP/s.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def traffic_from_profiles(kernel_tag: str):
    """Per-launch DRAM bytes recorded from an ncu capture of this kernel
    (profiles/traffic.txt, `tag = bytes`), or None."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    try:
        with open(path) as f:
            for line in f:
                line = line.split("#")[0].strip()
                if "=" in line:
                    k, v = line.split("=", 1)
                    if k.strip() == kernel_tag:
                        return float(v)
    except OSError:
        pass
    return None


# Wall-clock windows of the timed GPU loops of this run, for the clocks record.
GPU_WINDOWS: list = []


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while alive."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,"
              "clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.samples = []
        self.proc = None
        self.window = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.time(), line.strip()))

    def mark(self, t0, t1):
        self.window = (t0, t1)

    def summary_windows(self, wins):
        """summary() over the union of several (t0, t1) windows."""
        keep = []
        for (t, line) in list(self.samples):
            for (a, b) in wins:
                if a is None or a - 0.05 <= t <= b + 0.05:
                    keep.append((t, line))
                    break
        saved, self.samples = self.samples, keep
        try:
            return self.summary()
        finally:
            self.samples = saved

    def summary(self, t0=None, t1=None):
        """Median SM clock, max clock and throttle reasons of the samples
        taken between t0 and t1 (all samples if None)."""
        t0 = -1e30 if t0 is None else t0
        t1 = 1e30 if t1 is None else t1
        sel = [s for (t, s) in list(self.samples) if t0 - 0.05 <= t <= t1 + 0.05]
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        for s in sel:
            parts = [x.strip() for x in s.split(",")]
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [],
                    "samples": 0}
        # The headline's timed region can be a few milliseconds (one
        # sample at most), so the record covers the whole GPU run that
        # holds it: the forms' warm-up and timed steps back to back. The
        # samples inside the headline's own timed window are counted too.
        wins = GPU_WINDOWS or [(None, None)]
        out = self.summary_windows(wins)
        out["window"] = ("the timed loops of every form of this run (the "
                         "headline, the other storage forms, the ensemble, "
                         "D3Q15)")
        if self.window:
            inner = self.summary(*self.window)
            out["timed_window"] = {"samples": inner["samples"],
                                   "sm_mhz": inner["sm_mhz"],
                                   "reasons": inner["reasons"]}
        return out


def accept_sigma(N=None):
    """sigma draws whose lambda (from the library's host setup) is well
    conditioned: smallest eigenvalue > 1e-3 largest."""
    from paper_1904_12553_gb300 import LbmError, lbm_nphase_derive, workloads as W

    def ok(sig):
        try:
            d = lbm_nphase_derive(W.base_params(sig.shape[0], 4, 4, sig))
        except LbmError:
            return False
        return d["lambda_eig_min"] > 1e-3 * d["lambda_eig_max"]
    return ok


def max_over_ranks(value: float, dist, device) -> float:
    """Largest value over all ranks (the slowest replica sets the time)."""
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(world: int, nodes: int, steps: int, ms_max: float) -> float:
    """Whole-job MLUPS of `world` replicas of a grid of `nodes` nodes, each
    taking `steps` steps, timed by the slowest replica."""
    return world * nodes * steps / (ms_max / 1e3) / 1e6


def make_workload(prec="fp32", n=2048, accept=None):
    from paper_1904_12553_gb300 import workloads as W
    return W.droplets_interfaces(seed=SEED, n=n, precision=prec,
                                 accept=accept)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def time_form(w, prec, steps, warmup, dist=None, segments=None):
    """Device time of `steps` back-to-back time steps (CUDA events on the
    solver's stream), max over ranks. If `segments` is a list, the steps are
    also split into five equal runs bracketed by events and their times (ms)
    are appended to it."""
    import torch
    from paper_1904_12553_gb300 import Solver

    s = Solver({**w.params, "precision": prec})
    s.init(w.c0, w.u0, w.p0)
    for _ in range(warmup):
        s.step(1)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    nseg = 5 if segments is not None and steps >= 5 else 1
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(nseg + 1)]
    bounds = [steps * i // nseg for i in range(nseg + 1)]
    wall0 = time.time()
    ev[0].record(s.stream)
    for i in range(nseg):
        for _ in range(bounds[i + 1] - bounds[i]):
            s.step(1)
        ev[i + 1].record(s.stream)
    torch.cuda.synchronize()
    wall1 = time.time()
    GPU_WINDOWS.append((wall0, wall1))
    ms = ev[0].elapsed_time(ev[-1])
    if segments is not None and nseg > 1:
        segments.extend((ev[i].elapsed_time(ev[i + 1]), bounds[i + 1] - bounds[i])
                        for i in range(nseg))
    if dist:
        dist.barrier()
        ms = max_over_ranks(ms, dist, "cuda")
    mass, ke, _ = s.diagnostics()
    kernel = s.step_kernel
    s.close()
    return ms, (wall0, wall1), mass, ke, kernel


def e2e_run(w, prec, steps):
    """Whole job through the C ABI with host buffers: H2D of the initial
    fields from pinned memory (inside lbm_nphase_init), the steps, and the
    D2H of phi, c, u, p, rho into pinned memory (lbm_nphase_moments)."""
    import torch
    from paper_1904_12553_gb300 import (Solver, lbm_nphase_init,
                                        lbm_nphase_moments, lbm_nphase_step)

    s = Solver({**w.params, "precision": prec})
    N, V = s.N, s.V
    c_host = torch.from_numpy(w.c0).pin_memory()
    outs = {k: torch.empty(n * V, dtype=torch.float64).pin_memory()
            for k, n in (("phi", N - 1), ("c", N), ("u", 2), ("p", 1),
                         ("rho", 1))}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lbm_nphase_init(s.handle, c_host.data_ptr(), None, w.p0)
    for _ in range(steps):
        lbm_nphase_step(s.handle, 1)
    lbm_nphase_moments(s.handle, outs["phi"].data_ptr(), outs["c"].data_ptr(),
                       outs["u"].data_ptr(), outs["p"].data_ptr(),
                       outs["rho"].data_ptr())
    torch.cuda.synchronize()
    t = time.perf_counter() - t0
    s.close()
    h2d = N * V * 8
    d2h = (2 * N + 3) * V * 8
    return V * steps / t / 1e6, h2d / steps, d2h / steps


def d3q15_run(n=256, steps=100, prec="fp32"):
    """D3Q15 (three dimensions): three phases, two sphere drops R = n/6 in a
    periodic n^3 box, z-marching 3-D kernel; FP32 storage, or 16-bit
    storage relative to the advective and pressure parts of the
    equilibrium."""
    import torch
    from paper_1904_12553_gb300 import Solver, workloads as W

    w = W.sphere_drops3(n=n, N=3, R=n / 6.0, precision=prec)
    s = Solver(w.params)
    kernel = s.step_kernel
    s.init(w.c0)
    s.step(3)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    wall0 = time.time()
    e0.record(s.stream)
    for _ in range(steps):
        s.step(1)
    e1.record(s.stream)
    torch.cuda.synchronize()
    GPU_WINDOWS.append((wall0, time.time()))
    ms = e0.elapsed_time(e1) / steps
    s.close()
    N, V = 3, w.V
    if prec == "fp32":
        B = 2 * 4 * (15 * (N - 1) + 14 + (N - 1) + 3)
    else:
        # 14 moving h per phase and 14 g in 16 bits; d_0, phi(t-1), u(t-1),
        # p(t-1)
        B = 2 * (2 * (14 * (N - 1) + 14) + 4 * (2 * (N - 1) + 4))
    peak, _ = peaks()
    return {"workload": f"N=3 two spheres, D3Q15 {n}^3 periodic, {prec.upper()}",
            "mlups": V / (ms / 1e3) / 1e6, "ms_per_step": ms,
            "alg_bytes_per_node": B,
            "hbm_frac": B * V / (ms / 1e3) / 1e9 / peak,
            "kernel": kernel}


def batch_run(steps=50, ncases=256):
    """Batched ensemble (256 seeded static-drop / lens cases, sides 64..512,
    N = 3..5, FP32): one persistent launch per step under a CUDA graph with
    the autotuned schedule, against the same cases stepped one by one."""
    import torch
    from paper_1904_12553_gb300 import Batch, Solver, workloads as W

    cases = W.ensemble(seed=5, ncases=ncases, accept=accept_sigma(None))
    nodes = sum(w.V for w in cases)
    b = Batch([w.params for w in cases])
    for i, w in enumerate(cases):
        b.init(i, w.c0, w.u0)
    b.autotune(3)
    for i, w in enumerate(cases):
        b.init(i, w.c0, w.u0)
    b.step(2)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    wall0 = time.time()
    e0.record(b.stream)
    b.step(steps)
    e1.record(b.stream)
    torch.cuda.synchronize()
    GPU_WINDOWS.append((wall0, time.time()))
    ms_b = e0.elapsed_time(e1)
    sched = b.schedule()
    b.close()
    solvers = []
    for w in cases:
        s = Solver(w.params)
        s.init(w.c0, w.u0)
        s.step(1)
        solvers.append(s)
    torch.cuda.synchronize()
    e0.record(solvers[0].stream)
    for _ in range(steps):
        for s in solvers:
            s.step(1)
    e1.record(solvers[0].stream)
    torch.cuda.synchronize()
    ms_1 = e0.elapsed_time(e1)
    for s in solvers:
        s.close()
    bytes_step = sum(alg_bytes_per_node(w.params["N"], "fp32") * w.V
                     for w in cases)
    peak, _ = peaks()
    return {"cases": ncases, "nodes": nodes, "steps": steps,
            "batched_mlups": nodes * steps / (ms_b / 1e3) / 1e6,
            "batched_hbm_frac": bytes_step * steps / (ms_b / 1e3) / 1e9 / peak,
            "alg_bytes_per_step": bytes_step,
            "one_by_one_mlups": nodes * steps / (ms_1 / 1e3) / 1e6,
            "batched_ms_per_step": ms_b / steps,
            "one_by_one_ms_per_step": ms_1 / steps,
            "schedule": {"tile_height": sched["tile_height"],
                         "schedule": Batch.SCHEDULES[sched["schedule"]],
                         "ctas": sched["ctas"], "chunk": sched["chunk"],
                         "kernel": ("pipelined (TMA)" if sched["pipelined"]
                                    else "generic tile")},
            "kernel_launches_per_step": {"batched": 1,
                                         "one_by_one": ncases}}


def cpu_baseline(steps=3):
    """The FP64 oracle on the full workload, timed on this host's cores in a
    fresh process (OpenMP over rows): all cores over `steps` steps, and one
    thread over one step."""
    cores = os.cpu_count() or 1
    out = _oracle_run(steps, cores)
    one = _oracle_run(1, 1)
    if one.get("value") is not None:
        out["single_thread"] = one
    return out


def _oracle_run(steps, cores):
    code = (
        "import sys, time, json\n"
        f"sys.path.insert(0, {ROOT!r}); sys.path.insert(0, {os.path.join(ROOT, 'oracle')!r})\n"
        "import numpy as np, oracle\n"
        "from paper_1904_12553_gb300 import workloads as W\n"
        "def ok(sig):\n"
        "    ev = np.linalg.eigvalsh(oracle.lam(W.base_params(5, 4, 4, sig)))\n"
        "    return ev[0] > 1e-3 * ev[-1]\n"
        f"w = W.droplets_interfaces(seed={SEED}, n=2048, precision='fp64', accept=ok)\n"
        "s = oracle.OracleSim(w.params); s.init(w.c0)\n"
        "s.step(1)\n"
        "t = time.perf_counter()\n"
        f"s.step({steps})\n"
        "t = time.perf_counter() - t\n"
        f"print(json.dumps({{'seconds': t, 'mlups': w.V * {steps} / t / 1e6}}))\n")
    env = dict(os.environ, OMP_NUM_THREADS=str(cores))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True,
                       text=True, env=env, timeout=1800)
    if r.returncode != 0:
        return {"value": None, "unit": "MLUPS", "cores": cores,
                "kind": "oracle", "error": r.stderr[-300:]}
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": d["mlups"], "unit": "MLUPS", "cores": cores,
            "kind": "oracle",
            "sample": f"FP64 oracle, {steps} time steps of the full "
                      f"2048x2048 N=5 grid after one untimed step "
                      f"({d['seconds']:.1f} s)"}


def segment_summary(segs, V):
    """Best and median rate over the timed region's five equal runs."""
    if not segs:
        return None
    rates = [V * n / (t / 1e3) / 1e6 for t, n in segs]
    return {"n": len(rates), "mlups_best": max(rates),
            "mlups_median": statistics.median(rates),
            "mlups_worst": min(rates)}


def run_ours(args, dist, rank, world):
    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    from paper_1904_12553_gb300 import build
    if rank == 0:
        build.build()
    if dist:
        dist.barrier()
    w = make_workload("fp32", n=args.n, accept=accept_sigma(5))
    N, V = w.params["N"], w.V
    sampler = ClockSampler(local) if rank == 0 else None
    segs = []
    ms, (wa, wb), mass, ke, kernel = time_form(w, "fp32", args.steps,
                                               args.warmup, dist, segs)
    if sampler:
        sampler.mark(wa, wb)
    ms_step = ms / args.steps
    value = replica_value(world, V, args.steps, ms)
    if rank != 0:
        return
    peak, peak_kind = peaks()
    B = alg_bytes_per_node(N, "fp32")
    achieved = B * V / (ms_step / 1e3) / 1e9
    if args.kernel_only:
        clocks = sampler.stop() if sampler else None
        print(json.dumps({"metric": METRIC, "value": value, "unit": "MLUPS",
                          "n_gpus": world, "steps": args.steps,
                          "warmup": args.warmup, "ms_per_step": ms_step,
                          "kernel_only": True, "nx": w.params["nx"],
                          "kernel": kernel,
                          "hbm_frac": B * V / (ms_step / 1e3) / 1e9 / peak,
                          "clocks": clocks}), flush=True)
        return
    forms = {}
    if not args.quick:
        for prec, k in (("bf16", args.steps), ("fp16", args.steps),
                        ("fp64", max(10, args.steps // 20))):
            fms, _, fmass, _, fkernel = time_form(w, prec, k,
                                                  min(args.warmup, 5))
            fstep = fms / k
            fB = alg_bytes_per_node(N, prec)
            forms[prec] = {
                "mlups": V / (fstep / 1e3) / 1e6, "ms_per_step": fstep,
                "alg_bytes_per_node": fB, "kernel": fkernel,
                "hbm_frac": fB * V / (fstep / 1e3) / 1e9 / peak}
            if prec == "fp64" and N == 5:
                tf = FP64_FLOP_PER_NODE_N5 * V / (fstep / 1e3) / 1e12
                forms[prec]["roofline"] = {
                    "bound": "alu", "achieved": tf, "unit": "TFLOP/s",
                    "peak": FP64_PEAK_TFLOPS, "frac": tf / FP64_PEAK_TFLOPS,
                    "flop_per_node": FP64_FLOP_PER_NODE_N5,
                    "peak_kind": "derived (152 SMs x 2 FP64 FMA/clk x "
                                 "2070 MHz)"}
    if not args.quick:
        forms["batch"] = batch_run()
        for prec3 in ("fp32", "bf16", "fp16"):
            forms["d3q15_" + prec3] = d3q15_run(prec=prec3)
    e2e_v, h2d, d2h = e2e_run(w, "fp32", args.steps)
    clocks = sampler.stop() if sampler else None
    cpu = cpu_baseline() if (world == 1 and not args.quick) else None
    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic (seeded initial condition)",
        "config": {"workload": WORKLOAD, "N": N, "nx": w.params["nx"],
                   "ny": w.params["ny"], "precision": "fp32", "seed": SEED,
                   "l2": "state (%.2f GB) larger than L2, no flush"
                         % (B / 2 * V / 1e9),
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "kernel": kernel},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak,
                     "peak_kind": peak_kind,
                     "alg_bytes_per_node": B,
                     "traffic": traffic_from_profiles("tile_kernel_tma_fp32_n5_2048")},
        # through the C ABI from pinned host memory: init (H2D), the same
        # K steps, moments (D2H); at small K the init and read-back dominate
        "e2e": {"value": e2e_v, "unit": "MLUPS", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "steps": args.steps},
        "gpu_launches": args.steps,
        "segments": segment_summary(segs, V),
        # the same rate counted per LB equation (N per node update)
        "equation_mlups": value * N,
        "clocks": clocks,
        "forms": forms,
        "check": {"mass": list(map(float, mass)), "ke": float(ke)},
    }
    if cpu:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)


def run_only(args):
    """One form alone (for profiler captures): N=5 droplets and interfaces
    at side --n (2-D forms), the ensemble, or an --n^3 D3Q15 box."""
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    from paper_1904_12553_gb300 import build
    build.build()
    if args.only == "batch":
        out = batch_run(steps=args.steps)
    elif args.only == "d3q15":
        out = d3q15_run(n=args.n if args.n != 2048 else 128, steps=args.steps,
                        prec=args.d3_prec)
    else:
        w = make_workload(args.only, n=args.n, accept=accept_sigma())
        ms, _, _, _, kernel = time_form(w, args.only, args.steps, args.warmup)
        B = alg_bytes_per_node(5, args.only)
        peak, _ = peaks()
        step = ms / args.steps
        out = {"form": args.only, "nx": args.n, "kernel": kernel,
               "mlups": w.V / (step / 1e3) / 1e6, "ms_per_step": step,
               "hbm_frac": B * w.V / (step / 1e3) / 1e9 / peak}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------
# Reference arm: the FP64 CPU oracle as it stands
# ---------------------------------------------------------------------------

def run_reference(args, rank):
    if rank != 0:
        return
    sys.path.insert(0, os.path.join(ROOT, "oracle"))
    cores = os.cpu_count() or 1
    os.environ["OMP_NUM_THREADS"] = str(cores)
    import numpy as np
    import oracle
    from paper_1904_12553_gb300 import workloads as W

    def ok(sig):
        ev = np.linalg.eigvalsh(oracle.lam(W.base_params(5, 4, 4, sig)))
        return ev[0] > 1e-3 * ev[-1]

    # Each step: one oracle time step on an n x n window of the workload,
    # n chosen so that all warm-up and timed steps take about two minutes.
    probe = W.droplets_interfaces(seed=SEED, n=256, precision="fp64",
                                  accept=ok)
    s = oracle.OracleSim(probe.params)
    s.init(probe.c0)
    t = time.perf_counter()
    s.step(2)
    rate = 2 * probe.V / (time.perf_counter() - t)
    s.close()
    per_step = 120.0 / max(1, args.steps + args.warmup)
    n = int(math.sqrt(rate * per_step))
    n = max(64, min(2048, n - n % 32))
    w = W.droplets_interfaces(seed=SEED, n=n, precision="fp64", accept=ok,
                              ndrops=max(1, int(16 * (n / 2048) ** 2)))
    s = oracle.OracleSim(w.params)
    s.init(w.c0)
    s.step(args.warmup)
    t = time.perf_counter()
    s.step(args.steps)
    sec = time.perf_counter() - t
    s.close()
    value = w.V * args.steps / sec / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "MLUPS",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": sec / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded initial condition)",
        "config": {"workload": WORKLOAD, "N": 5, "nx": 2048, "ny": 2048,
                   "precision": "fp32", "seed": SEED},
        "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": cores,
                         "kind": "oracle",
                         "sample": f"FP64 oracle time steps on a {n}x{n} "
                                   "window of the workload, one per step"},
        "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--quick", action="store_true",
                    help="skip the other storage forms and the CPU baseline")
    ap.add_argument("--kernel-only", action="store_true",
                    help="time the FP32 step kernel only (profiling runs)")
    ap.add_argument("--only", default=None,
                    choices=["fp32", "bf16", "fp16", "fp64", "batch", "d3q15"],
                    help="time one form alone and print its line "
                         "(profiling captures)")
    ap.add_argument("--d3-prec", default="fp32", choices=["fp32", "bf16", "fp16"],
                    help="storage form of --only d3q15")
    ap.add_argument("--n", type=int, default=2048,
                    help="grid side (2048 is the benchmark workload; smaller "
                         "sides are for profiling captures)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if world > 1:
        import torch.distributed as dist_
        dist_.init_process_group("nccl")
        dist = dist_
    if args.only:
        run_only(args)
        return
    try:
        run_ours(args, dist, rank, world)
    finally:
        if dist:
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
