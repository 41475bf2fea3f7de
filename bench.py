#!/usr/bin/env python
"""Benchmark of the Feynman-Kac exit-probability march on GB300.

One step = one whole march (fk_solve) of the workload: for the default
``cellular_1025x513`` that is Scheme 1 over 2000 time steps on a 1025 x 513
mesh with 6 x 6 Gauss-Hermite points, FP32.  The metric is
node-quadrature updates per second: interior nodes x Q^2 x time steps per
second of march, summed over all ranks (each rank marches its own instance:
independent problems, weak scaling, no collective on the data path).

Printed (rank 0, one JSON line): value (inputs resident on the device),
e2e (the same through the public API with host buffers and host<->device
copies inside the timed region), roofline of the dominant kernel, the CPU
oracle timed on the host cores (cpu_baseline), clocks sampled during the
timed region, and the number of our kernel launches in the timed region.

``--impl reference`` times the FP64 CPU oracle on the host cores instead
(bounded samples of the same workload); it never touches the GPU.
"""
from __future__ import annotations

import argparse
import hashlib
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

import numpy as np  # noqa: E402

import fk_inputs  # noqa: E402

METRIC = "node-quadrature updates/s & HBM GB/s (2D, 36-pt GH, FP32/FP64); adjoint/forward"
UNIT = "node-quadrature updates/s"
L2_FLUSH_BYTES = 512 << 20          # > 129 MB L2
FLOP_PER_UPDATE = 26                # 13 multiply-adds per query: 12 Hermite terms + the weighted sum
FLOP_PER_UPDATE_3D = 66             # 33 multiply-adds: 8 corners x (value + 3 partials) + the sum
PROFILE_DIR = os.path.join(ROOT, "profiles")
HBM_FALLBACK_GBS = 6800.0


def hbm_peak():
    """Measured copy bandwidth of the GB300s, else the fallback."""
    try:
        v = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
        return v, "measured"
    except (OSError, ValueError, KeyError):
        return HBM_FALLBACK_GBS, "fallback"


def measure_alu_peaks(fk, stream, local_rank: int) -> dict:
    """FP32 and FP64 fused multiply-add throughput of this GPU, measured with
    the library's register-resident FMA-chain kernel (CUDA events), with the
    SM clock sampled while it runs.  The FP32 peak is the larger of the
    scalar and the packed f32x2 rates (the step kernels use both forms)."""
    import torch
    props = torch.cuda.get_device_properties(local_rank)
    clk = ClockSampler(local_rank)
    clk.start()
    f32 = fk.measure_fma_rate("fp32", False, 0.25, stream)
    f32x2 = fk.measure_fma_rate("fp32", True, 0.25, stream)
    f64 = fk.measure_fma_rate("fp64", False, 0.25, stream)
    clocks = clk.stop()
    return {"fp32_tflops": max(f32, f32x2) / 1e12, "fp32_scalar_tflops": f32 / 1e12,
            "fp32_packed_tflops": f32x2 / 1e12, "fp64_tflops": f64 / 1e12,
            "sm_count": props.multi_processor_count, "sm_mhz_median": clocks.get("sm_mhz"),
            "how": "fk_measure_fma_rate: 8 independent FMA chains per thread on every thread "
                   "slot of every SM, CUDA-event timed (about 0.25 s per precision)"}


def csr_bytes_per_step(w, nnz: int) -> float:
    """Algorithmic HBM bytes of one CSR step: the matrix stream (one record
    of 16 B in FP32, 32 B in FP64, per three stored entries: a node and its
    u, h u_x and h u_y weights), row offsets, exit constants, u^{n+1} read
    by the slope pass, the interleaved {u, h u_x, h u_y, 0} written by it and
    read once, and u^n written."""
    J = 1
    for n in w["n"]:
        J *= n
    e = 4 if w["precision"] == "fp32" else 8
    return (nnz // 3) * 4 * e + 8.0 * (J + 1) + e * J * (1 + 1 + 4 + 4 + 1)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="cellular_1025x513")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the FP64 march and the adjoint beside the headline march")
    # profiling aids: a smaller case of the same workload (not a benchmark line)
    ap.add_argument("--time-steps", type=int, default=None,
                    help="override the workload's number of time steps")
    ap.add_argument("--grid", type=int, nargs="+", default=None, metavar="N",
                    help="override the workload's mesh")
    ap.add_argument("--precision", choices=["fp32", "fp64"], default=None,
                    help="override the workload's precision")
    return ap.parse_args()


def headline(args) -> bool:
    """The workload the metric is quoted on, unmodified."""
    return (args.workload == "cellular_1025x513" and not args.time_steps and not args.grid
            and not args.precision)


def workload_of(args):
    over = {}
    if args.time_steps:
        over["n_steps"] = args.time_steps
    if args.grid:
        over["n"] = tuple(args.grid)
    if args.precision:
        over["precision"] = args.precision
    return fk_inputs.workload(args.workload, **over)


def units_per_solve(w) -> float:
    """Node-quadrature updates of one march: the updated nodes (interior
    ones; a periodic x axis has n - 1 distinct columns, all updated; the
    runaway model also updates the nodes of its mirroring faces, every xi
    node and r = 0) times the points per node times the steps."""
    updated = 1
    runaway = w["family"] in ("runaway", "runaway_quench")
    for m, n in enumerate(w["n"]):
        if m == 0 and w.get("periodic_x"):
            updated *= n - 1
        elif runaway and m > 0:
            updated *= n if m == 1 else n - 1
        else:
            updated *= n - 2
    return float(updated) * (w["q"] ** len(w["n"])) * w["n_steps"]


def l2_note(w) -> str:
    """How L2 is handled between timed marches, and whether the field fits."""
    mb = 2 * math.prod(w["n"]) * (4 if w["precision"] == "fp32" else 8) / 1e6
    where = ("stay L2-resident" if mb < 100 else "exceed the 129 MB L2")
    return (f"flushed (512 MB write) before every timed march; the two {mb:.0f} MB fields "
            f"{where} across the {w['n_steps']} time steps of one march")


def hbm_bytes_per_solve(w) -> float:
    """Algorithmic HBM traffic of the march: read u^{n+1} and write u^n once
    per time step (the matrix-free path keeps no other per-node array)."""
    J = 1
    for n in w["n"]:
        J *= n
    elem = 4 if w["precision"] == "fp32" else 8
    return 2.0 * J * elem * w["n_steps"]


# ------------------------------------------------------------- clocks ----
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------ oracle -----
def oracle_rate(w, max_seconds: float = 20.0):
    """FP64 CPU oracle on the host cores over a bounded sample of the
    workload's march (consecutive time steps from the terminal field)."""
    from oracle import fk_oracle as O
    fam = {"const_drift": O.CONST_DRIFT, "cellular_flow": O.CELLULAR_FLOW,
           "paper_cellular": O.PAPER_CELLULAR, "runaway": O.RUNAWAY,
           "runaway_quench": O.RUNAWAY_QUENCH}[w["family"]]
    g = O.Grid(tuple(w["n"]), tuple(w["lo"]), tuple(w["hi"]), int(w.get("periodic_x", False)),
               fk_inputs.axes_of(w))
    cores = os.cpu_count() or 1
    per_step = units_per_solve(w) / w["n_steps"]
    t = time.perf_counter()
    O.march(g, fam, list(w["params"]), w["q"], w["dt"], w["n_steps"], w["n_steps"] - 1,
            nthreads=cores)
    one = time.perf_counter() - t
    k = max(1, min(w["n_steps"] - 1, int(max_seconds / max(one, 1e-6))))
    t = time.perf_counter()
    O.march(g, fam, list(w["params"]), w["q"], w["dt"], w["n_steps"], w["n_steps"] - k,
            nthreads=cores)
    dt = time.perf_counter() - t
    return {"value": per_step * k / dt, "unit": UNIT, "cores": cores if O.has_openmp() else 1,
            "kind": "oracle",
            "sample": f"{k} of {w['n_steps']} time steps of {'x'.join(str(v) for v in w['n'])}"
                      f", FP64, OpenMP over nodes ({dt:.1f} s)"}


def run_reference(args, rank: int):
    if rank != 0:
        return
    from oracle import fk_oracle as O
    O.build()
    fams = {"const_drift": O.CONST_DRIFT, "cellular_flow": O.CELLULAR_FLOW,
            "paper_cellular": O.PAPER_CELLULAR, "runaway": O.RUNAWAY,
            "runaway_quench": O.RUNAWAY_QUENCH}
    # one benchmark step of the reference arm = one time step of the march
    # (of every instance, for the batched sweep): a bounded sample of the
    # workload, so that K + W steps take seconds to a minute
    ws = (fk_inputs.batch(args.workload) if args.workload in fk_inputs.BATCHES
          else [fk_inputs.workload(args.workload)])
    w = ws[0]
    cores = os.cpu_count() or 1
    per_step = sum(units_per_solve(x) / x["n_steps"] for x in ws)
    us = [None] * len(ws)
    times = []
    for s in range(args.warmup + args.steps):
        t = time.perf_counter()
        for b, x in enumerate(ws):
            n = x["n_steps"] - s
            g = O.Grid(tuple(x["n"]), tuple(x["lo"]), tuple(x["hi"]),
                       int(x.get("periodic_x", False)), fk_inputs.axes_of(x))
            us[b] = O.march(g, fams[x["family"]], list(x["params"]), x["q"], x["dt"], n, n - 1,
                            us[b], nthreads=cores)
        if s >= args.warmup:
            times.append(time.perf_counter() - t)
    sec = sum(times) / len(times)
    value = per_step / sec
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "grid": list(w["n"]), "q_per_dim": w["q"],
                       "dt": w["dt"], "step": "one time step of the march per benchmark step"},
            "cpu_baseline": {"kind": "oracle", "cores": cores if O.has_openmp() else 1,
                             "sample": f"{args.steps} time steps of "
                                       + (f"each of the {len(ws)} instances" if len(ws) > 1 else
                                          'x'.join(str(v) for v in w['n'])) + ", FP64",
                             "value": value, "unit": UNIT},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def sources_sha256(paths) -> str:
    """One digest over the given source files (repo-relative), in order."""
    h = hashlib.sha256()
    for rel in paths:
        h.update(open(os.path.join(ROOT, rel), "rb").read())
    return h.hexdigest()


def profile_traffic(kernel: str, workload: str):
    """DRAM bytes per launch of the kernel from the committed ncu summary,
    or None when a source it was built from changed since the capture."""
    try:
        prof = json.load(open(os.path.join(PROFILE_DIR, f"{kernel}_{workload}.json")))
        srcs = prof.get("sources") or [prof["source"]]
        if prof.get("source_sha256") != sources_sha256(srcs):
            return None
        return prof.get("dram_bytes_per_launch")
    except (OSError, ValueError, KeyError):
        return None


# ----------------------------------------------------------- batched -----
def run_batched(args, rank: int, world: int, local_rank: int):
    """The 64-instance sweep: one fk_solve_batched of all instances per
    benchmark step (the strategy its autotuner picks), with the persistent
    kernel forced and the plain march (one fk_solve per instance on the same
    stream) timed beside it."""
    import torch
    import paper_2104_14561_gb300 as fk
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    ws = fk_inputs.batch(args.workload)
    if args.time_steps:
        ws = [dict(x, n_steps=args.time_steps) for x in ws]
    plans = [fk.Plan(fk.PlanSpec(n=w["n"], lo=w["lo"], hi=w["hi"], family=w["family"],
                                 params=w["params"], q=w["q"], dt=w["dt"],
                                 n_steps=w["n_steps"], precision=w["precision"]))
             for w in ws]
    outs = [p.empty() for p in plans]
    units = sum(units_per_solve(w) for w in ws)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def timed(fn):
        return timed_ms(fn, stream, flush, args.warmup, args.steps)

    def batched():
        fk.solve_batched(plans, None, outs, stream=stream)

    def plain():
        for p, o in zip(plans, outs):
            p.solve(None, o, stream=stream)

    clk = ClockSampler(local_rank)
    clk.start()
    ms_b = timed(batched)
    clocks = clk.stop()
    mode = plans[0].info()["batch_mode"]
    if any(p.last_device_error() != 0 for p in plans):
        raise RuntimeError("device-side error in the batched march")
    os.environ["FK_BATCH_MODE"] = "persistent"
    try:
        ms_k = timed(batched)
    finally:
        del os.environ["FK_BATCH_MODE"]
    if plans[0].last_device_error() != 0:
        raise RuntimeError("device-side error in the persistent batched march")
    ms_p = timed(plain)
    grid = None
    nodes = sum(int(np.prod(w["n"])) for w in ws)
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": units / (ms_b * 1e-3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_b,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": args.workload, "instances": len(ws), "nodes": nodes,
                   "q_per_dim": 6, "time_steps": ws[0]["n_steps"], "dt": 1e-3,
                   "l2": "flushed (512 MB write) before every timed march"},
        "batch_mode": mode,
        "persistent_kernel": {"value": units / (ms_k * 1e-3), "ms_per_step": ms_k,
                              "how": "the cooperative persistent kernel, forced"},
        "plain_march": {"value": units / (ms_p * 1e-3), "ms_per_step": ms_p,
                        "how": f"{len(ws)} fk_solve calls (one CUDA graph each) on one stream"},
        "gpu_launches": args.steps * (sum(w["n_steps"] + 1 for w in ws) if mode == "streams"
                                      else 1 + len(ws)),
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    for p in plans:
        p.close()


# ----------------------------------------------------------- adjoint -----
def run_adjoint(args, rank: int, world: int, local_rank: int):
    """Adjoint workload: dL/d(A, eps, omega, D) and dL/du^N of the mean exit
    probability at T = 2 on 1025 x 513 (2000 FP32 steps, FP64 reduction),
    checkpoint every 50 steps.  One step = one fk_adjoint call (forward pass
    with checkpoints, segment recompute, backward pass); the forward march
    is timed beside it."""
    import torch
    import paper_2104_14561_gb300 as fk
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    w = workload_of(args)
    plan = fk.Plan(fk.PlanSpec(n=w["n"], lo=w["lo"], hi=w["hi"], family=w["family"],
                               params=w["params"], q=w["q"], dt=w["dt"], n_steps=w["n_steps"],
                               precision=w["precision"]))
    ny, nx = plan.shape
    cot = torch.zeros(plan.shape, dtype=torch.float64, device=dev)
    cot[1:-1, 1:-1] = 1.0 / ((nx - 2) * (ny - 2))
    out = plan.empty()
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    units = units_per_solve(w)

    def timed(fn):
        return timed_ms(fn, stream, flush, args.warmup, args.steps)

    clk = ClockSampler(local_rank)
    clk.start()
    ms_adj = timed(lambda: plan.adjoint(cot, None, checkpoint_every=50, stream=stream))
    clocks = clk.stop()
    ms_fwd = timed(lambda: plan.solve(None, out, stream=stream))
    dth, _ = plan.adjoint(cot, None, checkpoint_every=50)
    torch.cuda.synchronize()
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": units / (ms_adj * 1e-3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_adj,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "adjoint_1025x513", "grid": list(w["n"]), "q_per_dim": w["q"],
                   "time_steps": w["n_steps"], "checkpoint_every": 50,
                   "objective": "mean of u^0 over interior nodes",
                   "l2": "flushed (512 MB write) before every timed call"},
        "forward_ms": ms_fwd, "adjoint_over_forward": ms_adj / ms_fwd,
        "dtheta": [float(v) for v in dth.cpu()],
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    plan.close()


# ---------------------------------------------------------- horizons -----
def run_horizons(args, rank: int, world: int, local_rank: int):
    """Algorithm 1 workload: P(t_k, .) for every horizon k = 1..200 of the
    time-dependent flow on 1025 x 513 (FP32), one fk_solve_horizons call per
    step: N (N + 1) / 2 = 20100 field-steps, with all horizons still active
    at a step advanced by one launch.  The single march of N steps (the last
    horizon alone) is timed beside it."""
    import torch
    import paper_2104_14561_gb300 as fk
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    w = workload_of(args)
    plan = fk.Plan(fk.PlanSpec(n=w["n"], lo=w["lo"], hi=w["hi"], family=w["family"],
                               params=w["params"], q=w["q"], dt=w["dt"], n_steps=w["n_steps"],
                               precision=w["precision"]))
    N = w["n_steps"]
    out_all = torch.empty((N,) + plan.shape, dtype=plan.dtype, device=dev)
    out = plan.empty()
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    field_steps = N * (N + 1) // 2
    units = units_per_solve(w) / N * field_steps

    def timed(fn):
        return timed_ms(fn, stream, flush, args.warmup, args.steps)

    peaks = measure_alu_peaks(fk, stream, local_rank)
    clk = ClockSampler(local_rank)
    clk.start()
    ms_h = timed(lambda: plan.solve_horizons(None, out_all, stream=stream))
    clocks = clk.stop()
    ms_single = timed(lambda: plan.solve(None, out, stream=stream))
    torch.cuda.synchronize()
    if plan.last_device_error() != 0:
        raise RuntimeError("device-side error in the horizon march")
    info = plan.info()
    ms_max = max_over_ranks(ms_h)
    if rank != 0:
        plan.close()
        return
    flop = FLOP_PER_UPDATE * units
    peak = peaks["fp32_tflops"]
    achieved = flop / (ms_h * 1e-3) / 1e12
    line = {
        "metric": METRIC, "value": whole_job_rate(units, world, ms_max), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": args.workload, "grid": list(w["n"]), "q_per_dim": w["q"],
                   "horizons": N, "field_steps": field_steps, "dt": w["dt"],
                   "step_kernel": info["step_kernel"],
                   "l2": "flushed (512 MB write) before every timed call; the "
                         f"{2 * N * math.prod(w['n']) * 4 / 1e9:.1f} GB of fields exceed the L2"},
        "roofline": {"kernel": "k_step2dm (all horizons of a step per launch)", "bound": "alu",
                     "achieved": achieved, "peak": peak, "peak_source": "measured",
                     "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None},
        "alu_peaks": peaks,
        "single_march_ms": ms_single,
        "field_step_us": ms_h * 1e3 / field_steps,
        "single_step_us": ms_single * 1e3 / N,
        "gpu_launches": N + 1,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    plan.close()


def timed_ms(fn, stream, flush, warmup: int, steps: int) -> float:
    """Mean CUDA-event time (ms) of fn() on `stream` over `steps` calls after
    `warmup` untimed ones, with L2 flushed (a write larger than L2) before
    each timed call."""
    import torch
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            fn()
    stream.synchronize()
    ms = []
    with torch.cuda.stream(stream):
        for i in range(steps):
            flush.fill_(float(i))
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
    return sum(ms) / len(ms)


def plan_of(fk, w, **over):
    """A plan of workload w (entries of `over` replace the workload's)."""
    w = dict(w, **over)
    return fk.Plan(fk.PlanSpec(n=w["n"], lo=w["lo"], hi=w["hi"], family=w["family"],
                               params=w["params"], q=w["q"], dt=w["dt"], n_steps=w["n_steps"],
                               precision=w["precision"], path=w.get("path", "matrix_free"),
                               periodic_x=w.get("periodic_x", False),
                               axes=fk_inputs.axes_of(w)))


def fp64_line(fk, w, stream, flush, steps: int, peaks: dict) -> dict:
    """The same march in FP64 (the metric's FP64 half): whole marches timed
    with CUDA events, rate, algorithmic HBM bytes and the ALU roofline
    against the measured FP64 FMA rate."""
    plan = plan_of(fk, w, precision="fp64")
    out = plan.empty()
    ms = timed_ms(lambda: plan.solve(None, out, stream=stream), stream, flush, 1, steps)
    if plan.last_device_error() != 0:
        raise RuntimeError("device-side range check fired in the FP64 march")
    info = plan.info()
    plan.close()
    w64 = dict(w, precision="fp64")
    units = units_per_solve(w64)
    launch_ms = ms / w["n_steps"]
    flop_launch = FLOP_PER_UPDATE * units / w["n_steps"]
    achieved = flop_launch / (launch_ms * 1e-3) / 1e12
    peak = peaks["fp64_tflops"]
    kname = {"direct": "k_step2d", "window": "k_step2dw", "masked": "k_step2dm64"}.get(
        info.get("step_kernel"), info.get("step_kernel"))
    return {"value": units / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "steps": steps,
            "warmup": 1, "dtype": "f64",
            "hbm_gbs_algorithmic": hbm_bytes_per_solve(w64) / (ms * 1e-3) / 1e9,
            "roofline": {"kernel": kname, "bound": "alu", "achieved": achieved, "peak": peak,
                         "peak_source": "measured", "unit": "TFLOP/s", "frac": achieved / peak,
                         "traffic": profile_traffic(kname, "cellular_1025x513_fp64"),
                         "flop_per_launch": flop_launch, "launch_ms": launch_ms,
                         "step_kernel": info.get("step_kernel")}}


def adjoint_line(fk, w, stream, flush, steps: int, peaks: dict, forward_ms: float) -> dict:
    """The adjoint of the same march (the metric's adjoint/forward): dL/d(A,
    eps, omega, D) and dL/du^N of the mean of u^0 over the interior nodes,
    checkpoints every 50 steps, FP32 march with the FP64 gradient
    reduction.  One call = forward pass with checkpoints, segment recompute
    and the backward pass; the backward-step kernel's launches are timed
    live with CUDA events around each launch (fk_adjoint_kernel_times)."""
    import torch
    plan = plan_of(fk, w)
    ny, nx = plan.shape
    cot = torch.zeros(plan.shape, dtype=torch.float64, device=plan.device)
    cot[1:-1, 1:-1] = 1.0 / ((nx - 2) * (ny - 2))
    call = lambda: plan.adjoint(cot, None, checkpoint_every=50, stream=stream)  # noqa: E731
    ms = timed_ms(call, stream, flush, 1, steps)
    plan.adjoint_kernel_times(True)
    call()
    kms, launches = plan.adjoint_kernel_times(False)
    if plan.last_device_error() != 0:
        raise RuntimeError("device-side range check fired in the adjoint")
    info = plan.info()
    plan.close()
    units = units_per_solve(w)
    kname = {"scatter": "k_adj_scatter", "masked": "k_adj_masked"}.get(info.get("adjoint_kernel"),
                                                                       "?")
    launch_ms = kms / max(launches, 1)
    # the transposed step applies the transpose of the step's linear map: the
    # same 13 multiply-adds per node-quadrature update as the forward step
    flop_launch = FLOP_PER_UPDATE * units / w["n_steps"]
    achieved = flop_launch / (launch_ms * 1e-3) / 1e12
    peak = peaks["fp32_tflops"]
    return {"value": units / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "steps": steps,
            "warmup": 1, "adjoint_over_forward": ms / forward_ms, "checkpoint_every": 50,
            "objective": "mean of u^0 over interior nodes; gradients in (A, eps, omega, D) "
                         "and u^N",
            "backward_kernel_ms_per_launch": launch_ms, "backward_launches": launches,
            "roofline": {"kernel": kname, "bound": "alu", "achieved": achieved, "peak": peak,
                         "peak_source": "measured", "unit": "TFLOP/s", "frac": achieved / peak,
                         "traffic": profile_traffic(kname, "adjoint_1025x513"),
                         "flop_per_launch": flop_launch, "launch_ms": launch_ms}}


# ------------------------------------------------------------- ranks -----
def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The largest per-rank figure over all ranks (the value itself when the
    job has one rank)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, ms_max: float) -> float:
    """Throughput of the whole job when every rank marches its own instance
    (weak scaling): all ranks' units over the slowest rank's time."""
    return units_per_rank * world / (ms_max * 1e-3)


# --------------------------------------------------------------- ours ----
def run_ours(args, rank: int, world: int, local_rank: int):
    import torch
    import paper_2104_14561_gb300 as fk
    dist = None
    if world > 1:
        import torch.distributed as dist
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    w = workload_of(args)
    spec = fk.PlanSpec(n=w["n"], lo=w["lo"], hi=w["hi"], family=w["family"],
                       params=w["params"], q=w["q"], dt=w["dt"], n_steps=w["n_steps"],
                       precision=w["precision"], path=w["path"],
                       periodic_x=w.get("periodic_x", False), axes=fk_inputs.axes_of(w))
    plan = fk.Plan(spec)
    stream = torch.cuda.Stream(device=dev)
    out = plan.empty()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    units = units_per_solve(w)

    def barrier():
        if dist is not None:
            dist.barrier()

    peaks = measure_alu_peaks(fk, stream, local_rank)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            plan.solve(None, out, stream=stream)
    stream.synchronize()
    clk = ClockSampler(local_rank)
    clk.start()
    time.sleep(0.3)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for i in range(args.steps):
            flush.fill_(float(i))                 # evict L2 before each timed march
            starts[i].record(stream)
            plan.solve(None, out, stream=stream)
            ends[i].record(stream)
    torch.cuda.synchronize()
    barrier()
    wall = time.perf_counter() - wall0
    clocks = clk.stop()
    ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    ms_step = sum(ms) / len(ms)
    if plan.last_device_error() != 0:
        raise RuntimeError("device-side range check fired during the benchmark")
    ms_step_max = max_over_ranks(ms_step, dist, dev)
    value = whole_job_rate(units, world, ms_step_max)

    # end to end through the public API (fk_solve_host): pinned host in ->
    # device -> march -> host out, every copy inside the timed region
    host_in = torch.zeros(plan.shape, dtype=plan.dtype).pin_memory()
    for ax in range(host_in.dim()):  # the terminal indicator: 1 on the boundary
        host_in.narrow(ax, 0, 1).fill_(1.0)
        host_in.narrow(ax, host_in.shape[ax] - 1, 1).fill_(1.0)
    host_out = torch.empty(plan.shape, dtype=plan.dtype).pin_memory()
    e_ms = []
    with torch.cuda.stream(stream):
        for i in range(max(args.warmup, 1) + args.steps):
            flush.fill_(float(i))
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            plan.solve_host(host_in, host_out, stream=stream)  # copy in, march, copy out
            b.record(stream)
            b.synchronize()
            if i >= max(args.warmup, 1):
                e_ms.append(a.elapsed_time(b))
    e2e_value = whole_job_rate(units, world, max_over_ranks(sum(e_ms) / len(e_ms), dist, dev))
    field_bytes = int(host_in.numel() * host_in.element_size())

    # the metric's FP64 and adjoint/forward halves, on the headline workload
    extras = {}
    if rank == 0 and headline(args) and not args.no_extras:
        k = max(1, min(args.steps, 3))
        extras["fp64"] = fp64_line(fk, w, stream, flush, k, peaks)
        extras["adjoint"] = adjoint_line(fk, w, stream, flush, k, peaks, ms_step)

    if rank != 0:
        return
    info = plan.info()
    # one launch for every step (the persistent march), or a graph of
    # back-to-back step kernels
    persistent = info.get("march_mode") == "persistent"
    launch_ms = ms_step / w["n_steps"]
    if w["path"] == "csr":
        peak, peak_kind = hbm_peak()
        bytes_step = csr_bytes_per_step(w, info["csr_nnz"])
        achieved = bytes_step / (launch_ms * 1e-3) / 1e9
        roofline = {"kernel": "k_csr_slopes + k_csr_spmv (one time step)", "bound": "hbm",
                    "achieved": achieved, "peak": peak, "peak_source": peak_kind,
                    "unit": "GB/s", "frac": achieved / peak,
                    # (the SpMV's DRAM bytes, the dominant kernel's, from its summary,
                    # which covers the workload's own mesh only)
                    "traffic": (None if args.grid else
                                profile_traffic("k_csr_spmv", args.workload)),
                    "bytes_per_launch": bytes_step, "launch_ms": launch_ms,
                    "csr_nnz": info["csr_nnz"]}
    elif len(w["n"]) == 3:
        # two launches per time step (records, then the window sums); the
        # time of both is charged to the step, so the fraction is a floor
        flops_launch = FLOP_PER_UPDATE_3D * units / w["n_steps"]
        peak_flops = 1e12 * (peaks["fp32_tflops"] if w["precision"] == "fp32"
                             else peaks["fp64_tflops"])
        achieved = flops_launch / (launch_ms * 1e-3)
        roofline = {"kernel": "k_step3d (with k_rec3d: one time step)", "bound": "alu",
                    "achieved": achieved / 1e12, "peak": peak_flops / 1e12,
                    "peak_source": "measured", "unit": "TFLOP/s",
                    "frac": achieved / peak_flops,
                    "traffic": profile_traffic("k_step3d", args.workload),
                    "flop_per_launch": flops_launch, "launch_ms": launch_ms,
                    "window_rows": info.get("window_rows", 0),
                    "step_kernel": info.get("step_kernel")}
    else:
        if persistent:  # the whole march is one launch of the persistent kernel
            launch_ms = ms_step
        flops_launch = FLOP_PER_UPDATE * units / (1 if persistent else w["n_steps"])
        peak_flops = 1e12 * (peaks["fp32_tflops"] if w["precision"] == "fp32"
                             else peaks["fp64_tflops"])
        achieved = flops_launch / (launch_ms * 1e-3)
        kname = ({"resident": "k_march1d", "cluster": "k_march1d_cluster"}.get(
                     info.get("step_kernel"), "k_step1d")
                 if len(w["n"]) == 1 else "k_march2dm" if persistent else
                 {"direct": "k_step2d", "window": "k_step2dw",
                  "masked": "k_step2dm" if w["precision"] == "fp32" else "k_step2dm64"}[
                     info.get("step_kernel", "direct")])
        roofline = {"kernel": kname, "bound": "alu", "achieved": achieved / 1e12,
                    "peak": peak_flops / 1e12, "peak_source": "measured", "unit": "TFLOP/s",
                    "frac": achieved / peak_flops,
                    "traffic": profile_traffic(kname, args.workload),
                    "flop_per_launch": flops_launch, "launch_ms": launch_ms,
                    "window_rows": info.get("window_rows", 0),
                    "step_kernel": info.get("step_kernel"),
                    "march_mode": info.get("march_mode"),
                    "nodes_per_thread": info.get("nodes_per_thread", 1)}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step_max, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if w["precision"] == "fp32" else "f64", "data": "synthetic",
        "config": {"workload": args.workload, "grid": list(w["n"]), "q_per_dim": w["q"],
                   "time_steps": w["n_steps"], "dt": w["dt"], "path": w["path"],
                   "tile": info["tile"][:2], "halo": info["halo"][:2],
                   "march": info.get("march_mode"), "l2": l2_note(w),
                   "parallelism": f"{world} independent instances (one per GPU)"},
        "hbm_gbs_algorithmic": hbm_bytes_per_solve(w) * world / (ms_step_max * 1e-3) / 1e9,
        "roofline": roofline,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": field_bytes,
                "d2h_bytes_per_step": field_bytes},
        "gpu_launches": args.steps * (1 if info.get("step_kernel") in ("resident", "cluster") else
                                      2 if persistent else
                                      # 3D: records (with the quench's coefficients) + window
                                      (2 if w["path"] == "csr" or len(w["n"]) == 3 else 1)
                                      * w["n_steps"] + 1),
        "clocks": clocks,
        "wall_s_timed_region": wall,
        "alu_peaks": peaks,
        **extras,
    }
    if not args.no_cpu_baseline:
        try:
            line["cpu_baseline"] = oracle_rate(w)
        except Exception as exc:  # the oracle is optional for the GPU number
            line["cpu_baseline"] = {"value": None, "error": repr(exc)}
    print(json.dumps(line), flush=True)
    plan.close()


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    try:
        if args.workload in fk_inputs.BATCHES:
            run_batched(args, rank, world, local_rank)
        elif args.workload == "adjoint_1025x513":
            run_adjoint(args, rank, world, local_rank)
        elif args.workload == "horizons_1025x513":
            run_horizons(args, rank, world, local_rank)
        else:
            run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
