"""Benchmark of the RKL2 conduction super-step on GB300.

One step = one RKL2 super-step of the 3D tangled-field workload (256^3
periodic cells, FP32 state, Spitzer kappa_par = 0.01 T^(5/2), kappa_perp =
1e-4 kappa_par, super-step dt = 100 dt_expl(T at t = 0), so s = 20 stages):
the FP64 statistics pass that gives dt_expl, the host choice of s and the
FP64 coefficients, and the graph of s stage kernels.  The metric is
Gcell-stage/s = cells * stages / time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  ``--impl reference`` times the FP64 CPU oracle on a
bounded periodic window of the same workload on the host cores.  With N > 1
(torchrun) every rank advances its own independent problem (replicas; the
method needs no exchange between problems), and rank 0 reports the
aggregate over the slowest rank's time.
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
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_GRID = 256
RATIO = 100.0
SEED = 2
BYTES_PER_CELL_STAGE = 32          # Y_{j-1}, Y_{j-2}, Y_0, M(Y_0), bx, by, bz read; Y_j written (FP32)
WORKLOAD = "tangled256_spitzer_rkl2"

# DRAM traffic of one stage launch (j >= 2) of the 256^3 workload from one
# ncu capture (dram__bytes_read.sum + dram__bytes_write.sum of the stage
# kernel), valid only while the stage kernel's sources hash to source_hash
# (sha256 of STAGE_KERNEL_SOURCES, 16 hex).
MEASURED_TRAFFIC = {"source_hash": "f470e08b66f9d7b3", "bytes_per_launch": 546675968}


# the sources of the default stage kernel (stage_q_kernel, the row-pair
# kernel, built on the paired-cell kernel's face and copy helpers)
STAGE_KERNEL_SOURCES = ("rkl_xq.cuh", "rkl_xq.cu", "rkl_x2_tile.cuh", "rkl_x2.cuh", "rkl_pair.cuh", "rkl_device.cuh")


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1702_05487_gb300", "csrc")
    for fn in STAGE_KERNEL_SOURCES:
        h.update(open(os.path.join(csrc, fn), "rb").read())
    return h.hexdigest()[:16]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region.

    nvidia-smi writes to a pseudo-terminal, so that its C library flushes
    every row as it is printed (a pipe may hold them until exit), and
    every row carries nvidia-smi's own timestamp: the rows kept are those
    stamped between the end of __enter__ and the start of __exit__.
    Entering waits briefly for the first row so that sampling is under way
    when the timed region starts.  If no row falls in the window (a region
    shorter than the sampling period) the row closest to its end is kept and
    the summary says so."""
    QUERY = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    PERIOD_MS = 10
    REASONS = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.rows = []
        self.nearest = False
        self.window_ms = 0.0

    def _read(self):
        buf = b""
        while True:
            try:
                chunk = os.read(self.master, 4096)
            except OSError:          # EIO once the child has closed its side
                break
            if not chunk:
                break
            buf += chunk
            *done, buf = buf.split(b"\n")
            self.lines.extend(x.decode(errors="replace") for x in done)

    @staticmethod
    def _stamp(text):
        import datetime
        try:
            return datetime.datetime.strptime(text.strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            return None

    def __enter__(self):
        import threading
        import pty
        try:
            self.master, slave = pty.openpty()
        except OSError:              # no pseudo-terminals here: a pipe, rows may arrive late
            self.master, slave = os.pipe()
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", str(self.PERIOD_MS)], stdin=subprocess.DEVNULL, stdout=slave, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            os.close(self.master)
            return self
        finally:
            os.close(slave)
        self.reader = threading.Thread(target=self._read, daemon=True)
        self.reader.start()
        t_end = time.monotonic() + 2.0
        while not self.lines and time.monotonic() < t_end and self.proc.poll() is None:
            time.sleep(0.005)
        self.t0 = time.time()
        return self

    def __exit__(self, *a):
        if self.proc is None:
            return
        t1 = time.time()
        self.window_ms = 1e3 * (t1 - self.t0)
        time.sleep(2e-3 * self.PERIOD_MS)          # the row that closes the window
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
            self.proc.wait(timeout=5)
        self.reader.join(timeout=5)
        os.close(self.master)
        parsed = []
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            t = self._stamp(parts[0]) if len(parts) >= 10 else None
            if t is not None:
                parsed.append((t, parts[1:]))
        self.rows = [r for t, r in parsed if self.t0 <= t <= t1]
        if not self.rows and parsed:
            self.rows = [min(parsed, key=lambda tr: abs(tr[0] - t1))[1]]
            self.nearest = True

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        # row: index, clocks.sm, clocks.max.sm, power.draw, active mask, then the four reasons
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "", 1).isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "", 1).isdigit()]
        reasons = sorted({n for r in self.rows for n, v in zip(self.REASONS, r[5:9]) if v.lower() == "active"})
        out = {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
               "reasons": reasons, "samples": len(self.rows), "period_ms": self.PERIOD_MS,
               "window_ms": round(self.window_ms, 1)}
        if self.nearest:
            out["note"] = "region shorter than the sampling period: the nearest sample"
        return out


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


WORKLOADS = {
    # name: (generator, dtype, algorithmic bytes per cell-stage of the stage kernel)
    "tangled256": ("tangled", "f32", 32),
    "blob512": ("blob", "f32", 32),
    # the blob recipe at 256^3: the saturated stage kernel on a grid small
    # enough for a multi-pass ncu capture
    "blob256": ("blob", "f32", 32),
    "ring100": ("ring", "f64", 56),
}


def workload_config(W, world: int, name: str = "tangled256") -> dict:
    """The workload as both arms report it (no kernel or sample details)."""
    ncell = int(W.T.size)
    return {"workload": WORKLOAD if name == "tangled256" else W.name, "shape": list(W.T.shape),
            "cells": ncell, "dt_over_dtexpl": W.ratio,
            "step": "one RKL2 super-step (dt_expl pass + s stages)",
            "l2": ("inputs larger than L2: 8 grid arrays per stage" if ncell * 32 > 129e6
                   else "working set fits in L2"),
            "parallelism": f"replicas{world}" if world > 1 else "single"}


def make_inputs(name="tangled256"):
    import workloads
    gen = WORKLOADS[name][0]
    if gen == "tangled":
        return workloads.tangled(N_GRID, seed=SEED)
    if gen == "blob":
        return workloads.blob(256 if name == "blob256" else 512, seed=SEED)
    return workloads.ring(100)


def cpu_oracle_sample(W, target_seconds: float = 12.0, size: int | None = None):
    """Time the FP64 oracle on a bounded sample of the workload: for a 3D
    grid one super-step of s stages on a (nz_w, ny, nx) window of it
    (periodic in z), nz_w doubled until the run takes about a quarter of
    target_seconds; for a 2D grid whole super-steps of the full grid,
    repeated likewise.  A given size (nz_w, or the repeat count) skips the
    search.  Returns (dict, seconds of the last timed run, size)."""
    import oracle
    from oracle import Problem
    P = Problem(W.T.shape, **W.params)
    dt = W.ratio * oracle.dt_expl(P, W.T)
    s = oracle.num_stages(W.ratio)
    threads = oracle.set_threads(0)
    if W.T.ndim == 3:
        nz_full, ny, nx = W.T.shape
        nz = min(nz_full, size) if size else 4
        while True:
            Tw = np.ascontiguousarray(W.T[:nz])
            bw = np.ascontiguousarray(W.b[:, :nz])
            Pw = Problem(Tw.shape, **W.params)
            t0 = time.perf_counter()
            oracle.super_step(Pw, Tw, bw, dt, s)
            el = time.perf_counter() - t0
            if size or el >= target_seconds / 4 or nz >= nz_full:
                break
            nz = min(nz_full, nz * 2)
        cells = Tw.size * s
        sample = (f"one {s}-stage super-step of a {nz}x{ny}x{nx} window of the {W.name} workload "
                  f"(periodic in z), FP64, {el:.1f} s wall")
    else:
        reps = size or 1
        while True:
            T = W.T.copy()
            t0 = time.perf_counter()
            for _ in range(reps):
                T, _ = oracle.super_step(P, T, W.b, dt, s)
            el = time.perf_counter() - t0
            if size or el >= target_seconds / 4:
                break
            reps *= 2
        cells = W.T.size * s * reps
        sample = (f"{reps} {s}-stage super-steps of the whole {'x'.join(map(str, W.T.shape))} {W.name} grid, "
                  f"FP64, {el:.1f} s wall")
    return {"value": cells / el / 1e9, "unit": "Gcell-stage/s", "cores": threads, "kind": "oracle",
            "sample": sample}, el, (nz if W.T.ndim == 3 else reps)


def cpu_baseline_all_and_one(W):
    """The oracle on all host cores (the cpu_baseline value) and, on a
    smaller window, on one thread; with the host's architecture and CPU
    count."""
    import platform
    import oracle
    cpu, _, _ = cpu_oracle_sample(W)
    n_all = cpu["cores"]
    oracle.set_threads(1)
    try:
        one, _, _ = cpu_oracle_sample(W, target_seconds=8.0)
    finally:
        oracle.set_threads(n_all)
    cpu["single_thread"] = {"value": one["value"], "sample": one["sample"]}
    cpu["host"] = f"{platform.machine()}, {os.cpu_count()} logical CPUs"
    return cpu


def run_reference(args):
    world, rank, local = dist_env()
    if rank != 0:
        return
    W = make_inputs()
    res = None
    times = []
    # the sample size is chosen in the first warm-up step (about a minute in
    # all), then every step runs that same sample
    size = None
    for k in range(args.warmup + args.steps):
        r, el, size = cpu_oracle_sample(W, target_seconds=max(0.5, 60.0 / max(1, args.steps + args.warmup)),
                                        size=size)
        if k >= args.warmup:
            times.append(el)
            res = r
    line = {"impl": "reference", "metric": "Gcell-stage/s per RKL2 stage", "value": res["value"],
            "unit": "Gcell-stage/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.mean(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(W, world),
            "cpu_baseline": res,
            "e2e": {"value": res["value"], "unit": "Gcell-stage/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def aggregate_over_ranks(dist, elapsed: float, units: float, device="cpu"):
    """Replicas: the slowest rank's elapsed time and the units all ranks
    processed (value = units / elapsed).  dist=None on one process."""
    if dist is None:
        return elapsed, units
    import torch
    t = torch.tensor([elapsed, units], device=device, dtype=torch.float64)
    mx = t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    sm = t.clone()
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(sm[1])


def stage_launches_per_step(variant: int, s: int) -> int:
    """Stage-kernel launches of one super-step: s, or with the two-stage
    kernel stage 1, the pairs (j, j+1) for j + 1 < s, then the rest singly."""
    if variant != 5:
        return s
    pairs = max(0, (s - 2) // 2)
    return 1 + pairs + (s - 1 - 2 * pairs)


def run_ours(args):
    import torch
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        dist = None
        torch.cuda.set_device(0)
    import paper_1702_05487_gb300 as rk

    W = make_inputs(args.workload)
    _, dtype, bytes_per_cs = WORKLOADS[args.workload]
    npdt = np.float32 if dtype == "f32" else np.float64
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    T0 = torch.from_numpy(W.T.astype(npdt))
    b0 = torch.from_numpy(W.b.astype(npdt))
    T = T0.to(dev)
    b = b0.to(dev).contiguous()
    params = dict(W.params)
    if args.limiter != "none":
        # Appendix C: MC-limited transverse gradients (generic kernel)
        params.update(limiter=args.limiter, limiter_floor=float("inf"))
    plan = rk.Plan(W.T.shape, dtype, stream=stream, params=params)
    if args.variant or args.nzchunk:
        plan.set_variant(args.variant, args.nzchunk)
    dt = W.ratio * plan.dt_expl(T)
    ncell = T.numel()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # warm-up (also builds the cached graph)
    s_used = []
    for _ in range(args.warmup):
        s_used.append(plan.super_step(dt, T, b))
    barrier()
    plan.set_timing(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clocks:
        barrier()
        ev0.record(stream)
        stages = 0
        launches = 0
        s_timed = []
        for _ in range(args.steps):
            s = plan.super_step(dt, T, b)
            stages += s
            s_timed.append(s)
            launches += stage_launches_per_step(args.variant, s)
        ev1.record(stream)
        barrier()
    ms = ev0.elapsed_time(ev1)
    stage_ms, stage_launches = plan.timing()
    plan.set_timing(False)
    status = plan.check()
    if status != 0:
        raise RuntimeError(f"device status {status} after the timed region")

    # slowest rank's time, all ranks' cell-stages
    ms_max, total_cell_stages = aggregate_over_ranks(dist, ms, float(ncell) * stages, dev)
    value = total_cell_stages / (ms_max * 1e-3) / 1e9

    # end to end through the public host-buffer API: every step copies T and
    # b from pinned host memory, runs one super-step and copies T back.
    # rkl_run_host_batch streams the steps as jobs whose copies overlap the
    # previous and next job's super-step (three host buffer pairs rotate:
    # job i + 3 starts from job i's result); rkl_run_host does one job per
    # call with its copies in series.
    Th = [T0.clone().pin_memory() for _ in range(3)]
    bh = [b0.clone().pin_memory() for _ in range(3)]
    plan.run_host_batch(dt, 1, Th, bh)        # warm the staging buffers and graphs
    barrier()
    t0 = time.perf_counter()
    e_stages = sum(plan.run_host_batch(dt, 1, [Th[i % 3] for i in range(args.steps)],
                                       [bh[i % 3] for i in range(args.steps)]))
    barrier()
    e_s = time.perf_counter() - t0
    e_s, e_cell_stages = aggregate_over_ranks(dist, e_s, float(ncell) * e_stages, dev)
    e2e_value = e_cell_stages / e_s / 1e9
    plan.run_host(dt, 1, Th[0], bh[0])
    barrier()
    t0 = time.perf_counter()
    e_stages = 0
    for _ in range(args.steps):
        e_stages += plan.run_host(dt, 1, Th[0], bh[0])
    barrier()
    e_s = time.perf_counter() - t0
    e_s, e_cell_stages = aggregate_over_ranks(dist, e_s, float(ncell) * e_stages, dev)
    e2e_serial = e_cell_stages / e_s / 1e9

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    peak, peak_kind = measured_peaks()
    avg_launch_ms = stage_ms / max(1, stage_launches)
    achieved = bytes_per_cs * ncell / (avg_launch_ms * 1e-3) / 1e9
    traffic = None
    default_kernel = args.variant in (0, 10) and args.nzchunk == 0 and args.limiter == "none"
    if args.workload == "tangled256" and default_kernel and MEASURED_TRAFFIC["source_hash"] == kernel_source_hash():
        traffic = MEASURED_TRAFFIC["bytes_per_launch"]
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_all_and_one(W)
    line = {
        "metric": "Gcell-stage/s per RKL2 stage", "value": value, "unit": "Gcell-stage/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": dtype, "data": "synthetic",
        "config": workload_config(W, world, args.workload),
        "run": {"s": stages / max(1, args.steps), "s_range": [min(s_timed), max(s_timed)],
                "s_note": "mean stage count of the timed super-steps (T cools at fixed dt, so s may drop)",
                "kernel_variant": args.variant, "nzchunk": args.nzchunk, "limiter": args.limiter},
        "roofline": {"bound": "hbm", "kernel": "rkl2 stage", "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "algorithmic_bytes_per_launch": bytes_per_cs * ncell,
                     "avg_launch_ms": avg_launch_ms, "launches_timed": stage_launches},
        "e2e": {"value": e2e_value, "unit": "Gcell-stage/s",
                "h2d_bytes_per_step": int(T0.numel() * T0.element_size() + b0.numel() * b0.element_size()),
                "d2h_bytes_per_step": int(T0.numel() * T0.element_size()),
                "api": "rkl_run_host_batch (copies overlap compute)", "serial_run_host": e2e_serial},
        "gpu_launches": int(launches + args.steps),     # stage launches + one statistics pass per step
        "clocks": clocks.summary(),
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_ensemble(args):
    """The batched workload: 64 uneven periodic problems, one step = one
    super-step of every problem (autotuned schedule)."""
    import torch
    import paper_1702_05487_gb300 as rk
    import workloads
    torch.cuda.set_device(0)
    specs = workloads.ensemble_specs(64, seed=4)
    probs = []
    for sp in specs:
        shape = (sp["nz"], sp["ny"], sp["nx"])
        probs.append((shape, dict(dx=(sp["h"],) * 3, kappa_model="spitzer",
                                  kappa_par0=sp["kappa_par0"], kappa_perp_ratio=1e-4)))
    ens = rk.Ensemble(probs)
    T_all = torch.empty(ens.offsets[-1], device="cuda")
    b_all = torch.empty(3 * ens.offsets[-1], device="cuda")
    dts = []
    for sp, (Tv, bv), (shape, prm) in zip(specs, ens.views(T_all, b_all), probs):
        T, b = workloads.tangled_box(sp["nx"], sp["ny"], sp["nz"], sp["seed"])
        Tv.copy_(torch.from_numpy(T.astype(np.float32)))
        bv.copy_(torch.from_numpy(b.astype(np.float32)))
        kmax = prm["kappa_par0"] * float(T.max()) ** 2.5 * (1 + 1e-4)
        dts.append(sp["ratio"] * 0.5 / (kmax * 3.0 / sp["h"] ** 2))
    pers, nz, _ = ens.autotune(dts, T_all, b_all)
    for _ in range(args.warmup):
        ens.super_step(dts, T_all, b_all)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    cs = 0.0
    with ClockSampler(0) as clocks:
        ev0.record()
        for _ in range(args.steps):
            s = ens.super_step(dts, T_all, b_all)
            cs += sum(float(np.prod(sh)) * sp for (sh, _), sp in zip(probs, s))
        ev1.record()
        torch.cuda.synchronize()
    assert ens.check() == 0
    ms = ev0.elapsed_time(ev1)
    value = cs / (ms * 1e-3) / 1e9
    peak, peak_kind = measured_peaks()
    line = {"metric": "Gcell-stage/s per RKL2 stage", "value": value, "unit": "Gcell-stage/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "ensemble64", "problems": 64, "cells": int(ens.offsets[-1]),
                       "schedule": ("persistent" if pers & 1 else "per-launch")
                       + (", row-pair tiles" if pers & 2 else ", paired-cell tiles"), "nzchunk": nz,
                       "step": "one super-step of every problem (statistics pass + stages)"},
            "roofline": {"bound": "hbm", "kernel": "whole ensemble step", "achieved": 32 * value,
                         "peak": peak, "peak_kind": peak_kind, "unit": "GB/s", "frac": 32 * value / peak,
                         "traffic": None},
            "clocks": clocks.summary()}
    print(json.dumps(line), flush=True)


def run_split(args):
    """Operator splitting on the 256^3 tangled-field problem: one step =
    donor-cell advection by an ABC flow over dt_h (Eq. dt_h, C_h = 0.8,
    flow scaled so that dt_h = 100 dt_expl at t = 0) followed by the
    conduction over dt_h.  Times the three strategies of Table 1 (RKL2
    super-step, sub-cycled explicit conduction, fully explicit) and reports
    the RKL2 one; the others and the Table 1 run-time model (from the
    measured hyperbolic step and conduction stage) ride along."""
    import torch
    import paper_1702_05487_gb300 as rk
    from paper_1702_05487_gb300.split import SplitDriver, table1_costs
    W = make_inputs("tangled256")
    n = N_GRID
    c = 2 * math.pi * (np.arange(n) + 0.5) / n
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    u0 = np.stack([np.sin(z) + np.cos(y), np.sin(x) + np.cos(z), np.sin(y) + np.cos(x)])
    stream = torch.cuda.current_stream()
    T0 = torch.from_numpy(W.T.astype(np.float32)).cuda()
    b = torch.from_numpy(W.b.astype(np.float32)).cuda().contiguous()
    probe = rk.Plan(W.T.shape, "f32", stream=stream, params=W.params)
    dte = probe.dt_expl(T0)
    u_unit = torch.from_numpy(u0.astype(np.float32)).cuda().contiguous()
    scale = probe.dt_hyperbolic(u_unit, 0.8) / (100.0 * dte)
    u = (u_unit * scale).contiguous()
    probe.close()
    out = {}
    for strategy in ("rkl2", "subcycle", "explicit"):
        drv = SplitDriver(W.T.shape, "f32", params=W.params, stream=stream, ch=0.8, strategy=strategy)
        Ta, Tb = T0.clone(), torch.empty_like(T0)
        dth = drv.dt_h(u)
        nsub = drv.substeps(dth, Ta)
        steps = args.steps if strategy == "rkl2" else max(1, args.steps // 5)
        cur, oth = Ta, Tb
        for k in range(args.warmup + steps):
            if k == args.warmup:
                torch.cuda.synchronize()
                ev0 = torch.cuda.Event(enable_timing=True)
                ev1 = torch.cuda.Event(enable_timing=True)
                ev0.record(stream)
            new, _, stages = drv.step(cur, oth, b, u, dth, None if strategy == "rkl2" else nsub)
            oth = cur if new is not cur else oth
            cur = new
        ev1.record(stream)
        torch.cuda.synchronize()
        out[strategy] = {"ms_per_step": ev0.elapsed_time(ev1) / steps, "conduction_stages": int(stages)}
        drv.close()
    # Table 1 inputs: one advection step and one conduction stage
    plan = rk.Plan(W.T.shape, "f32", stream=stream, params=W.params)
    Tb = torch.empty_like(T0)
    for _ in range(3):
        plan.advect(dth, u, T0, Tb)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(20):
        plan.advect(dth, u, T0, Tb)
    e1.record(stream)
    torch.cuda.synchronize()
    t_hyp = e0.elapsed_time(e1) / 20
    s = out["rkl2"]["conduction_stages"]
    t_stage = (out["rkl2"]["ms_per_step"] - t_hyp) / s
    model = table1_costs(t_hyp, t_stage, nsub, s)
    value = 1e3 / out["rkl2"]["ms_per_step"]
    line = {"metric": "operator-split steps/s (advection + RKL2 conduction over dt_h)", "value": value,
            "unit": "step/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": out["rkl2"]["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "split256", "shape": list(W.T.shape), "dt_h_over_dtexpl": nsub,
                       "flow": "ABC, C_h = 0.8", "conduction": "Spitzer, tangled b"},
            "strategies": out,
            "table1": {"t_hyp_ms": t_hyp, "t_stage_ms": t_stage, "r": t_hyp / t_stage,
                       "model_ms_per_step": model,
                       "speedup_vs_explicit": out["explicit"]["ms_per_step"] / out["rkl2"]["ms_per_step"],
                       "speedup_vs_subcycle": out["subcycle"]["ms_per_step"] / out["rkl2"]["ms_per_step"]}}
    print(json.dumps(line), flush=True)


def measured_bf16_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured (cuBLAS bf16 burst)"
    except Exception:
        return 1900.0, "fallback"


# channels (cin, cout) of the six surrogate convolutions as the network uses
# them, and as the kernels compute them (layer 0 input and layer 5 output
# padded to 16 channels)
SUR_CH_USED = [(6, 32), (32, 32), (32, 32), (32, 32), (32, 32), (32, 3)]
SUR_CH_RUN = [(16, 32), (32, 32), (32, 32), (32, 32), (32, 32), (32, 16)]


def surrogate_forward_timing(n=128, reps=10):
    """Device time of one surrogate forward pass (six 3x3x3 convolutions,
    features already in place) on an n^3 patch with each convolution
    backend, CUDA events on the surrogate's stream after three warm-up
    passes.  Returns {backend: ms} and the FLOPs per pass (used, run)."""
    import torch
    import paper_1702_05487_gb300 as rk
    L = rk._lib
    stream = torch.cuda.current_stream()
    sur = L.rkl_sur_create(n, n, n, (1.0 / n,) * 3, stream.cuda_stream)
    g = torch.Generator(device="cuda").manual_seed(7)
    T = 1.0 + 0.2 * torch.rand(n, n, n, device="cuda", generator=g)
    b = torch.randn(3, n, n, n, device="cuda", generator=g)
    b = (b / b.norm(dim=0, keepdim=True)).contiguous()
    L.rkl_sur_features(sur, T, b, 0.01, True, 100.0)
    out = {}
    for backend in (0, 1):
        L.rkl_sur_set_backend(sur, backend)
        for _ in range(3):
            L.rkl_sur_forward(sur, 2e-3)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            L.rkl_sur_forward(sur, 2e-3)
        e1.record(stream)
        torch.cuda.synchronize()
        L.rkl_sur_check(sur)
        out[backend] = e0.elapsed_time(e1) / reps
    L.rkl_sur_destroy(sur)
    cells = n ** 3
    flops = tuple(2.0 * 27 * cells * sum(ci * co for ci, co in ch) for ch in (SUR_CH_USED, SUR_CH_RUN))
    return out, flops


def surrogate_roofline(fwd_ms, flops):
    peak, kind = measured_bf16_peak()
    achieved = flops[0] / (fwd_ms[1] * 1e-3) / 1e12
    return {"bound": "tensor", "kernel": "surrogate forward (tcgen05 convolutions)", "achieved": achieved,
            "peak": peak, "peak_kind": kind, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
            "algorithmic_flops_per_pass": flops[0], "executed_flops_per_pass": flops[1],
            "executed_tflops": flops[1] / (fwd_ms[1] * 1e-3) / 1e12, "forward_ms": fwd_ms[1],
            "forward_ms_mma_sync": fwd_ms[0]}


def run_surrogate_forward(args):
    """Surrogate inference kernels alone: one forward pass on a 128^3 patch
    with the tcgen05 convolutions and with the warp-level mma.sync ones."""
    import torch
    torch.cuda.set_device(0)
    with ClockSampler(0) as clocks:
        fwd, flops = surrogate_forward_timing(128, max(args.steps, 10))
    line = {"metric": "surrogate forward passes/s (128^3 patch)", "value": 1e3 / fwd[1], "unit": "pass/s",
            "n_gpus": 1, "steps": max(args.steps, 10), "warmup": 3, "ms_per_step": fwd[1],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16/f32",
            "data": "synthetic", "config": {"workload": "surrogate128-forward", "shape": [128, 128, 128],
                                            "l2": "activations 128 MB per layer in BF16 (L2-sized)"},
            "roofline": surrogate_roofline(fwd, flops), "clocks": clocks.summary(),
            "gpu_launches": int(max(args.steps, 10) * 7)}
    print(json.dumps(line), flush=True)


def run_surrogate(args):
    """The learned surrogate on 128^3 patches: training on RKL2-generated
    pairs, threshold calibration at 1e-3 relative L2 on held-out pairs, then
    time-to-solution of surrogate + fallback against plain RKL2."""
    import torch
    from paper_1702_05487_gb300.surrogate import Surrogate, SurrogateConfig
    torch.cuda.set_device(0)
    sur = Surrogate(SurrogateConfig(n=128, pool=16))
    t0 = time.perf_counter()
    losses = sur.train(args.pairs)
    train_s = time.perf_counter() - t0
    thr, rows = sur.calibrate(64, accuracy=1e-3)
    errs = [e for _, e in rows]
    # the configured super-step (dt = 100 dt_expl) and the short end of the
    # training range, where more predictions pass the residual check
    tts = sur.time_to_solution(10, ratio=100.0, accuracy=1e-3)
    tts50 = sur.time_to_solution(10, ratio=50.0, accuracy=1e-3)
    fwd, flops = surrogate_forward_timing(128)
    line = {"metric": "surrogate vs RKL2 time-to-solution @1e-3 L2", "value": tts["speedup"],
            "unit": "x (RKL2 time / surrogate+fallback time)", "n_gpus": 1, "higher_is_better": True,
            "dtype": "bf16/f32", "data": "synthetic",
            "config": {"workload": "surrogate128", "pairs": args.pairs, "train_s": train_s,
                       "final_loss": float(np.mean(losses[-50:])), "threshold": thr,
                       "heldout_rel_l2_median": float(np.median(errs)), "heldout_rel_l2_min": float(min(errs)),
                       "heldout_within_1e-3": int(sum(e <= 1e-3 for e in errs)), "heldout": len(errs)},
            "time_to_solution": tts, "time_to_solution_dt50": tts50, "roofline": surrogate_roofline(fwd, flops)}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--variant", type=int, default=0,
                    help="stage kernel: 0 auto, 1 generic, 2 tiled, 3/4 paired-cell at 5/6 CTAs per SM, 5 two-stage, "
                         "6 bulk copies, 7 tensor-map Y copies, 8 every bundle from tensor maps, "
                         "9 32-column tiles, 10 row-pair (two cell pairs per thread), 11 row-pair with 32-column tiles")
    ap.add_argument("--nzchunk", type=int, default=0, help="planes per CTA (0 automatic, < 0 balanced runs)")
    ap.add_argument("--limiter", default="none", choices=["none", "mc"],
                    help="transverse gradients: plain averages, or MC-limited at every face (Appendix C; "
                         "the paired-cell kernel's limited build, --variant 2 the tiled kernel)")
    ap.add_argument("--workload", default="tangled256",
                    choices=list(WORKLOADS) + ["ensemble64", "surrogate128", "split256"])
    ap.add_argument("--pairs", type=int, default=20000, help="training pairs of the surrogate workload")
    ap.add_argument("--forward-only", action="store_true",
                    help="surrogate128: time the inference convolutions only (no training)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "ensemble64":
        run_ensemble(args)
    elif args.workload == "surrogate128":
        run_surrogate_forward(args) if args.forward_only else run_surrogate(args)
    elif args.workload == "split256":
        run_split(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
