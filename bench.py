"""Benchmark: KMC events/s of the fractional-step sweep on one GB300.

Workload (default): the 2D Ising spin-flip Arrhenius benchmark of Section 7
on a 1024x1024 periodic lattice at betaJ = 0.4407, 16x16 cells, Lie
splitting with dt = 1, binary64 window clocks. One step = 10 units of
physical time (20 fractional windows) plus the observables (coverage,
energy, pair correlations up to r = 32): every stage of the hot path.

Prints one JSON line (rank 0). ``--impl reference`` times the CPU oracle on
a bounded sample of the same workload instead. Under torchrun each rank runs
its own independent lattice (replicas only: the path needs no collective);
the barrier and the max-over-ranks timing use torch.distributed.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from workloads import WORKLOADS, sample_shape  # noqa: E402

METRIC = "KMC events/sec on 1 GB300 (batched FP32-clock vs plain FP64) at stated Δt-error"
STEP_WINDOWS_DT = 10  # one bench step advances the lattice by 10 dt of physical time
RMAX = 32
L2_FLUSH_BYTES = 256 << 20


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="ising1024")
    p.add_argument("--cpu-seconds", type=float, default=10.0)
    p.add_argument("--no-variants", action="store_true")
    p.add_argument("--engine", default="plain", choices=["plain", "persistent"])
    p.add_argument("--clock", default="fp64", choices=["fp64", "fp32"])
    p.add_argument("--wpb", type=int, default=0, help="warps per CTA (0: the library default)")
    p.add_argument("--order", default="auto", choices=["auto", "natural", "workload"],
                   help="issue order of a window's active cells")
    p.add_argument("--cell", type=int, default=0,
                   help="ensemble512: square cell side (0: the library's autotuner picks cells and warps per CTA)")
    p.add_argument("--grouping", default="auto", choices=["auto", "on", "off"],
                   help="several small spin-flip cells per warp (on), one cell per warp (off), "
                        "or the library's choice (auto)")
    return p.parse_args()


def dist_setup(n):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[3 + i] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


# Roofline of the window kernels. The per-event arithmetic of the clock
# contract is K + 4 operations: the ordered fused multiply-add chain over
# the model's K classes (binary64) or the exact fixed-point class sums
# (binary32 clock), the threshold multiply, the clock add, the divide and
# the logarithm. They are uniform within a cell, so one warp instruction
# serves every cell that shares the warp: 1 in the one-cell kernels, 32 / W
# in the grouped kernels (W lanes per cell). Algorithmic warp operations per
# event = (K + 4) / cells per warp.
NCLASSES = {"ADSDES": 10, "ISING": 10, "DIFFUSION": 15, "ZGB": 4, "ISING1D": 6}
# Peak (binary64): the nominal GB300 FP64 rate (1.25 TFLOP/s) as warp
# instructions, 1.25e12 / (2 flops per FMA x 32 lanes) = 19.5 G warp-ops/s.
FP64_WARP_OPS_PEAK_G = 1.25e12 / 64 / 1e9
# Peak (binary32 clock): the warp-instruction issue rate, 152 SMs x 4
# schedulers x 2.07 GHz.
ISSUE_PEAK_G = 152 * 4 * 2.07
# Measured dependent latency of one binary64 fused multiply-add on GB300
# (cycles): the binary64 chain of K + 2 dependent operations per event is
# the latency floor of the binary64 kernels.
FP64_DEP_LATENCY_CYCLES = 64

# DRAM traffic per launch of the bench's kernel on the 1024^2 Ising workload
# (bit-packed lattice) from one ncu capture (profiles/), valid only for the
# kernel source it was taken on.
PROFILED_TRAFFIC = {
    "fs_group_kernel<ISING,double,packed,W=8>": {
        "src": ["fskmc_group.cuh", "fskmc_device.cuh"], "bytes_per_launch": 186880,
        "src_sha256": "196fdfa90747162fac54f84b80f0c113dcf7fbf75a77738ef23ecd32cccc9b96"},
}


def init_state(ctx, w, seed):
    """The workload's initial state: the seeded Gaussian bump of species A on
    an empty lattice where the workload names one, else Bernoulli coverage."""
    if "bump" in w:
        ctx.init_bump(seed, w["bump"]["amp"], w["bump"]["width"], 1)
    else:
        ctx.init_random(seed, w.get("coverage", 0.5))


def stage_bytes_per_site(w):
    """Algorithmic bytes one window moves per active site: the cell and its
    one-site halo read, the cell written, (1 + 2/q)^2 + 1 sites, at one byte
    per site or one bit per site when bit-packed."""
    q = w["q"][0]
    return ((1.0 + 2.0 / q) ** 2 + 1.0) / (8.0 if w.get("bitpacked") else 1.0)


def src_sha(names):
    """SHA-256 over the kernel's source files, in order."""
    import hashlib
    h = hashlib.sha256()
    for name in names:
        h.update(open(os.path.join(ROOT, "paper_1105_4673_gb300", "csrc", name), "rb").read())
    return h.hexdigest()


def kernel_name(engine, model, fp64, packed, lanes):
    """The window kernel the bench's configuration launches."""
    grouped = lanes < 32
    base = {("plain", False): "fs_window_kernel", ("persistent", False): "fs_persistent_kernel",
            ("plain", True): "fs_group_kernel", ("persistent", True): "fs_group_persistent_kernel"}
    args = [model, "double" if fp64 else "float"] + (["packed"] if packed else [])
    if grouped:
        args.append(f"W={lanes}")
    return f"{base[(engine, grouped)]}<{','.join(args)}>"


def cpu_baseline(w, seconds):
    """The oracle as it stands on a bounded sample of the workload: a 256x256
    lattice (a ring of 8192 sites for the 1D model) of the same model, rates,
    cell shape and schedule, advanced step by step until `seconds` of CPU
    time. Events/s do not depend on the lattice size for the cell-by-cell
    oracle (cost per event ~ cell size)."""
    import oracle
    lx, ly = sample_shape(w)
    run = oracle.FSRun(lx, ly, *w["q"], w["model"], w["rates"],
                       oracle.init_bernoulli(lx, ly, w["seed"], w.get("coverage", 0.5)))
    t0 = time.process_time()
    steps = 0
    while steps == 0 or time.process_time() - t0 < seconds:
        run.run(w["scheme"], w["dt"], w["dt"], w["seed"])
        steps += 1
    dt = max(time.process_time() - t0, 1e-9)
    return {"value": run.events / dt, "unit": "events/s", "cores": 1, "kind": "oracle",
            "sample": f"{lx}x{ly} lattice, same model/rates/cells/schedule, {steps} steps "
                      f"of dt={w['dt']} ({run.events} events, {dt:.1f} s CPU, single thread)"}


def ensemble_sample(w, reps, q):
    """A single-lattice stand-in of the ensemble for the host-CPU oracle:
    replica 0's rates, the ensemble's model, schedule and cells."""
    return dict(model=w["model"], rates=reps[0]["rates"], q=tuple(q), scheme=w["scheme"], dt=w["dt"],
                coverage=w["coverage"], seed=w["seed"])


def run_reference(args, rank, world):
    w = WORKLOADS[args.workload]
    if args.workload == "ensemble512":
        from workloads import ensemble_replicas
        w = ensemble_sample(w, ensemble_replicas(w["n"], w["seed"]), (16, 16))
    if rank != 0:
        return
    cb = None
    vals = []
    import oracle
    lx, ly = sample_shape(w)
    run = oracle.FSRun(lx, ly, *w["q"], w["model"], w["rates"],
                       oracle.init_bernoulli(lx, ly, w["seed"], w.get("coverage", 0.5)))
    for i in range(args.warmup + args.steps):
        e0 = run.events
        t0 = time.perf_counter()
        run.run(w["scheme"], w["dt"], w["dt"], w["seed"])
        t1 = time.perf_counter()
        if i >= args.warmup:
            vals.append(((run.events - e0), t1 - t0))
    ev = sum(v[0] for v in vals)
    tt = sum(v[1] for v in vals)
    value = ev / tt
    cb = {"value": value, "unit": "events/s", "cores": 1, "kind": "oracle",
          "sample": f"{lx}x{ly} lattice of the {args.workload} workload, one step of dt="
                    f"{w['dt']} per bench step, single thread"}
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "events/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * tt / max(len(vals), 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload + f" ({lx}x{ly} sample on the host CPU)"},
        "cpu_baseline": cb,
        "e2e": {"value": value, "unit": "events/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0}}), flush=True)


def run_ensemble(args, rank, world, local):
    """The batched ensemble (512 replicas of uneven size and rates) advanced
    in one persistent, graph-launched kernel per step; one step = 10 dt of
    physical time for every replica. Cell size and warps per block come from
    the library's autotuner."""
    import torch

    import paper_1105_4673_gb300 as F
    from workloads import ensemble_replicas
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    w = WORKLOADS["ensemble512"]
    seed = rank_seed(w["seed"], rank)
    reps = ensemble_replicas(w["n"], w["seed"])
    clock = args.clock.upper()
    if args.cell:
        q, wpb = (args.cell, args.cell), args.wpb or 2
    else:
        q, wpb, _ = F.autotune(reps, w["model"], w["scheme"], w["dt"], clock=clock, engine="PERSISTENT",
                               coverage=w["coverage"], seed=w["seed"], stream=stream)
    b = F.Context(model=w["model"], q=q, batch=reps, stream=stream)
    b.set_engine("PERSISTENT")
    b.set_warps_per_block(wpb)
    b.set_clock(clock)
    b.set_cell_grouping({"auto": "AUTO", "on": True, "off": False}[args.grouping])
    b.init_random(seed, w["coverage"])
    step_t = STEP_WINDOWS_DT * w["dt"]
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        b.run(w["scheme"], w["dt"], step_t, seed)
    torch.cuda.synchronize()
    ev0 = b.stats()["events"]
    barrier(world)
    kev = []
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.zero_()
            a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            b.run(w["scheme"], w["dt"], step_t, seed)
            c.record(stream)
            kev.append((a, c))
        torch.cuda.synchronize()
    barrier(world)
    events = b.stats()["events"] - ev0
    t_ms = max_over_ranks(sum(a.elapsed_time(c) for a, c in kev), world)
    value = sum_over_ranks(events, world) / (t_ms / 1000.0)
    # end to end: every replica's state in from pinned host memory, the step,
    # every state out
    hosts = [torch.empty(r["lx"] * r["ly"], dtype=torch.uint8, pin_memory=True) for r in reps]
    for r, h in enumerate(hosts):
        b.get_state(r, h.numpy())
    torch.cuda.synchronize()
    e_ev0 = b.stats()["events"]
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for r, h in enumerate(hosts):
            b.set_state(h.numpy(), r)
        b.run(w["scheme"], w["dt"], step_t, seed)
        for r, h in enumerate(hosts):
            b.get_state(r, h.numpy())
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world)
    e2e_events = sum_over_ranks(b.stats()["events"] - e_ev0, world)
    if rank != 0:
        b.close()
        return
    fp64 = clock == "FP64"
    lanes = b.info()["lanes_per_cell"]
    cells_per_warp = 32 // lanes if lanes < 32 else 1
    ops = NCLASSES[w["model"]] + 4
    k_avg_s = t_ms / 1000.0 / args.steps
    achieved = events / args.steps * ops / cells_per_warp / k_avg_s / 1e9
    peak = FP64_WARP_OPS_PEAK_G if fp64 else ISSUE_PEAK_G
    nbytes = sum(r["lx"] * r["ly"] for r in reps)
    cb = cpu_baseline(ensemble_sample(w, reps, q), args.cpu_seconds)
    cb["sample"] = "replica 0's rates and the autotuned cells: " + cb["sample"]
    print(json.dumps({
        "metric": METRIC, "value": value, "unit": "events/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if fp64 else "f32+u64", "data": "synthetic",
        "config": {"workload": f"ensemble512: {len(reps)} replicas, sides 64..512, {w['model']}, betaJ "
                               f"U[0.2,0.8], ka/kd logU[0.1,10], {w['scheme']} dt={w['dt']}",
                   "step": f"{step_t:g} time units for every replica, one persistent launch",
                   "clock": args.clock, "engine": "persistent", "cell": f"{q[0]}x{q[1]}" + ("" if args.cell else " (autotuned)"),
                   "warps_per_cta": wpb, "lanes_per_cell": lanes, "sites": nbytes,
                   "cells": b.info()["cells"], "l2": "flushed between timed steps"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak,
                     "unit": "G fp64 warp-ops/s" if fp64 else "G warp-ops/s", "frac": achieved / peak,
                     "traffic": None,
                     "kernel": kernel_name("persistent", w["model"], fp64, False, lanes),
                     "kernel_ms_avg": k_avg_s * 1000, "launches": args.steps,
                     "events_per_launch": events / args.steps, "algorithmic_ops_per_event": ops,
                     "cells_per_warp": cells_per_warp,
                     "algorithmic_warp_ops_per_event": ops / cells_per_warp,
                     "peak_note": ("derived: nominal 1.25 TFLOP/s FP64 / 64 flops per warp FMA"
                                   if fp64 else "derived: 152 SMs x 4 schedulers x 2.07 GHz")},
        "cpu_baseline": cb,
        "e2e": {"value": e2e_events / e2e_s, "unit": "events/s", "h2d_bytes_per_step": nbytes,
                "d2h_bytes_per_step": nbytes},
        "gpu_launches": args.steps,
        "clocks": clk.summary(),
    }), flush=True)
    b.close()


def main():
    args = parse()
    rank, world, local = dist_setup(args.gpus)
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload == "ensemble512":
        from paper_1105_4673_gb300 import build as B
        B.build()
        run_ensemble(args, rank, world, local)
        return
    import torch

    import paper_1105_4673_gb300 as F
    from paper_1105_4673_gb300 import build as B
    B.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    w = WORKLOADS[args.workload]
    lx, ly = w["lx"], w["ly"]
    seed = rank_seed(w["seed"], rank)
    ctx = F.Context(lx, ly, w["model"], w["rates"], w["q"], stream=stream,
                    bitpacked=w.get("bitpacked", False))
    ctx.set_engine(args.engine.upper())
    ctx.set_clock(args.clock.upper())
    if args.wpb:
        ctx.set_warps_per_block(args.wpb)
    ctx.set_task_order(args.order.upper())
    ctx.set_cell_grouping({"auto": "AUTO", "on": True, "off": False}[args.grouping])
    init_state(ctx, w, seed)
    step_t = STEP_WINDOWS_DT * w["dt"]
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def step(kernel_events=None):
        # plain engine: one window-kernel launch per window, each bracketed by
        # events on the context's stream; persistent: one launch per run
        if args.engine == "plain":
            col, hh = F.schedule(w["scheme"], w["dt"], step_t, seed, 0, ctx.window_index)
            for c, h in zip(col, hh):
                if kernel_events is not None:
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    ctx.window(int(c), float(h), seed)
                    b.record(stream)
                    kernel_events.append((a, b))
                else:
                    ctx.window(int(c), float(h), seed)
        else:
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ctx.run(w["scheme"], w["dt"], step_t, seed)
            b.record(stream)
            if kernel_events is not None:
                kernel_events.append((a, b))
        return ctx.observables(0, RMAX)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ev0 = ctx.stats()["events"]
    barrier(world)
    torch.cuda.synchronize()
    kev = []
    step_times = []
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.zero_()  # L2 flush between timed steps (outside the step's events)
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            step(kev)
            s1.record(stream)
            step_times.append((s0, s1))
        torch.cuda.synchronize()
    barrier(world)
    events = ctx.stats()["events"] - ev0
    t_ms = sum(a.elapsed_time(b) for a, b in step_times)
    t_ms = max_over_ranks(t_ms, world)
    events_all = sum_over_ranks(events, world)
    kernel_ms = [a.elapsed_time(b) for a, b in kev]
    value = events_all / (t_ms / 1000.0)

    # end to end through the C ABI with host buffers: H2D of the state from
    # pinned memory, the step, D2H of the state and the observables
    host = torch.empty(lx * ly, dtype=torch.uint8, pin_memory=True)
    hnp = host.numpy()
    ctx.get_state(0, hnp)
    torch.cuda.synchronize()
    e_ev0 = ctx.stats()["events"]
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ctx.set_state(hnp)
        ctx.run(w["scheme"], w["dt"], step_t, seed)
        ctx.observables(0, RMAX)
        ctx.get_state(0, hnp)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world)
    e2e_events = sum_over_ranks(ctx.stats()["events"] - e_ev0, world)

    variants = {}
    if not args.no_variants and rank == 0:
        variants = measure_variants(F, w, stream, seed, steps=max(2, args.steps // 2))

    if rank != 0:
        ctx.close()
        return
    cs = clk.summary()
    k_events_per_launch = events / max(len(kernel_ms), 1)
    k_avg_s = float(np.mean(kernel_ms)) / 1000.0
    lanes = ctx.info()["lanes_per_cell"]
    cells_per_warp = 32 // lanes if lanes < 32 else 1
    ops_per_event = NCLASSES[w["model"]] + 4
    warp_ops_per_event = ops_per_event / cells_per_warp
    achieved = k_events_per_launch * warp_ops_per_event / k_avg_s / 1e9
    fp64 = args.clock == "fp64"
    peak = FP64_WARP_OPS_PEAK_G if fp64 else ISSUE_PEAK_G
    kname = kernel_name(args.engine, w["model"], fp64, bool(w.get("bitpacked")), lanes)
    traffic = None
    prof = PROFILED_TRAFFIC.get(kname)
    if prof and args.workload == "ising1024" and prof["src_sha256"] == src_sha(prof["src"]):
        traffic = prof["bytes_per_launch"]
    # the critical path: the slowest cell's events in the last window set the
    # window's duration; cycles per event of that cell vs the binary64 floor
    wl_max = int(ctx.workload(0).max()) if args.engine == "plain" else 0
    sm_mhz = clk.summary().get("sm_mhz") or 2070.0
    cb = cpu_baseline(w, args.cpu_seconds)
    out = {
        "metric": METRIC, "value": value, "unit": "events/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if fp64 else "f32+u64", "data": "synthetic",
        "config": {"workload": f"{args.workload}: {lx}x{ly} {w['model']} betaJ="
                               f"{w['rates'].get('betaJ')} q={w['q'][0]} {w['scheme']} dt={w['dt']}",
                   "step": f"{step_t:g} time units ({kernel_windows_per_step(F, w, step_t)} windows) "
                           "+ observables",
                   "clock": args.clock, "engine": args.engine,
                   "warps_per_cta": ctx.info()["warps_per_block"],
                   "lanes_per_cell": ctx.info()["lanes_per_cell"], "task_order": args.order,
                   "storage": "1 bit/site" if w.get("bitpacked") else "1 byte/site",
                   "l2": "flushed between timed steps"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak,
                     "unit": "G fp64 warp-ops/s" if fp64 else "G warp-ops/s", "frac": achieved / peak,
                     "traffic": traffic,
                     "kernel": kname,
                     "kernel_ms_avg": k_avg_s * 1000, "launches": len(kernel_ms),
                     "events_per_launch": k_events_per_launch,
                     "algorithmic_ops_per_event": ops_per_event,
                     "cells_per_warp": cells_per_warp,
                     "algorithmic_warp_ops_per_event": warp_ops_per_event,
                     "peak_note": ("derived: nominal 1.25 TFLOP/s FP64 / 64 flops per warp FMA"
                                   if fp64 else "derived: 152 SMs x 4 schedulers x 2.07 GHz") +
                                  f"; HBM is not the bound ({stage_bytes_per_site(w):.2f} B per "
                                  "active site per window)",
                     "critical_path": None if not wl_max else {
                         "slowest_cell_events": wl_max,
                         "cycles_per_event": k_avg_s * sm_mhz * 1e6 / wl_max,
                         "binary64_floor_cycles_per_event":
                             (NCLASSES[w["model"]] + 2) * FP64_DEP_LATENCY_CYCLES if fp64 else None}},
        "cpu_baseline": cb,
        "e2e": {"value": e2e_events / e2e_s, "unit": "events/s",
                "h2d_bytes_per_step": lx * ly, "d2h_bytes_per_step": lx * ly + 8 * (4 + 2 * RMAX)},
        "gpu_launches": len(kernel_ms) + args.steps,
        "clocks": cs,
        "variants": variants,
    }
    print(json.dumps(out), flush=True)
    ctx.close()


def measure_variants(F, w, stream, seed, steps):
    """The same workload through the persistent engine (one graph-launched
    kernel per run) with binary64 and binary32 window clocks; the 512-replica
    ensemble in one persistent launch per run (binary32 clock, the batched
    form); and the binary32-vs-binary64 difference of the observables."""
    import torch
    res = {}
    res["ensemble512_persistent_fp32"] = ensemble_rate(F, stream, "FP32")
    res["ensemble512_persistent_fp64"] = ensemble_rate(F, stream, "FP64")
    res["fp32_vs_fp64"] = clock_error(F, stream, w)
    forms = [("PERSISTENT", "FP64", "AUTO"), ("PERSISTENT", "FP32", "AUTO"), ("PLAIN", "FP32", "AUTO")]
    if _group_width_default(F, w) < 32:  # the same workload with one cell per warp
        forms += [("PLAIN", "FP64", False)]
    for engine, clock, grouped in forms:
        c = F.Context(w["lx"], w["ly"], w["model"], w["rates"], w["q"], stream=stream,
                      bitpacked=w.get("bitpacked", False))
        c.set_engine(engine)
        c.set_clock(clock)
        c.set_cell_grouping(grouped)
        init_state(c, w, seed)
        step_t = STEP_WINDOWS_DT * w["dt"]
        c.run(w["scheme"], w["dt"], step_t, seed)
        torch.cuda.synchronize()
        e0 = c.stats()["events"]
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            c.run(w["scheme"], w["dt"], step_t, seed)
        b.record(stream)
        torch.cuda.synchronize()
        ev = c.stats()["events"] - e0
        key = f"{engine.lower()}_{clock.lower()}" + ("" if grouped else "_one_cell_per_warp")
        res[key] = {"events_per_s": ev / (a.elapsed_time(b) / 1000), "events": ev,
                    "lanes_per_cell": c.info()["lanes_per_cell"]}
        c.close()
    return res


def _group_width_default(F, w):
    """Lanes per cell the library picks for the workload's cells."""
    c = F.Context(w["lx"], w["ly"], w["model"], w["rates"], w["q"],
                  bitpacked=w.get("bitpacked", False))
    n = c.info()["lanes_per_cell"]
    c.close()
    return n


def ensemble_rate(F, stream, clock, T=5.0):
    """Events/s of the 512-replica ensemble (sides 64..512, betaJ in
    [0.2, 0.8], ka/kd log-uniform) advanced by T in one persistent run."""
    import torch
    from workloads import ensemble_replicas
    w = WORKLOADS["ensemble512"]
    reps = ensemble_replicas(w["n"], w["seed"])
    q, wpb, _ = F.autotune(reps, w["model"], w["scheme"], w["dt"], clock=clock,
                           engine="PERSISTENT", coverage=w["coverage"], seed=w["seed"],
                           stream=stream)
    b = F.Context(model=w["model"], q=q, batch=reps, stream=stream)
    b.set_engine("PERSISTENT")
    b.set_warps_per_block(wpb)
    b.set_clock(clock)
    b.init_random(w["seed"], w["coverage"])
    b.run(w["scheme"], w["dt"], 1.0, w["seed"])
    torch.cuda.synchronize()
    e0 = b.stats()["events"]
    a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    b.run(w["scheme"], w["dt"], T, w["seed"])
    c.record(stream)
    torch.cuda.synchronize()
    ev = b.stats()["events"] - e0
    out = {"events_per_s": ev / (a.elapsed_time(c) / 1000), "events": ev, "replicas": len(reps),
           "sites": int(sum(r["lx"] * r["ly"] for r in reps)), "T": T, "cells": b.info()["cells"],
           "autotuned": {"q": q[0], "warps_per_block": wpb}}
    b.close()
    return out


def clock_error(F, stream, w, n=64, L=128, T=10.0):
    """Binary32 minus binary64 clock, per observable, over n independent
    replicas of an L x L lattice of the workload's model (mean difference and
    its standard error), and each form's dt-error estimate against dt/16."""
    import torch
    shape = (L * L, 1) if w["model"] == "ISING1D" else (L, L)
    reps = [dict(lx=shape[0], ly=shape[1], rates=w["rates"]) for _ in range(n)]

    def run(clock, dt, seed):
        b = F.Context(model=w["model"], q=w["q"], batch=reps, stream=stream)
        b.set_engine("PERSISTENT")
        b.set_clock(clock)
        b.init_random(seed, w.get("coverage", 0.5))
        b.run(w["scheme"], dt, T, seed)
        obs = []
        for r in range(n):
            cov, en, _ = b.observables(r, 1)
            obs.append([cov[1], en])
        obs = np.array(obs)
        b.close()
        return obs

    out = {"replicas": n, "lattice": f"{shape[0]}x{shape[1]}", "T": T, "dt": w["dt"]}
    f64 = run("FP64", w["dt"], 101)
    f32 = run("FP32", w["dt"], 202)
    ref = run("FP64", w["dt"] / 16, 303)
    for j, name in enumerate(("coverage", "energy")):
        d = f32[:, j].mean() - f64[:, j].mean()
        se = float(np.sqrt(f32[:, j].var(ddof=1) / n + f64[:, j].var(ddof=1) / n))
        e64 = f64[:, j].mean() - ref[:, j].mean()
        e32 = f32[:, j].mean() - ref[:, j].mean()
        se_r = float(np.sqrt(f64[:, j].var(ddof=1) / n + ref[:, j].var(ddof=1) / n))
        out[name] = {"fp32_minus_fp64": float(d), "se": se, "within_3se": bool(abs(d) < 3 * se),
                     "dt_error_fp64": float(e64), "dt_error_fp32": float(e32), "dt_error_se": se_r}
    torch.cuda.synchronize()
    return out


def kernel_windows_per_step(F, w, step_t):
    return len(F.schedule(w["scheme"], w["dt"], step_t)[0])


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _reduce(x, world, op):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    device = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(x, world):
    """Slowest rank's time (the job's time)."""
    import torch.distributed as dist
    return _reduce(x, world, dist.ReduceOp.MAX) if world > 1 else x


def sum_over_ranks(x, world):
    """Whole-job count (events of all ranks)."""
    import torch.distributed as dist
    return _reduce(x, world, dist.ReduceOp.SUM) if world > 1 else x


def rank_seed(base, rank):
    """Each rank simulates its own independent lattice (weak scaling)."""
    return base + 7919 * rank


if __name__ == "__main__":
    main()
