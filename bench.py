"""Benchmark: KMC events/s of the fractional-step sweep on one GB300.

Workload (default): the ZGB catalytic surface of Section 7.1 on a 16384 x
16384 periodic lattice (three states, one byte per site, 32 x 32 cells),
empty with a seeded Gaussian bump of species A, Strang splitting with
dt = 0.02. One step = 10 dt of physical time (30 fractional windows) through
fskmc_run, plus the observables (coverage per species, energy, pair
correlations up to r = 32): every stage of the hot path.

The line compares, on the same workload in the same run, the batched
binary32-clock form (the persistent, graph-launched engine with per-cell
binary32 clocks over exact integer class sums; `value`) with the plain
binary64 form (one launch per window, the oracle's arithmetic bit for bit),
and states the dt-error of each observable (against the same scheme at
dt/8, the serial-SSA limit up to 1/64 of the error for a second-order
splitting) with its standard error over independent runs.

``--impl reference`` times the CPU oracle on a bounded sample of the same
workload instead. Under torchrun each rank runs its own independent lattice
(replicas only: the path needs no collective); the barrier and the
max-over-ranks timing use torch.distributed.
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

from workloads import WORKLOADS, cpu_sample  # noqa: E402

METRIC = "KMC events/sec on 1 GB300 (batched FP32-clock vs plain FP64) at stated Δt-error"
STEP_WINDOWS_DT = 10  # one bench step advances the lattice by 10 dt of physical time
RMAX = 32
L2_FLUSH_BYTES = 256 << 20
FORMS = {"batched_fp32": ("PERSISTENT", "FP32"), "plain_fp64": ("PLAIN", "FP64"),
         "plain_fp32": ("PLAIN", "FP32"), "persistent_fp64": ("PERSISTENT", "FP64")}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="zgb16384")
    p.add_argument("--form", default="batched_fp32", choices=list(FORMS),
                   help="the form `value` reports (the metric's batched binary32-clock form by default)")
    p.add_argument("--compare", default="plain_fp64", choices=list(FORMS) + ["none"],
                   help="the form timed beside it on the same workload")
    p.add_argument("--cpu-seconds", type=float, default=10.0)
    p.add_argument("--no-variants", action="store_true", help="skip the other two forms")
    p.add_argument("--dt-error-runs", type=int, default=8,
                   help="independent runs per arm of the dt-error estimate (0: skip)")
    p.add_argument("--dt-error-T", type=float, default=2.56, help="physical time of the dt-error runs")
    p.add_argument("--wpb", type=int, default=0, help="warps per CTA (0: the library default)")
    p.add_argument("--order", default="auto", choices=["auto", "natural", "workload"],
                   help="issue order of a window's active cells")
    p.add_argument("--cell", type=int, default=0,
                   help="ensemble512: square cell side (0: the library's autotuner picks cells and warps per CTA)")
    p.add_argument("--grouping", default="auto", choices=["auto", "on", "off"],
                   help="several small spin-flip cells per warp (on), one cell per warp (off), "
                        "or the library's choice (auto)")
    p.add_argument("--clock", default="fp32", choices=["fp64", "fp32"], help="ensemble512 only")
    p.add_argument("--study", default=None,
                   choices=["weak-order", "weak-order-replicas", "clock-error", "nested", "dt-error-scaling",
                            "cpu-ssa"],
                   help="instead of the throughput line: the weak-order study of the 1024^2 Ising "
                        "workload (Lie and Strang, dt in {1, 1/2, 1/4, 1/8} against the dt -> 0 "
                        "limit), or the binary32-vs-binary64 clock error of the workload's observables")
    p.add_argument("--betaJ", type=float, default=None, help="weak-order study: coupling (default: the workload's)")
    p.add_argument("--dts", default="1,0.5,0.25,0.125", help="weak-order studies: the window lengths")
    p.add_argument("--ref-dt", type=float, default=1.0 / 32, help="weak-order studies: the reference window")
    p.add_argument("--study-T", type=float, default=1.0, help="weak-order-replicas: physical time")
    p.add_argument("--replicas", type=int, default=8192, help="weak-order-replicas: replicas per batch")
    p.add_argument("--batches", type=int, default=4, help="weak-order-replicas: batches per point")
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


# ---------------------------------------------------------------------------
# Roofline of the window kernels: plain ALU lanes. The method's own work per
# event (the per-event work list of the hot path), counted once per event in
# 32-bit lane operations, whatever the kernel's layout:
#   draw        one Philox4x32-10 block: 10 rounds x (2 mul.lo + 2 mul.hi +
#               4 xor) + 9 key bumps x 2 = 98, and 6 to form u_t, u_c, j
#   clock       the waiting time and the edge test: binary32 6 (log, divide,
#               add, compare); binary64 18 (the 14-operation logarithm, the
#               divide, the add, the compare)
#   class       the class choice over K classes: binary64 2K (the ordered
#               fused multiply-add chain and its compares), fixed point 3K
#               (64-bit products and compares)
#   member      the rank search in the chosen class's bit set: one popcount
#               per 32-bit word of the set (a site class has ceil(n/32) words
#               of a cell of n sites, a slot class 8 times that), a 5-step
#               scan and a 10-operation select in the owner word; weighted by
#               the fraction of events in slot classes
#   update      4 operations (class, mask bit, two counts) per member whose
#               class the event can change: 5 (spin flip), 3 (ring), 2 sites
#               and 14 slots (ZGB), 25 sites and 40 slots (diffusion)
# Peak: 152 SMs x 128 lanes x 2.07 GHz.
ALU_PEAK_G = 152 * 128 * 2.07
NCLASSES = {"ADSDES": 10, "ISING": 10, "DIFFUSION": 15, "ZGB": 4, "ISING1D": 6}
UPDATE_MEMBERS = {"ADSDES": 5, "ISING": 5, "ISING1D": 3, "ZGB": 16, "DIFFUSION": 65}
SLOT_EVENT_FRACTION = {"ZGB": 0.5, "DIFFUSION": 0.5}


def algo_lane_ops_per_event(model, q, fp64):
    K = NCLASSES[model]
    words = -(-(q[0] * q[1]) // 32)
    f = SLOT_EVENT_FRACTION.get(model, 0.0)
    member = (1 - f) * words + f * 8 * words + 5 + 10
    return 98 + 6 + (18 if fp64 else 6) + (2 * K if fp64 else 3 * K) + member + \
        4 * UPDATE_MEMBERS[model]


# ncu figures of the bench's kernels (profiles/), valid only for the kernel
# source they were taken on: DRAM bytes per fractional window of the
# workload, the issue-slot utilisation and the ALU pipe's utilisation.
PROFILED = {
    ("fs_zgbq_persistent_kernel<8>", "zgb16384"): {
        "src": ["fskmc_zgbquad.cu", "fskmc_zgb32x4.cuh", "fskmc_zgb32x2.cuh", "fskmc_zgb32.cuh", "fskmc_device.cuh",
                "fskmc_internal.h", "fskmc_logtab.h", "philox.cuh"],
        "dram_bytes_per_window": 586420480, "issue_active": 0.685, "alu_pipe": 0.799,
        "src_sha256": "abf4aeed91e150c109bf9e5e2f546c36db65eac90c51d42c7c2adefe06678f28"},
}


def src_sha(names):
    """SHA-256 over the kernel's source files, in order."""
    import hashlib
    h = hashlib.sha256()
    for name in names:
        h.update(open(os.path.join(ROOT, "paper_1105_4673_gb300", "csrc", name), "rb").read())
    return h.hexdigest()


def kernel_name(engine, model, fp64, packed, lanes, q=None):
    """The window kernel the bench's configuration launches."""
    grouped = lanes < 32
    if model == "ZGB" and grouped:  # 32 / lanes 32-wide cells per warp, binary32
        if lanes == 16:
            return {"PLAIN": "fs_zgbp_window_kernel", "PERSISTENT": "fs_zgbp_persistent_kernel"}[engine]
        kind = {"PLAIN": "fs_zgbq_window_kernel", "PERSISTENT": "fs_zgbq_persistent_kernel"}[engine]
        return f"{kind}<{32 // lanes}>"
    base = {("PLAIN", False): "fs_window_kernel", ("PERSISTENT", False): "fs_persistent_kernel",
            ("PLAIN", True): "fs_group_kernel", ("PERSISTENT", True): "fs_group_persistent_kernel"}
    args = [model, "double" if fp64 else "float"] + (["packed"] if packed else [])
    if grouped:
        args.append(f"W={lanes}")
    if model == "ZGB" and not fp64 and q is not None and q[0] == 32 and q[1] >= 2:
        args.append("rows in registers")
    return f"{base[(engine, grouped)]}<{','.join(args)}>"


def stage_bytes_per_site(w):
    """Algorithmic bytes one window moves per active site: the cell and its
    halo read, the cell written, (1 + 2 hw/q)^2 + 1 sites, at one byte per
    site or one bit per site when bit-packed (hw = 2 for diffusion)."""
    q = w["q"][0]
    hw = 2 if w["model"] == "DIFFUSION" else 1
    return ((1.0 + 2.0 * hw / q) ** 2 + 1.0) / (8.0 if w.get("bitpacked") else 1.0)


# ---------------------------------------------------------------------------
# CPU baseline: the oracle on a bounded sample of the workload
# ---------------------------------------------------------------------------
def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_sample(w, threads):
    """The oracle's run object on the workload's CPU sample: the same model,
    rates, cells and schedule on a smaller lattice (the all-core form gets a
    lattice with enough active cells for every thread), the same kind of
    initial state."""
    import oracle
    lx, ly = cpu_sample(w, threads)
    if "bump" in w:
        init = oracle.init_bump(lx, ly, w["seed"], w["bump"]["amp"], lx / 8.0, 1)
    else:
        init = oracle.init_bernoulli(lx, ly, w["seed"], w.get("coverage", 0.5))
    return oracle.FSRun(lx, ly, *w["q"], w["model"], w["rates"], init), (lx, ly)


def oracle_step(run, w, threads):
    if threads > 1:
        run.run_threads(w["scheme"], w["dt"], w["dt"], w["seed"], threads)
    else:
        run.run(w["scheme"], w["dt"], w["dt"], w["seed"])


def cpu_baseline(w, seconds, threads):
    """The oracle as it stands on a bounded sample of the workload, one step
    of dt at a time until `seconds` of wall time; events/s (the oracle's cost
    per event depends on the cell size, not the lattice size)."""
    run, (lx, ly) = oracle_sample(w, threads)
    t0 = time.perf_counter()
    steps = 0
    while steps == 0 or time.perf_counter() - t0 < seconds:
        oracle_step(run, w, threads)
        steps += 1
    dt = max(time.perf_counter() - t0, 1e-9)
    return {"value": run.events / dt, "unit": "events/s", "cores": threads, "kind": "oracle",
            "sample": f"{lx}x{ly} lattice, same model/rates/cells/schedule, {steps} steps of "
                      f"dt={w['dt']} ({run.events} events in {dt:.1f} s wall), "
                      + ("cells of each window over %d threads" % threads if threads > 1
                         else "single thread")}


def run_reference(args, rank, world):
    """The reference arm: the oracle (all host cores, cells of each window
    over threads) on the workload's CPU sample, one step of dt per bench
    step. Rank 0 only."""
    w = WORKLOADS[args.workload]
    if args.workload == "ensemble512":
        from workloads import ensemble_replicas
        w = ensemble_sample(w, ensemble_replicas(w["n"], w["seed"]), (16, 16))
    if rank != 0:
        return
    threads = host_cores()
    run, (lx, ly) = oracle_sample(w, threads)
    vals = []
    for i in range(args.warmup + args.steps):
        e0 = run.events
        t0 = time.perf_counter()
        oracle_step(run, w, threads)
        t1 = time.perf_counter()
        if i >= args.warmup:
            vals.append(((run.events - e0), t1 - t0))
    ev = sum(v[0] for v in vals)
    tt = sum(v[1] for v in vals)
    value = ev / tt
    cb = {"value": value, "unit": "events/s", "cores": threads, "kind": "oracle",
          "sample": f"{lx}x{ly} lattice of the {args.workload} workload, one step of dt="
                    f"{w['dt']} per bench step, cells of each window over {threads} threads"}
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "events/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * tt / max(len(vals), 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload + f" ({lx}x{ly} sample on the host CPU)"},
        "cpu_baseline": cb,
        "e2e": {"value": value, "unit": "events/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0}}), flush=True)


def ensemble_sample(w, reps, q):
    """A single-lattice stand-in of the ensemble for the host-CPU oracle:
    replica 0's rates, the ensemble's model, schedule and cells."""
    return dict(model=w["model"], rates=reps[0]["rates"], q=tuple(q), scheme=w["scheme"], dt=w["dt"],
                coverage=w["coverage"], seed=w["seed"])


# ---------------------------------------------------------------------------
# The GPU forms
# ---------------------------------------------------------------------------
def init_state(ctx, w, seed):
    """The workload's initial state: the seeded Gaussian bump of species A on
    an empty lattice where the workload names one, else Bernoulli coverage."""
    if "bump" in w:
        ctx.init_bump(seed, w["bump"]["amp"], w["bump"]["width"], 1)
    else:
        ctx.init_random(seed, w.get("coverage", 0.5))


def make_ctx(F, w, form, stream, seed, args):
    engine, clock = FORMS[form]
    c = F.Context(w["lx"], w["ly"], w["model"], w["rates"], w["q"], stream=stream,
                  bitpacked=w.get("bitpacked", False))
    c.set_engine(engine)
    c.set_clock(clock)
    if args.wpb:
        c.set_warps_per_block(args.wpb)
    c.set_task_order(args.order.upper())
    c.set_cell_grouping({"auto": "AUTO", "on": True, "off": False}[args.grouping])
    init_state(c, w, seed)
    return c


def time_form(F, w, form, stream, seed, args, flush, world, clk=None, snapshot=None):
    """W untimed steps, then K steps each bracketed by CUDA events on the
    context's stream (L2 flushed between steps, outside the events): one step
    = fskmc_run over 10 dt + the observables. Returns the form's figures;
    `snapshot` (host array), if given, receives the lattice the timed steps
    start from."""
    import torch
    ctx = make_ctx(F, w, form, stream, seed, args)
    step_t = STEP_WINDOWS_DT * w["dt"]
    for _ in range(args.warmup):
        ctx.run(w["scheme"], w["dt"], step_t, seed)
        ctx.observables(0, RMAX)
    torch.cuda.synchronize()
    if snapshot is not None:
        ctx.get_state(0, snapshot)
    st0 = ctx.stats()
    barrier(world)
    marks = []
    for _ in range(args.steps):
        flush.zero_()
        a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        a.record(stream)
        ctx.run(w["scheme"], w["dt"], step_t, seed)
        b.record(stream)
        ctx.observables(0, RMAX)
        c.record(stream)
        marks.append((a, b, c))
    torch.cuda.synchronize()
    barrier(world)
    st1 = ctx.stats()
    step_ms = [a.elapsed_time(c) for a, b, c in marks]
    run_ms = [a.elapsed_time(b) for a, b, c in marks]
    info = ctx.info()
    out = {"ctx": ctx, "events": st1["events"] - st0["events"], "windows": st1["windows"] - st0["windows"],
           "ambiguous": st1["ambiguous"] - st0["ambiguous"], "check_failures": st1["check_failures"],
           "timeouts": st1["timeouts"], "step_ms": step_ms, "run_ms": run_ms, "info": info}
    t_ms = max_over_ranks(sum(step_ms), world)
    out["events_all"] = sum_over_ranks(out["events"], world)
    out["t_ms"] = t_ms
    out["events_per_s"] = out["events_all"] / (t_ms / 1000.0)
    return out


def end_to_end(F, w, ctx, stream, seed, args, world, hnp):
    """The same steps through the C ABI with host buffers, from the lattice
    the timed steps started from (hnp, pinned host memory; a lattice that
    relaxes has fewer events later on): every step copies the lattice in,
    runs, computes the observables and copies the lattice out."""
    import torch
    lx, ly = w["lx"], w["ly"]
    e0 = ctx.stats()["events"]
    step_t = STEP_WINDOWS_DT * w["dt"]
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ctx.set_state(hnp)
        ctx.run(w["scheme"], w["dt"], step_t, seed)
        ctx.observables(0, RMAX)
        ctx.get_state(0, hnp)
    torch.cuda.synchronize()
    s = max_over_ranks(time.perf_counter() - t0, world)
    ev = sum_over_ranks(ctx.stats()["events"] - e0, world)
    return {"value": ev / s, "unit": "events/s", "h2d_bytes_per_step": lx * ly,
            "d2h_bytes_per_step": lx * ly + 8 * (4 + 2 * RMAX)}


def observable_vector(ctx, model):
    """Coverage of every state, energy (not for ZGB), G_x(1..4), G_y(1..4)."""
    cov, en, pc = ctx.observables(0, 4)
    names = [f"coverage[{s}]" for s in range(3 if model == "ZGB" else 2)]
    vals = list(cov[:len(names)])
    if model != "ZGB":
        names.append("energy")
        vals.append(en)
    names += [f"Gx({r})" for r in range(1, 5)] + [f"Gy({r})" for r in range(1, 5)]
    vals += list(pc[:4]) + list(pc[4:8])
    return names, np.array(vals, np.float64)


def dt_error(F, w, stream, runs, T, args):
    """Per-observable dt-error at time T from the workload's initial state:
    the plain binary64 form and the batched binary32 form at the workload's
    dt against the binary64 form at dt/8 (the serial-SSA limit of the
    splitting up to 1/64 of the error at dt for a second-order scheme, 1/8
    for a first-order one), each over `runs` independent seeds; and the
    binary32-minus-binary64 difference. Means and standard errors."""
    res = {}
    arms = {"fp64": ("plain_fp64", w["dt"]), "fp32": ("batched_fp32", w["dt"]),
            "ref": ("plain_fp64", w["dt"] / 8)}
    names = None
    ambiguous = cellwin = 0
    for arm, (form, dt) in arms.items():
        vals = []
        for s in range(runs):
            c = make_ctx(F, w, form, stream, w["seed"] + 1000 + s, args)
            c.run(w["scheme"], dt, T, w["seed"] + 1000 + s)
            names, v = observable_vector(c, w["model"])
            st = c.stats()
            if arm != "fp32":
                ambiguous += st["ambiguous"]
                cellwin += st["windows"] * c.info()["cells"] // 2
            vals.append(v)
            c.close()
        res[arm] = np.array(vals)
    out = {"T": T, "runs_per_arm": runs, "reference": f"binary64 form at dt/8 = {w['dt'] / 8:g}",
           "observables": {}}

    def mse(a):
        return a.mean(axis=0), a.std(axis=0, ddof=1) / np.sqrt(len(a))

    # the two forms agree if their difference lies within the two-sided
    # 99.7% interval of Student's t with 2 (runs - 1) degrees of freedom (3 SE
    # for many runs; the standard errors of a few runs are themselves uncertain)
    from scipy.stats import t as student_t
    crit = float(student_t.ppf(0.9985, 2 * (runs - 1)))
    m64, s64 = mse(res["fp64"])
    m32, s32 = mse(res["fp32"])
    mr, sr = mse(res["ref"])
    for i, n in enumerate(names):
        e64, se64 = m64[i] - mr[i], float(np.hypot(s64[i], sr[i]))
        e32, se32 = m32[i] - mr[i], float(np.hypot(s32[i], sr[i]))
        d, sd = m32[i] - m64[i], float(np.hypot(s32[i], s64[i]))
        out["observables"][n] = {"value": float(mr[i]), "dt_error_fp64": float(e64), "se_fp64": se64,
                                 "dt_error_fp32": float(e32), "se_fp32": se32,
                                 "fp32_minus_fp64": float(d), "se_diff": sd,
                                 "same_dt_error": bool(abs(d) <= crit * sd)}
    out["t_crit"] = crit
    out["all_same"] = all(o["same_dt_error"] for o in out["observables"].values())
    out["ambiguous_cell_windows"] = int(ambiguous)
    out["cell_windows"] = int(cellwin)
    return out


def run_workload(args, rank, world, local):
    import torch

    import paper_1105_4673_gb300 as F
    from paper_1105_4673_gb300 import build as B
    B.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    w = WORKLOADS[args.workload]
    seed = rank_seed(w["seed"], rank)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    forms = [args.form] + ([args.compare] if args.compare not in ("none", args.form) else [])
    if not args.no_variants:
        forms += [f for f in FORMS if f not in forms]
    res = {}
    snap = torch.empty(w["lx"] * w["ly"], dtype=torch.uint8, pin_memory=True).numpy()
    with ClockSampler(local) as clk:
        for f in forms:
            res[f] = time_form(F, w, f, stream, seed, args, flush, world, snapshot=snap if f == args.form else None)
            if f != args.form:
                res[f]["ctx"].close()
    head = res[args.form]
    e2e = end_to_end(F, w, head["ctx"], stream, seed, args, world, snap)
    info = head["info"]
    head["ctx"].close()
    if rank != 0:
        return
    dterr = dt_error(F, w, stream, args.dt_error_runs, args.dt_error_T, args) if args.dt_error_runs > 0 else None
    engine, clock = FORMS[args.form]
    fp64 = clock == "FP64"
    lanes = info["lanes_per_cell"]
    kname = kernel_name(engine, w["model"], fp64, bool(w.get("bitpacked")), lanes, tuple(w["q"]))
    nwin_step = kernel_windows_per_step(F, w, STEP_WINDOWS_DT * w["dt"])
    launches_per_step = 1 if engine == "PERSISTENT" else nwin_step
    launch_s = float(np.mean(head["run_ms"])) / 1000.0 / launches_per_step
    ev_launch = head["events"] / args.steps / launches_per_step
    ops = algo_lane_ops_per_event(w["model"], w["q"], fp64)
    achieved = ev_launch * ops / launch_s / 1e9
    prof = PROFILED.get((kname, args.workload))
    traffic = issue = alu = None
    if prof and prof["src_sha256"] and prof["src_sha256"] == src_sha(prof["src"]):
        if prof["dram_bytes_per_window"]:
            traffic = prof["dram_bytes_per_window"] * nwin_step / launches_per_step
        issue = prof["issue_active"]
        alu = prof.get("alu_pipe")
    active_cells = info["cells"] // 2
    comparisons = {}
    for f, r in res.items():
        comparisons[f] = {"events_per_s": r["events_per_s"], "ms_per_step": r["t_ms"] / args.steps,
                          "engine": FORMS[f][0], "clock": FORMS[f][1],
                          "lanes_per_cell": r["info"]["lanes_per_cell"],
                          "warps_per_cta": r["info"]["warps_per_block"],
                          "ambiguous_fraction": r["ambiguous"] / max(1, r["windows"] * active_cells),
                          "check_failures": r["check_failures"], "timeouts": r["timeouts"]}
    base = res.get(args.compare)
    statement = None
    if base is not None:
        ratio = head["events_per_s"] / base["events_per_s"]
        statement = (f"{args.form} {head['events_per_s']:.3e} events/s vs {args.compare} "
                     f"{base['events_per_s']:.3e} events/s ({ratio:.2f}x) on {args.workload}, "
                     f"{w['scheme']} dt={w['dt']}")
        if dterr:
            same = "within" if dterr["all_same"] else "NOT within"
            statement += (f"; the two forms' observables differ by {same} {dterr['t_crit']:.2f} SE "
                          f"(99.7% t-interval) at T={dterr['T']} ({dterr['runs_per_arm']} runs each)")
    sb = stage_bytes_per_site(w)
    out = {
        "metric": METRIC, "value": head["events_per_s"], "unit": "events/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["t_ms"] / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if fp64 else "f32+u64", "data": "synthetic",
        "config": {"workload": f"{args.workload}: {w['lx']}x{w['ly']} {w['model']} {w['rates']} "
                               f"q={w['q'][0]}x{w['q'][1]} {w['scheme']} dt={w['dt']}"
                               + (" from a Gaussian bump of A" if "bump" in w else ""),
                   "form": args.form, "engine": engine, "clock": clock,
                   "step": f"{STEP_WINDOWS_DT * w['dt']:g} time units ({nwin_step} windows) through "
                           "fskmc_run + observables (r <= 32)",
                   "warps_per_cta": info["warps_per_block"], "lanes_per_cell": lanes,
                   "storage": "1 bit/site" if w.get("bitpacked") else "1 byte/site",
                   "l2": "flushed between timed steps (256 MiB buffer)"},
        "comparison": comparisons,
        "statement": statement,
        "dt_error": dterr,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": ALU_PEAK_G,
                     "unit": "G lane-ops/s", "frac": achieved / ALU_PEAK_G, "traffic": traffic,
                     "kernel": kname, "kernel_ms_avg": launch_s * 1000,
                     "launches_per_step": launches_per_step, "events_per_launch": ev_launch,
                     "algorithmic_lane_ops_per_event": ops,
                     "issue_active_ncu": issue, "alu_pipe_ncu": alu,
                     "peak_note": "derived: 152 SMs x 128 lanes x 2.07 GHz (plain ALU lanes; the "
                                  "path has no dense contraction)",
                     "hbm_note": f"{sb:.2f} algorithmic bytes per active site per window; "
                                 f"{sb * active_cells * w['q'][0] * w['q'][1] * nwin_step / launches_per_step / launch_s / 1e9:.1f}"
                                 " GB/s of algorithmic traffic: HBM is not the bound"},
        "cpu_baseline": cpu_baseline(w, args.cpu_seconds, host_cores()),
        "cpu_baseline_1core": cpu_baseline(w, args.cpu_seconds, 1),
        "e2e": e2e,
        "gpu_launches": args.steps * (launches_per_step + 1),
        "clocks": clk.summary(),
    }
    print(json.dumps(out), flush=True)


def run_ensemble(args, rank, world, local):
    """The batched ensemble (512 replicas of uneven size and rates) advanced
    in one persistent, graph-launched kernel per step; one step = 10 dt of
    physical time for every replica. Cell size and warps per block come from
    the library's autotuner. Beside it: the same replicas one at a time
    through the plain binary64 form."""
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
    b.set_task_order(args.order.upper())
    b.init_random(seed, w["coverage"])
    step_t = STEP_WINDOWS_DT * w["dt"]
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        b.run(w["scheme"], w["dt"], step_t, seed)
    torch.cuda.synchronize()
    # the lattices the timed steps start from, for the end-to-end leg
    host = torch.empty(int(b.state_layout()[-1]), dtype=torch.uint8, pin_memory=True).numpy()
    b.get_state_all(host)
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
    # end to end, from the timed steps' starting lattices: every replica's
    # state in from pinned host memory (one copy for the batch, in the layout
    # of fskmc_state_layout), the step, every state out
    torch.cuda.synchronize()
    e_ev0 = b.stats()["events"]
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        b.set_state_all(host)
        b.run(w["scheme"], w["dt"], step_t, seed)
        b.get_state_all(host)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world)
    e2e_events = sum_over_ranks(b.stats()["events"] - e_ev0, world)
    lanes = b.info()["lanes_per_cell"]
    cells = b.info()["cells"]
    b.close()
    if rank != 0:
        return
    one_at_a_time = ensemble_one_at_a_time(F, reps, w, stream, seed, q)
    fp64 = clock == "FP64"
    k_avg_s = t_ms / 1000.0 / args.steps
    ops = algo_lane_ops_per_event(w["model"], q, fp64)
    achieved = events / args.steps * ops / k_avg_s / 1e9
    nbytes = sum(r["lx"] * r["ly"] for r in reps)
    cb = cpu_baseline(ensemble_sample(w, reps, q), args.cpu_seconds, host_cores())
    cb["sample"] = "replica 0's rates and the autotuned cells: " + cb["sample"]
    print(json.dumps({
        "metric": METRIC, "value": value, "unit": "events/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if fp64 else "f32+u64", "data": "synthetic",
        "config": {"workload": f"ensemble512: {len(reps)} replicas, sides 64..512, {w['model']}, betaJ "
                               f"U[0.2,0.8], ka/kd logU[0.1,10], {w['scheme']} dt={w['dt']}",
                   "step": f"{step_t:g} time units for every replica, one persistent launch",
                   "clock": args.clock, "engine": "persistent", "cell": f"{q[0]}x{q[1]}" + ("" if args.cell else " (autotuned)"),
                   "warps_per_cta": wpb, "lanes_per_cell": lanes, "sites": nbytes, "task_order": args.order,
                   "cells": cells, "l2": "flushed between timed steps"},
        "comparison": {"one_replica_at_a_time_plain_fp64": one_at_a_time},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": ALU_PEAK_G,
                     "unit": "G lane-ops/s", "frac": achieved / ALU_PEAK_G, "traffic": None,
                     "kernel": kernel_name("PERSISTENT", w["model"], fp64, False, lanes),
                     "kernel_ms_avg": k_avg_s * 1000, "launches": args.steps,
                     "events_per_launch": events / args.steps, "algorithmic_lane_ops_per_event": ops,
                     "peak_note": "derived: 152 SMs x 128 lanes x 2.07 GHz"},
        "cpu_baseline": cb,
        "e2e": {"value": e2e_events / e2e_s, "unit": "events/s", "h2d_bytes_per_step": host.size,
                "d2h_bytes_per_step": host.size},
        "gpu_launches": args.steps,
        "clocks": clk.summary(),
    }), flush=True)


def ensemble_one_at_a_time(F, reps, w, stream, seed, q, T=1.0):
    """The ensemble's baseline: the same replicas advanced one at a time,
    each through its own plain binary64 context (one launch per window per
    replica), for T time units after 1 time unit of warm-up."""
    import torch
    ev = 0
    ms = 0.0
    for r, rp in enumerate(reps):
        c = F.Context(rp["lx"], rp["ly"], w["model"], rp["rates"], q, stream=stream)
        c.set_replica_id(r)
        c.init_random(seed, w["coverage"])
        c.run(w["scheme"], w["dt"], 1.0, seed)
        torch.cuda.synchronize()
        e0 = c.stats()["events"]
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        c.run(w["scheme"], w["dt"], T, seed)
        b.record(stream)
        torch.cuda.synchronize()
        ev += c.stats()["events"] - e0
        ms += a.elapsed_time(b)
        c.close()
    return {"events_per_s": ev / (ms / 1000.0), "events": ev, "T": T, "replicas": len(reps)}


def time_average(F, w, form, stream, seed, dt, scheme, burn, T, args, every=1.0):
    """Observables averaged over samples every `every` time units in
    [burn, T] of one run from the workload's initial state."""
    c = make_ctx(F, w, form, stream, seed, args)
    c.run(scheme, dt, burn, seed)
    acc = []
    t = burn
    names = None
    while t < T - 1e-9:
        c.run(scheme, dt, every, seed)
        t += every
        names, v = observable_vector(c, w["model"])
        acc.append(v)
    c.close()
    return names, np.mean(np.array(acc), axis=0)


def fit_order(dts, errs, ses):
    """Weighted least-squares fit of log|e| = log C + p log dt (weights from
    the standard errors); returns p and its standard error."""
    x = np.log(np.asarray(dts))
    y = np.log(np.abs(np.asarray(errs)))
    sy = np.asarray(ses) / np.maximum(np.abs(np.asarray(errs)), 1e-300)
    wgt = 1.0 / np.maximum(sy, 1e-12) ** 2
    A = np.stack([np.ones_like(x), x], axis=1)
    cov = np.linalg.inv(A.T @ (A * wgt[:, None]))
    beta = cov @ (A.T @ (wgt * y))
    return float(beta[1]), float(np.sqrt(cov[1, 1]))


def study_weak_order(args):
    """Weak-error order of Lie and Strang splitting (Eqs. error, error2) on
    the 1024^2 Ising workload: time-averaged observables (samples every time
    unit over [T/2, T]) at dt in {1, 1/2, 1/4, 1/8} against the same
    average at dt = 1/32 (the serial-SSA limit of the splitting, up to 1/32
    of the Lie error at dt = 1 and 1/1024 of the Strang error), several
    independent runs per point; the error's order by a weighted log-log fit
    over the points resolved beyond 3 standard errors."""
    import torch

    import paper_1105_4673_gb300 as F
    stream = torch.cuda.current_stream()
    w = dict(WORKLOADS["ising1024"])
    if args.betaJ is not None:
        w["rates"] = dict(w["rates"], betaJ=args.betaJ)
    runs, T = max(2, args.dt_error_runs), 200.0
    burn = T / 2
    dts = [1.0, 0.5, 0.25, 0.125]

    def arm(scheme, dt):
        vals = [time_average(F, w, "plain_fp64", stream, w["seed"] + 100 + s, dt, scheme, burn, T, args)
                for s in range(runs)]
        names = vals[0][0]
        a = np.array([v[1] for v in vals])
        return names, a.mean(axis=0), a.std(axis=0, ddof=1) / np.sqrt(runs)

    t0 = time.time()
    names, ref_m, ref_s = arm("STRANG", 1.0 / 32)
    out = {"workload": f"ising1024 betaJ={w['rates']['betaJ']}", "T": T, "average_over": [burn, T],
           "runs_per_point": runs, "reference": "Strang at dt = 1/32", "schemes": {}}
    for scheme in ("LIE", "STRANG"):
        rows = {}
        for dt in dts:
            _, m, s = arm(scheme, dt)
            rows[dt] = (m - ref_m, np.hypot(s, ref_s))
        per_obs = {}
        for i, n in enumerate(names):
            e = [float(rows[d][0][i]) for d in dts]
            se = [float(rows[d][1][i]) for d in dts]
            ok = [j for j in range(len(dts)) if abs(e[j]) > 3 * se[j]]
            fit = fit_order([dts[j] for j in ok], [e[j] for j in ok], [se[j] for j in ok]) if len(ok) >= 2 else None
            per_obs[n] = {"reference_value": float(ref_m[i]), "error": e, "se": se,
                          "resolved_points": [dts[j] for j in ok],
                          "order": None if fit is None else fit[0], "order_se": None if fit is None else fit[1]}
        out["schemes"][scheme] = {"dt": dts, "observables": per_obs}
    out["seconds"] = time.time() - t0
    print(json.dumps(out), flush=True)


def study_weak_order_replicas(args, L=32, q=2):
    """Weak-error order resolved on many small replicas (cells of 2 x 2 sites
    put every site on a cell edge, where the splitting error lives): batches
    of M replicas of an L x L Ising lattice, each batch advanced to time T
    in one persistent binary64 launch, every replica from its own
    Bernoulli(1/2) draw (the same draws in every arm); the replica mean of
    the energy, coverage and G(1) at T for Lie and Strang at the given
    window lengths against Strang at a much shorter one, and the order
    fitted over the points resolved beyond 3 standard errors."""
    import torch

    import paper_1105_4673_gb300 as F
    stream = torch.cuda.current_stream()
    betaJ = 0.6 if args.betaJ is None else args.betaJ
    rates = dict(ka=1.0, kd=1.0, betaJ=betaJ)
    dts = [float(x) for x in args.dts.split(",")]
    M, batches, T = args.replicas, args.batches, args.study_T

    def arm(scheme, dt):
        vals = []
        for b in range(batches):
            reps = [dict(lx=L, ly=L, rates=rates) for _ in range(M)]
            c = F.Context(model="ISING", q=(q, q), batch=reps, stream=stream)
            c.set_engine("PERSISTENT")
            c.init_random(4242 + b, 0.5)
            c.run(scheme, dt, T, 777 + 1000 * b)
            for r in range(M):
                cov, en, pc = c.observables(r, 1)
                vals.append([en, cov[1], pc[0]])
            c.close()
        a = np.array(vals)
        return a.mean(axis=0), a.std(axis=0, ddof=1) / np.sqrt(len(a))

    t0 = time.time()
    ref_m, ref_s = arm("STRANG", args.ref_dt)
    names = ["energy", "coverage", "Gx(1)"]
    out = {"workload": f"{M * batches} replicas of {L}x{L} ISING betaJ={betaJ}, {q}x{q} cells, T={T}, "
                       "from Bernoulli(1/2) states", "reference": f"Strang at dt = {args.ref_dt:g}",
           "schemes": {}}
    for scheme in ("LIE", "STRANG"):
        rows = [arm(scheme, dt) for dt in dts]
        per = {}
        for i, n in enumerate(names):
            e = [float(m[i] - ref_m[i]) for m, _ in rows]
            se = [float(np.hypot(s[i], ref_s[i])) for _, s in rows]
            ok = [j for j in range(len(dts)) if abs(e[j]) > 3 * se[j]]
            fit = fit_order([dts[j] for j in ok], [e[j] for j in ok], [se[j] for j in ok]) if len(ok) >= 2 else None
            per[n] = {"reference_value": float(ref_m[i]), "error": e, "se": se,
                      "resolved_points": [dts[j] for j in ok],
                      "order": None if fit is None else fit[0], "order_se": None if fit is None else fit[1]}
        out["schemes"][scheme] = {"dt": dts, "observables": per}
    out["seconds"] = time.time() - t0
    print(json.dumps(out), flush=True)


def study_nested(args, L=4096, steps=4):
    """The nested two-level scheme (Section 5) beside the one-level scheme on
    the same lattice: a 4096^2 Ising lattice (betaJ = 0.4407, Lie dt = 1),
    one-level with 16x16 cells (the grouped kernels) and nested with 64x64
    super-cells of 16x16 sub-cells (n_in inner Lie steps per outer window),
    both clocks; events/s over `steps` runs of 10 dt after 3 warm-up runs."""
    import torch

    import paper_1105_4673_gb300 as F
    stream = torch.cuda.current_stream()
    rates = dict(ka=1.0, kd=1.0, betaJ=0.4407)
    out = {"lattice": f"{L}x{L} ISING betaJ=0.4407, Lie dt=1", "forms": {}}
    forms = [("one-level 16x16 cells", None, 1)] + [(f"nested 64x64 / 16x16, n_in={n}", (64, 64), n)
                                                    for n in (1, 2, 4)]
    for name, sup, n_in in forms:
        for clock in ("FP64", "FP32"):
            c = F.Context(L, L, "ISING", rates, (16, 16), stream=stream)
            c.set_clock(clock)
            if sup:
                c.set_nesting(sup, "LIE", n_in)
            c.init_random(99, 0.5)
            for _ in range(3):
                c.run("LIE", 1.0, 10.0, 99)
            torch.cuda.synchronize()
            e0 = c.stats()["events"]
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(steps):
                c.run("LIE", 1.0, 10.0, 99)
            b.record(stream)
            torch.cuda.synchronize()
            ev = c.stats()["events"] - e0
            out["forms"][f"{name} {clock}"] = {"events_per_s": ev / (a.elapsed_time(b) / 1000.0),
                                              "events": ev, "ms": a.elapsed_time(b)}
            c.close()
    print(json.dumps(out), flush=True)


def study_dt_error_scaling(args):
    """The workload's dt-error at larger windows, where it is resolved, and
    its order: the binary64 form at dt in {16, 8, 4, 2, 1} x the workload's
    dt against dt/4 of the workload, each over independent runs to time
    --dt-error-T from the initial state; the weighted fit e = C dt^p over the
    resolved points gives the error expected at the workload's own dt (with
    its standard error from the fit)."""
    import torch

    import paper_1105_4673_gb300 as F
    stream = torch.cuda.current_stream()
    w = WORKLOADS[args.workload]
    runs, T = max(2, args.dt_error_runs), args.dt_error_T
    mults = [16, 8, 4, 2, 1]

    def arm(dt):
        vals = []
        for s in range(runs):
            c = make_ctx(F, w, "plain_fp64", stream, w["seed"] + 1000 + s, args)
            c.run(w["scheme"], dt, T, w["seed"] + 1000 + s)
            names, v = observable_vector(c, w["model"])
            vals.append(v)
            c.close()
        a = np.array(vals)
        return names, a.mean(axis=0), a.std(axis=0, ddof=1) / np.sqrt(runs)

    t0 = time.time()
    names, ref_m, ref_s = arm(w["dt"] / 4)
    rows = {m: arm(w["dt"] * m)[1:] for m in mults}
    out = {"workload": args.workload, "T": T, "runs_per_point": runs,
           "reference": f"binary64 form at dt/4 = {w['dt'] / 4:g}", "dts": [w["dt"] * m for m in mults],
           "observables": {}}
    for i, n in enumerate(names):
        e = [float(rows[m][0][i] - ref_m[i]) for m in mults]
        se = [float(np.hypot(rows[m][1][i], ref_s[i])) for m in mults]
        ok = [j for j in range(len(mults)) if abs(e[j]) > 3 * se[j]]
        entry = {"error": e, "se": se, "resolved_dts": [w["dt"] * mults[j] for j in ok]}
        if len(ok) >= 2 and len({np.sign(e[j]) for j in ok}) == 1:
            p_, sp = fit_order([w["dt"] * mults[j] for j in ok], [e[j] for j in ok], [se[j] for j in ok])
            # C from the largest resolved point, the error at the workload's dt
            j0 = ok[0]
            C = e[j0] / (w["dt"] * mults[j0]) ** p_
            pred = C * w["dt"] ** p_
            entry.update(order=p_, order_se=sp, predicted_error_at_dt=float(pred),
                         predicted_rel_se=float(np.hypot(se[j0] / abs(e[j0]), sp * np.log(mults[j0]))))
        out["observables"][n] = entry
    out["seconds"] = time.time() - t0
    print(json.dumps(out), flush=True)


def study_cpu_ssa(args):
    """The serial SSA (the process the splitting approximates) timed on one
    host core for every workload's model and rates: the class-list form on a
    256 x 256 lattice (a 65,536-site ring) in slices of one time unit, and
    the direct-recount form on 32 x 32 (its cost per event grows with the
    lattice) in slices of dt, until `--cpu-seconds` of wall time; events/s."""
    import oracle
    out = {"cores": 1, "workloads": {}}
    for name, w in WORKLOADS.items():
        if "lx" not in w:
            w = ensemble_sample(w, __import__("workloads").ensemble_replicas(w["n"], w["seed"]), (16, 16))
        row = {}
        for form, side in (("class_lists", 256), ("direct", 32)):
            lx, ly = (side * side, 1) if w["model"] == "ISING1D" else (side, side)
            if "bump" in w:
                lat = oracle.init_bump(lx, ly, w["seed"], w["bump"]["amp"], lx / 8.0, 1)
            else:
                lat = oracle.init_bernoulli(lx, ly, w["seed"], w.get("coverage", 0.5))
            run = oracle.ssa_bkl_run if form == "class_lists" else oracle.ssa_run
            slice_t = 1.0 if form == "class_lists" else w["dt"]  # the class lists are rebuilt per call
            t0 = time.perf_counter()
            ev = 0
            k = 0
            while k == 0 or time.perf_counter() - t0 < args.cpu_seconds:
                lat, n = run(lx, ly, w["model"], w["rates"], lat, slice_t, w["seed"], replica=k)
                ev += n
                k += 1
            dt = time.perf_counter() - t0
            row[form] = {"events_per_s": ev / dt, "lattice": f"{lx}x{ly}", "events": ev, "seconds": dt}
        out["workloads"][name] = row
    print(json.dumps(out), flush=True)


def study_clock_error(args):
    """Binary32 minus binary64 window clock, per observable, on the
    workload's own lattice and schedule: several independent runs of each
    form to time 10 dt * 10 from the initial state, and each form's dt-error
    against the binary64 form at dt/8."""
    import torch

    import paper_1105_4673_gb300 as F
    stream = torch.cuda.current_stream()
    w = WORKLOADS[args.workload]
    T = STEP_WINDOWS_DT * w["dt"] * 10
    t0 = time.time()
    out = dt_error(F, w, stream, max(2, args.dt_error_runs), T, args)
    out["workload"] = args.workload
    out["seconds"] = time.time() - t0
    print(json.dumps(out), flush=True)


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


def main():
    args = parse()
    rank, world, local = dist_setup(args.gpus)
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.study == "cpu-ssa":
        study_cpu_ssa(args)
        return
    from paper_1105_4673_gb300 import build as B
    B.build()
    if args.study == "weak-order":
        study_weak_order(args)
        return
    if args.study == "weak-order-replicas":
        study_weak_order_replicas(args)
        return
    if args.study == "dt-error-scaling":
        study_dt_error_scaling(args)
        return
    if args.study == "nested":
        study_nested(args)
        return
    if args.study == "clock-error":
        study_clock_error(args)
        return
    if args.workload == "ensemble512":
        run_ensemble(args, rank, world, local)
        return
    run_workload(args, rank, world, local)


if __name__ == "__main__":
    main()
