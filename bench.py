"""Benchmark: trajectories/s of the batched Picard-Chebyshev propagator on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload precision|flyby|uneven|adjoint]

Default workload (the headline pairing): 65,536 trajectories of the Sun +
Venus + Earth system (a = 0.75 AU, e = 0.3, i = 2 deg, seeded jitter), 2-year
arcs in 25 segments at Chebyshev degree 128, tol 1e-13.  One step = one
pc_propagate call over all of them.  The mixed-precision batched path (FP32
sweeps until the change is below 1e-6, then FP64 sweeps with FP32 correction
solves, to 1e-13) is the line's value; the plain FP64 GPU sweep runs on the
same inputs, timed the same way (same steps, graph replay, no per-kernel
instrumentation), in stats.plain_fp64.  Both arms use the second-order form
of the sweep (--order 1: the paper's first-order sweep) and the FP64
contraction by exact digit products on the bf16 tensor cores (--contraction
dmma: on the FP64 tensor cores).  Every step runs the whole hot path on
the GPU: per-trajectory segment schedule, ephemeris at the nodes, Keplerian
warm start, force, operator contraction, convergence tests, stitching.

value: trajectories/s with inputs resident in HBM (CUDA events on the launch
stream, L2 flushed between steps).  e2e: the same through the C ABI with the
initial states copied from pinned host memory and the final states + status
copied back inside the timed region.  --impl reference times the CPU oracle
on a bounded sample of the same workload on the host cores.

--workload flyby runs the 4096-trajectory Venus-flyby workload (Sun + 8
planets + Moon, 4 years, segment halving) with the same pairing; uneven and
adjoint run the 1,048,576-trajectory uneven batch and the reverse-mode
workload, each printing its own line.

With N > 1 (torchrun) each rank propagates its own trajectories (weak
scaling, no data-path collective); rank 0 prints the max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "trajectories/s (N-body, <=1e-10 rel err): mixed+batched vs plain FP64 GPU"
UNIT = "trajectories/s"
IC_PER_RANK = {"precision": 65536, "flyby": 4096}

# DRAM bytes (read + write) per trajectory-sweep of each kernel, from one ncu
# capture of that kernel (dram__bytes_read.sum + dram__bytes_write.sum over the
# captured launches / their trajectory-sweeps); None until taken on the current
# kernel.  A line's traffic is this figure times the launch's sweeps.
# contract: k_contract_split, both passes of a second-order FP64 round with all
# 16,384 trajectories of config 3 on the FP64 list (plain FP64 run, rounds 1
# and 2): 334.5 and 331.8 MB per round, 20.3 KB per trajectory-sweep.
TRAFFIC_BYTES_PER_SWEEP = {"contract": 20_300, "fp32": None}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def fp64_tensor_peak_tflops():
    """FP64 tensor-core peak: the measured bf16 dense peak times the nominal
    FP64/bf16 ratio (1.25 / 2250 TFLOP/s); fallback 1.9 PFLOP/s bf16."""
    pk = _peaks()
    bf16 = pk.get("bf16_tflops")
    src = "measured bf16 x nominal fp64/bf16 ratio"
    if bf16 is None:
        bf16, src = 1900.0, "fallback bf16 x nominal fp64/bf16 ratio"
    return bf16 * 1.25 / 2250.0, src


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int = 0):
        self.idx = gpu_index
        self.proc = None
        self.lines = []
        self.thr = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thr = threading.Thread(target=self._read, daemon=True)
        self.thr.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thr:
            self.thr.join(timeout=2)
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
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- distributed
def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x: float, world: int, device=None) -> float:
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def shard(n_total: int, world: int, rank: int):
    """Contiguous slice of the trajectory index space owned by `rank`."""
    lo = n_total * rank // world
    hi = n_total * (rank + 1) // world
    return lo, hi


# ----------------------------------------------------------------------------- oracle timing
def oracle_rate(w, n_sample: int, threads: int, order: int = 1):
    """Times the CPU oracle on the first n_sample trajectories, with the sweep
    of the given order; returns (traj/s, seconds)."""
    from oracle import oracle as ora
    ora.build()
    m = ora.Model.from_workload(w)
    o = ora.Opts(N=w.N, segments=w.segments, seg_mode=w.seg_mode, tol=w.tol, max_iters=w.max_iters,
                 max_depth=w.max_depth, order=order)
    x = w.x0[:n_sample]
    t = time.perf_counter()
    ora.propagate(m, o, x, w.t0, w.tf, threads=threads)
    dt = time.perf_counter() - t
    return n_sample / dt, dt


def headline_workload(args, n_total):
    """The workload of the paired line: config 3 (precision study) or config 2 (flyby)."""
    from paper_2301_03989_gb300 import workloads as W
    if args.workload == "precision":
        return W.config3(M=n_total)
    return W.config2(M=n_total, years=args.years)


def cpu_sample_note(w, n, secs, cores, order=1):
    arc = "2-year" if w.name.startswith("cfg3") else f"{(w.tf - w.t0) / 31557600.0:g}-year"
    kind = "second-order" if order == 2 else "first-order"
    return (f"seeded subset: first {n} of the workload's trajectories, full {arc} arcs, {kind} sweeps, "
            f"{secs:.1f} s on {cores} threads")


def run_reference(args, world, rank):
    """--impl reference: the oracle as it stands on the host cores."""
    if rank != 0:
        return 0
    cores = os.cpu_count() or 1
    w = headline_workload(args, IC_PER_RANK[args.workload])
    n_sample = args.ref_sample or (1024 if args.workload == "precision" else 128)
    for _ in range(args.warmup):
        oracle_rate(w, max(cores, n_sample // 8), cores, args.order)
    times = []
    for _ in range(args.steps):
        _, dt = oracle_rate(w, n_sample, cores, args.order)
        times.append(dt)
    ms = 1000.0 * sum(times) / len(times)
    value = n_sample / (ms / 1000.0)
    sample = cpu_sample_note(w, n_sample, ms / 1000.0, cores, args.order) + " per step"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "n_ic": n_sample, "N": w.N, "parallelism": "host threads"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ----------------------------------------------------------------------------- our arm
def fp32_mma_choice(args) -> int:
    """pc_options.fp32_mma: the FP32 sweeps' contraction on the tensor cores
    (three TF32 products) for the large synchronised batches (precision study,
    uneven batch), FP32 multiply-adds with the autotuner's kernel choice for the
    flyby workload's short lists with many bodies (one trajectory per CTA)."""
    if args.fp32_mma != "auto":
        return int(args.fp32_mma)
    return 0 if args.workload == "flyby" else 1


def fp32_contraction_note(args) -> str:
    return ("tensor cores, three TF32 products (fp32_mma = 1)" if fp32_mma_choice(args)
            else "FP32 multiply-adds (fp32_mma = 0)")


def contract_flops_per_sweep(N: int) -> float:
    """Useful FP64 flops of one trajectory-sweep of the contraction: rows 1..N
    of K (row 0 is zero) times N+1 nodes times 6 components, 2 flops each."""
    return 2.0 * N * (N + 1) * 6


def fp32_flops_per_sweep(N: int, B: int) -> float:
    """Useful FP32 flops of one trajectory-sweep of the FP32 phase: the
    contraction (as above) plus the force, (B+1) pair terms of 20 flops plus a
    square root and a division per node."""
    return contract_flops_per_sweep(N) + (N + 1) * (B + 1) * 22.0


def fp32_alu_peak_tflops():
    """FP32 FMA peak from the unit counts and clock: 152 SMs x 128 FP32 lanes x
    2 flops x the measured maximum SM clock (2070 MHz)."""
    mhz = _peaks().get("sm_max_mhz", 2070.0)
    return 152 * 128 * 2 * mhz * 1e6 / 1e12, "152 SMs x 128 FP32 lanes x 2 flops x max SM clock"


def timed_plain(pc, plan, w, x0, xf, st, it, stream, flush, steps, dev):
    """The timed region: `steps` propagations (L2 flushed before each), CUDA
    events on the launch stream around each, no per-kernel instrumentation.
    Returns per-step ms, rounds and the kernel launches counted by the library."""
    import torch
    pc.kernel_times(plan)                       # clear the counters
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    rounds = 0
    torch.cuda.synchronize(dev)
    for k in range(steps):
        flush.zero_()
        ev0[k].record(stream)
        _, r = pc.propagate(plan, x0, w.t0, w.tf, xf, status=st, iters=it, stream=stream)
        rounds += r
        ev1[k].record(stream)
    torch.cuda.synchronize(dev)
    ms = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
    kt = pc.kernel_times(plan)
    return ms, rounds, kt


def timed_steps(pc, plan, w, x0, xf, st, it, stream, flush, steps, dev):
    """Instrumented replay of the timed steps: a CUDA event on the launch stream
    between consecutive kernels of every round (direct launches, one stream),
    summed per kernel.  Returns per-step ms, rounds and kernel times."""
    import torch
    pc.set_profiling(plan, True)
    pc.kernel_times(plan)                       # clear
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    rounds = 0
    torch.cuda.synchronize(dev)
    for k in range(steps):
        flush.zero_()
        ev0[k].record(stream)
        _, r = pc.propagate(plan, x0, w.t0, w.tf, xf, status=st, iters=it, stream=stream)
        rounds += r
        ev1[k].record(stream)
    torch.cuda.synchronize(dev)
    ms = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
    kt = pc.kernel_times(plan)
    pc.set_profiling(plan, False)
    return ms, rounds, kt


def rel_errors(a, b):
    """Per-trajectory relative position / velocity differences of planar [6][M] arrays."""
    er = np.linalg.norm(a[:3] - b[:3], axis=0) / np.linalg.norm(b[:3], axis=0)
    ev = np.linalg.norm(a[3:] - b[3:], axis=0) / np.linalg.norm(b[3:], axis=0)
    return er, ev


def split_flops_per_sweep(N: int) -> float:
    """bf16 tensor-core flops of one trajectory-sweep of the split-digit
    contraction: 28 digit-pair products over 16 ceil((N+1)/16) nodes, 8 ceil(N/8)
    output nodes and 6 components, 2 flops each."""
    return 28 * 2.0 * 16 * ((N + 16) // 16) * 8 * ((N + 7) // 8) * 6


def bf16_peak_tflops():
    """Measured dense bf16 peak (cuBLAS, sustained: the contraction runs inside
    a long step); fallback 1.7 PFLOP/s."""
    pk = _peaks()
    v = pk.get("bf16_tflops_sustained")
    return (v, "measured bf16 dense, sustained") if v else (1700.0, "fallback bf16 dense, sustained")


def kernel_roofline(name, kt, steps, w, B, peaks, split=False, order=2):
    """Roofline of one kernel from the instrumented replay: algorithmic flops of
    the trajectory-sweeps it ran / its summed launch time."""
    launches, ms = kt[name]
    extra = {}
    tb_key = name
    if name == "contract" and split and w.N <= 255:
        if order != 2:
            tb_key = None                   # the traffic figure is of the second-order passes
        sweeps = kt["sweeps64"]
        flops = split_flops_per_sweep(w.N) * sweeps
        peak, src = peaks["bf16_tensor"]
        bound, kern, dt = "tensor", "k_contract_split (exact 8-bit digit products, bf16 mma.sync m16n8k16)", "bf16"
        if ms > 0:
            extra["fp64_equivalent_tflops"] = contract_flops_per_sweep(w.N) * sweeps / (ms / 1000.0) / 1e12
            extra["fp64_equivalent_frac_of_fp64_peak"] = extra["fp64_equivalent_tflops"] / peaks["fp64_tensor"][0]
    elif name == "contract":
        tb_key = None                       # no capture of the DMMA kernel in this build
        flops = contract_flops_per_sweep(w.N) * kt["sweeps64"]
        peak, src = peaks["fp64_tensor"]
        bound, kern, dt = "tensor", "k_contract (FP64 DMMA mma.sync m16n8k4)", "f64"
        sweeps = kt["sweeps64"]
    elif name == "fp32":
        flops = fp32_flops_per_sweep(w.N, B) * kt["sweeps32"]
        peak, src = peaks["fp32_alu"]
        bound, kern, dt = "alu", "k_fp32 (FP32 sweeps: force + contraction, both modes)", "f32"
        sweeps = kt["sweeps32"]
    else:
        return None
    achieved = flops / (ms / 1000.0) / 1e12 if ms > 0 else 0.0
    tb = TRAFFIC_BYTES_PER_SWEEP.get(tb_key) if tb_key else None
    return dict({"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                 "frac": achieved / peak if peak else None,
                 "traffic": None if tb is None else tb * sweeps / max(1, launches),
                 "kernel": kern, "dtype": dt, "peak_source": src, "launches": launches,
                 "avg_launch_us": 1000.0 * ms / max(1, launches),
                 "algorithmic_flops_per_launch": flops / max(1, launches),
                 "trajectory_sweeps_per_launch": sweeps / max(1, launches)}, **extra)


def run_ours(args, world, rank, local):
    import torch
    from paper_2301_03989_gb300 import build as B
    from paper_2301_03989_gb300 import pcprop as pc
    from paper_2301_03989_gb300 import workloads as W

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    B.build()
    wall = headline_workload(args, args.n_ic * world)
    lo, hi = shard(wall.n_ic, world, rank)
    w = wall.subset(np.arange(lo, hi))
    M = w.n_ic
    nB = len(w.mu)
    mixed = args.precision == "mixed"
    switch_tol = args.switch_tol if args.switch_tol is not None else (1e-6 if args.workload == "precision" else 0.0)
    torch.cuda.synchronize(dev)
    t_plan = time.perf_counter()
    contraction = pc.PC_CONTRACT_SPLIT if args.contraction == "split" else pc.PC_CONTRACT_DMMA
    plan = pc.plan_from_workload(w, precision=pc.PC_PREC_MIXED if mixed else pc.PC_PREC_FP64,
                                 switch_tol=switch_tol, contraction=contraction, order=args.order,
                                 fp32_mma=fp32_mma_choice(args))
    torch.cuda.synchronize(dev)
    plan_ms = 1000.0 * (time.perf_counter() - t_plan)   # operator build + uploads, reported apart
    stream = torch.cuda.Stream(device=dev)
    x0 = torch.as_tensor(W.to_planar(w.x0), device=dev)
    xf = torch.zeros_like(x0)
    st = torch.zeros(M, dtype=torch.int32, device=dev)
    it = torch.zeros(M, dtype=torch.int32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > 129 MB L2

    with torch.cuda.stream(stream):
        tuning = pc.get_tuning(plan)
        if args.autotune:
            tuning = pc.autotune(plan, x0, w.t0, w.tf, max_rounds=256, stream=stream)
        for _ in range(args.warmup):
            pc.propagate(plan, x0, w.t0, w.tf, xf, status=st, iters=it, stream=stream)
        torch.cuda.synchronize(dev)
        if world > 1:
            torch.distributed.barrier()
        clocks = ClockSampler(local)
        clocks.start()
        step_ms, rounds_total, kt_plain = timed_plain(pc, plan, w, x0, xf, st, it, stream, flush, args.steps, dev)
        if world > 1:
            torch.distributed.barrier()
        clk = clocks.stop()
        xf_main = xf.clone()
        status = st.cpu().numpy()
        # per-kernel times: the same steps again with an event between kernels
        prof_ms, _, ktimes = timed_steps(pc, plan, w, x0, xf, st, it, stream, flush, args.prof_steps, dev)

        # end to end through the C ABI with host buffers
        hx0 = torch.as_tensor(W.to_planar(w.x0)).pin_memory()
        hxf = torch.empty_like(hx0).pin_memory()
        hst = torch.empty(M, dtype=torch.int32).pin_memory()
        e2e_ms = []
        for k in range(max(1, args.steps)):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize(dev)
            a.record(stream)
            x0.copy_(hx0, non_blocking=True)
            pc.propagate(plan, x0, w.t0, w.tf, xf, status=st, iters=it, stream=stream)
            hxf.copy_(xf, non_blocking=True)
            hst.copy_(st, non_blocking=True)
            b.record(stream)
            b.synchronize()
            e2e_ms.append(a.elapsed_time(b))

        # the plain FP64 GPU sweep on the same inputs (the metric's comparator),
        # timed exactly like the headline: same warm-up and step counts, graph
        # replay, no instrumentation; then a separate instrumented replay
        plain = None
        if mixed and not args.no_plain:
            plan64 = pc.plan_from_workload(w, precision=pc.PC_PREC_FP64, contraction=contraction, order=args.order)
            xf64 = torch.zeros_like(x0)
            st64 = torch.zeros_like(st)
            it64 = torch.zeros_like(it)
            if args.autotune:
                pc.autotune(plan64, x0, w.t0, w.tf, max_rounds=256, stream=stream)
            for _ in range(args.warmup):
                pc.propagate(plan64, x0, w.t0, w.tf, xf64, status=st64, iters=it64, stream=stream)
            clk64 = ClockSampler(local)
            clk64.start()
            ms64, rounds64, _ = timed_plain(pc, plan64, w, x0, xf64, st64, it64, stream, flush, args.steps, dev)
            clk64 = clk64.stop()
            _, _, kt64 = timed_steps(pc, plan64, w, x0, xf64, st64, it64, stream, flush, 1, dev)
            er, ev = rel_errors(xf_main.cpu().numpy(), xf64.cpu().numpy())
            plain = dict(ms=sum(ms64) / len(ms64), ms_all=ms64, kt=kt64, rounds=rounds64 / len(ms64), er=er, ev=ev,
                         clocks=clk64, status=int((st64.cpu().numpy() != 0).sum()))
            plan64.close()

    ms = sum(step_ms) / len(step_ms)
    ms_max = max_over_ranks(ms, world, dev)
    e2e = sum(e2e_ms) / len(e2e_ms)
    e2e_max = max_over_ranks(e2e, world, dev)
    total_ic = wall.n_ic
    value = total_ic / (ms_max / 1000.0)
    e2e_value = total_ic / (e2e_max / 1000.0)

    # roofline of the dominant kernel (by time in the instrumented replay)
    names = pc.KERNEL_NAMES
    peaks = {"fp64_tensor": fp64_tensor_peak_tflops(), "fp32_alu": fp32_alu_peak_tflops(),
             "bf16_tensor": bf16_peak_tflops()}
    tsum = sum(ktimes[k][1] for k in names)
    kname = max(names, key=lambda k: ktimes[k][1])
    by_kernel = {k: kernel_roofline(k, ktimes, args.prof_steps, w, nB, peaks, split=args.contraction == "split",
                                    order=args.order)
                 for k in ("contract", "fp32")}
    roof = by_kernel.get(kname) or by_kernel["contract"]
    roof = dict(roof, dominant_by_time=kname,
                kernel_share={k: ktimes[k][1] / max(1e-9, tsum) for k in names},
                timing="CUDA events between consecutive kernels on the launch stream, over an instrumented replay "
                       "of the timed steps (direct launches, one stream)")

    line = None
    if rank == 0:
        cores = os.cpu_count() or 1
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            n_cpu = min(M, args.cpu_sample or (4096 if args.workload == "precision" else 256))
            rate, secs = oracle_rate(w, n_cpu, cores, args.order)
            n1 = min(M, max(1, n_cpu // 16))
            rate1, secs1 = oracle_rate(w, n1, 1, args.order)
            cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": cpu_sample_note(w, n_cpu, secs, cores, args.order),
                   "single_thread": {"value": rate1, "unit": UNIT, "cores": 1,
                                     "sample": f"first {n1} trajectories, {secs1:.1f} s"}}
        stats = {"sweep_rounds_per_step": rounds_total / max(1, args.steps),
                 "trajectory_sweeps_fp64_per_step": ktimes["sweeps64"] / max(1, args.prof_steps),
                 "trajectory_sweeps_fp32_per_step": ktimes["sweeps32"] / max(1, args.prof_steps),
                 "status_nonzero": int((status != 0).sum()),
                 "kernel_ms_per_step": {k: ktimes[k][1] / args.prof_steps for k in names},
                 "instrumented_ms_per_step": sum(prof_ms) / len(prof_ms),
                 "plan_create_ms": plan_ms,
                 "ms_per_step_all": step_ms,
                 "ms_per_step_median": statistics.median(step_ms),
                 "roofline_by_kernel": by_kernel}
        if plain is not None:
            stats["plain_fp64"] = {
                "value": total_ic / (plain["ms"] / 1000.0), "unit": UNIT, "ms_per_step": plain["ms"],
                "ms_per_step_all": plain["ms_all"], "steps": args.steps, "warmup": args.warmup,
                "timing": "same as the headline: graph replay, no instrumentation, L2 flushed, CUDA events",
                "sweep_rounds_per_step": plain["rounds"],
                "trajectory_sweeps_fp64_per_step": plain["kt"]["sweeps64"],
                "kernel_ms_per_step_instrumented": {k: plain["kt"][k][1] for k in names},
                "status_nonzero": plain["status"], "clocks": plain["clocks"],
                "speedup_mixed_over_plain": plain["ms"] / ms}
            stats["mixed_vs_plain_fp64_rel_err"] = {
                "pos_max": float(plain["er"].max()), "pos_median": float(np.median(plain["er"])),
                "vel_max": float(plain["ev"].max()), "vel_median": float(np.median(plain["ev"]))}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "mixed fp32->f64" if mixed else "f64", "data": "synthetic",
            "config": {"workload": w.name, "n_ic_per_gpu": M, "N": w.N,
                       "arc_years": round((w.tf - w.t0) / 31557600.0, 3), "tol": w.tol,
                       "path": ("mixed FP32->FP64 batched sweep" if mixed else "plain FP64 batched sweep")
                               + " (per-trajectory segments, compaction, "
                               + ("second-order" if args.order == 2 else "first-order") + " sweeps)",
                       "switch_tol": switch_tol if mixed else None,
                       "sweep_order": args.order,
                       "fp64_contraction": ("exact 8-bit digit products on the bf16 tensor cores"
                                            if args.contraction == "split" else "FP64 tensor cores (DMMA)"),
                       "fp32_contraction": fp32_contraction_note(args) if mixed else None,
                       "l2": "flushed between steps (256 MB write)", "parallelism": f"dp{world}",
                       "tuning": tuning},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(hx0.numel() * 8),
                    "d2h_bytes_per_step": int(hxf.numel() * 8 + hst.numel() * 4)},
            "gpu_launches": int(kt_plain["kernel_launches"]),
            "roofline": roof,
            "cpu_baseline": cpu,
            "clocks": clk,
            "stats": stats,
        }
        print(json.dumps(line))
    plan.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


# ----------------------------------------------------------------------------- other workloads
def _time_calls(fn, steps, warmup, stream, flush, dev):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize(dev)
    ms = []
    for _ in range(steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    return ms


def run_aux(args, world, rank, local):
    """--workload uneven | adjoint (1 GPU): uneven batching (up to 1,048,576
    trajectories of mixed arc length, degree and segment count, degree groups
    on concurrent streams; mixed precision, or plain FP64 with --precision
    fp64) and reverse mode (config-4 flybys: forward pass with tape plus one
    reverse sweep).  Each prints one JSON line with its own metric.  Their
    errors against the CPU oracle are checked by the GPU tests
    (tests/test_gpu_uneven.py, tests/test_gpu_adjoint.py), not here."""
    import torch
    from paper_2301_03989_gb300 import build as B
    from paper_2301_03989_gb300 import pcprop as pc
    from paper_2301_03989_gb300 import workloads as W
    if world > 1:
        raise SystemExit("the extra workloads run on one GPU")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    B.build()
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    cores = os.cpu_count() or 1
    rng = np.random.default_rng(0)
    stats, config = {}, {}
    clocks = ClockSampler(local)
    with torch.cuda.stream(stream):
        if args.workload == "uneven":
            uw = W.config5(M=args.n_ic or 1048576)
            M = uw.n_ic
            perm, degs, counts = uw.groups()
            plans = []
            b = uw.base
            prec = pc.PC_PREC_FP64 if args.precision == "fp64" else pc.PC_PREC_MIXED
            for d in degs:
                o = pc.options_default(tol=b.tol, max_iters=b.max_iters, max_depth=b.max_depth, seg_mode=0,
                                       precision=prec, fp32_mma=fp32_mma_choice(args))
                plans.append(pc.plan_create(int(d), 4, b.mu_central, b.mu, b.t_begin, b.granule, b.coef,
                                            b.indirect, o))
            x0 = torch.as_tensor(W.to_planar(uw.x0[perm]), device=dev)
            t0 = torch.as_tensor(uw.t0[perm], device=dev)
            tf = torch.as_tensor(uw.tf[perm], device=dev)
            sg = torch.as_tensor(uw.S[perm].astype(np.int32), device=dev)
            xf = torch.zeros_like(x0)
            st = torch.zeros(M, dtype=torch.int32, device=dev)
            for p_ in plans:
                pc.kernel_times(p_)
            clocks.start()
            ms = _time_calls(lambda: pc.propagate_groups(plans, counts, x0, t0, tf, xf, segments=sg, status=st,
                                                         stream=stream), args.steps, args.warmup, stream, flush, dev)
            clk = clocks.stop()
            n_steps = args.steps + args.warmup
            launches = sum(pc.kernel_times(p_)["kernel_launches"] for p_ in plans) // n_steps * args.steps
            stats["status_nonzero"] = int((st.cpu().numpy() != 0).sum())
            stats["groups"] = {int(d): int(c) for d, c in zip(degs, counts)}
            for p_ in plans:
                p_.close()
            ms = float(np.mean(ms))
            metric = ("trajectories/s (uneven arcs 0.5-10 yr, N in {32,64,128,256}, 4-80 segments): "
                      + ("plain FP64" if args.precision == "fp64" else "mixed precision"))
            config = {"workload": uw.name, "n_ic": M, "degrees": [int(d) for d in degs], "precision": args.precision,
                      "fp32_contraction": fp32_contraction_note(args)}
        else:  # adjoint
            w = W.config4(M=args.n_ic or 1024)
            M = w.n_ic
            plan = pc.plan_from_workload(w)
            x0 = torch.as_tensor(W.to_planar(w.x0), device=dev)
            cap = 256
            rec = pc.tape_record(plan)
            tape = torch.zeros(M * cap * rec, dtype=torch.float64, device=dev)
            t0 = torch.full((M,), w.t0, dtype=torch.float64, device=dev)
            tf = torch.full((M,), w.tf, dtype=torch.float64, device=dev)
            xf = torch.zeros_like(x0)
            ns = torch.zeros(M, dtype=torch.int32, device=dev)
            xb = torch.as_tensor(rng.standard_normal((6, M)), device=dev)
            x0b = torch.zeros_like(xb)

            def fwd():
                pc.propagate_tape(plan, x0, t0, tf, xf, ns, tape, cap, stream=stream)

            def both():
                fwd()
                pc.adjoint_tape(plan, ns, cap, tape, xb, x0b, stream=stream)
            pc.kernel_times(plan)
            clocks.start()
            ms = _time_calls(both, args.steps, args.warmup, stream, flush, dev)
            clk = clocks.stop()
            launches = pc.kernel_times(plan)["kernel_launches"] // (args.steps + args.warmup) * args.steps
            ms_f = _time_calls(fwd, args.steps, 1, stream, flush, dev)
            ms = float(np.mean(ms))
            stats["forward_with_tape_ms"] = float(np.mean(ms_f))
            stats["reverse_sweep_ms"] = ms - float(np.mean(ms_f))
            stats["segments_max"] = int(ns.max().item())
            plan.close()
            metric = "trajectory gradients/s (config-4 Venus flybys, 1 revolution, N=128): forward tape + reverse sweep"
            config = {"workload": w.name, "n_ic": M, "N": w.N, "tape_segments": cap}
    ms_step = ms if isinstance(ms, float) else float(np.mean(ms))
    line = {"metric": metric, "value": M / (ms_step / 1000.0), "unit": UNIT if args.workload != "adjoint"
            else "trajectory gradients/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "mixed fp32->f64" if args.workload == "uneven" and args.precision == "mixed" else "f64",
            "data": "synthetic", "config": config, "gpu_launches": int(launches),
            "clocks": clk, "stats": stats}
    print(json.dumps(line))
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-sample", type=int, default=None,
                    help="trajectories in the CPU-baseline sample (default 4096 precision, 256 flyby)")
    ap.add_argument("--ref-sample", type=int, default=None,
                    help="trajectories per step of the reference arm (default 1024 precision, 128 flyby)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--switch-tol", type=float, default=None,
                    help="FP32 -> FP64 switch threshold (default 1e-6 precision, 0 flyby: when the FP32 change "
                         "stops falling)")
    ap.add_argument("--order", type=int, choices=[1, 2], default=2,
                    help="1: the paper's sweep; 2: its second-order form (both arms; the default)")
    ap.add_argument("--fp32-mma", choices=["auto", "0", "1"], default="auto",
                    help="FP32 sweeps' contraction on the tensor cores (auto: 1 except for the flyby workload)")
    ap.add_argument("--contraction", choices=["split", "dmma"], default="split",
                    help="FP64 contraction: exact digit products on the bf16 tensor cores, or the FP64 tensor cores")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP64 comparison run")
    ap.add_argument("--prof-steps", type=int, default=2, help="steps of the instrumented per-kernel replay")
    ap.add_argument("--workload", choices=["precision", "flyby", "uneven", "adjoint"], default="precision",
                    help="precision: the headline pairing (config 3); flyby: config 2; uneven, adjoint: their own "
                         "lines")
    ap.add_argument("--n-ic", type=int, default=None, help="trajectories (per GPU for precision / flyby)")
    ap.add_argument("--years", type=float, default=4.0, help="arc length of the flyby workload")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false")
    args = ap.parse_args(argv)
    world, rank, local = dist_setup()
    if args.impl == "reference":
        if args.workload not in IC_PER_RANK:
            args.workload = "precision"
        return run_reference(args, world, rank)
    if args.workload not in IC_PER_RANK:
        return run_aux(args, world, rank, local)
    if args.n_ic is None:
        args.n_ic = IC_PER_RANK[args.workload]
    return run_ours(args, world, rank, local)


if __name__ == "__main__":
    sys.exit(main())
