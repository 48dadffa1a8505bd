"""Benchmark: 3-D compressible Navier-Stokes cell-updates per second of one TVD-RK3 step.

Workload (default): the compressible Taylor-Green vortex on a 128^3 periodic box, Ma 0.1, Re 1600,
Pr 0.71, power-law viscosity, WENO5-Z + HLLC + fourth-order central dissipative fluxes, CFL 0.5,
FP64 state and arithmetic.  Synthetic: the textbook closed-form initial condition.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl fluid|reference] [--workload NAME]

Prints one JSON line.  `value` = interior cells x steps x ranks / (max over ranks of the summed
CUDA-event time of the K timed steps); L2 is flushed before every timed step.  With N > 1 (launched
by torch.distributed.run) the ranks share one solve: the workload's grid is extended N times along
z and split into z-slabs of the workload's size, one per rank (weak scaling), with a halo exchange
over NCCL before every RK3 stage and the time step minimised over the ranks (Section 2.2's block
decomposition).  `--impl reference` times the CPU oracle on a bounded sample of the same workload
instead.
"""
import argparse
import datetime
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

from paper_2406_19494_gb300 import accounting, workloads  # noqa: E402

METRIC = "3D NS cell-updates/s per RK3 step, FP64 vs mixed; adjoint/forward time ratio"
UNIT = "cell-updates/s"

WORKLOADS = {
    "tgv128": lambda: workloads.tgv_case(128),
    "tgv64": lambda: workloads.tgv_case(64),
    "channel192": lambda: workloads.channel_case(192, 128, 128),
    "channel256": lambda: workloads.channel_case(256, 128, 128),
}


def initial_prims(case, centres):
    xc, yc, zc = centres
    if case["name"].startswith("tgv"):
        return workloads.tgv_prims(case, xc, yc, zc)
    return workloads.channel_prims(case, xc, yc, zc, seed=0)


def describe(name, case):
    return {"workload": "%s: %s" % (name, {
        "tgv": "compressible Taylor-Green vortex, periodic [0,2pi]^3, Ma 0.1, Re 1600, Pr 0.71, power-law mu",
        "cha": "compressible channel, Ma_b 1.5, Re_b 3000, tanh(beta=2) walls, isothermal, body force"}[name[:3]]),
        "grid": list(case["n"]), "scheme": "WENO5-%s + HLLC + 4th-order central viscous, TVD-RK3, CFL %.1f"
        % (case["weno"].upper(), case["cfl"]), "precision": "fp64",
        "l2": "flushed before every timed step (256 MiB write)",
        "launch": "face-kernel segment lengths timed once per solver on the initial state (fluid_autotune_faces), before timing"}


# ------------------------------------------------------------------------------------------------
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(ms, device):
    """The largest of the ranks' times (ms); every rank returns the same value.  One rank: ms."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def whole_job_rate(cells, steps, ranks, ms):
    """Cell-updates/s of the whole job: every rank advances its own replica of `cells` cells by
    `steps` steps; the job takes the slowest rank's time `ms`."""
    return cells * steps * ranks / (ms * 1e-3)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 50 ms from before the warm-up (the tool
    takes longer to start than a short timed region lasts); the summary keeps the samples whose
    timestamps fall inside the host-side window of the timed region (mark_start / mark_end)."""
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.t0 = self.t1 = None
        self.out = ""

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def mark_start(self):
        self.t0 = datetime.datetime.now()

    def mark_end(self):
        self.t1 = datetime.datetime.now()

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def _rows(self):
        rows = []
        for line in (self.out or "").strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f")
            except ValueError:
                continue
            rows.append((ts, f[1:]))
        return rows

    def summary(self):
        rows = self._rows()
        window = "timed region"
        if self.t0 is not None and self.t1 is not None:
            slack = datetime.timedelta(milliseconds=60)
            inside = [r for ts, r in rows if self.t0 - slack <= ts <= self.t1 + slack]
        else:
            inside = [r for _, r in rows]
        if not inside and rows:
            # a region shorter than the sampling interval: the samples nearest to it
            mid = self.t0 + (self.t1 - self.t0) / 2 if self.t0 and self.t1 else rows[-1][0]
            inside = [min(rows, key=lambda tr: abs(tr[0] - mid))[1]]
            window = "nearest sample to the timed region"
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        num = lambda x: x.replace(".", "").isdigit()
        sm = [float(r[1]) for r in inside if num(r[1])]
        mx = [float(r[2]) for r in inside if num(r[2])]
        pw = [float(r[3]) for r in inside if num(r[3])]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in inside for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(inside), "window": window,
                "power_w_max": max(pw) if pw else None}


# ------------------------------------------------------------------------------------------------
def timed_steps(s, U, steps, warmup, flush, stream, clock_gpu=None):
    """Warm up, then time `steps` RK3 steps with CUDA events (L2 flushed before each); then, outside
    the timed region, `steps` more steps with the library's event profiler recording every kernel
    (its event records between launches would add to the timed steps).  Returns (total ms of the
    timed steps, per-kernel profile of the profiled ones, clocks of the timed region)."""
    import torch
    clk = ClockSampler(clock_gpu) if clock_gpu is not None else None
    if clk:
        clk.__enter__()
    for _ in range(warmup):
        s.step(U, 1)
    s.check()
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    if clk:
        clk.mark_start()
    for k in range(steps):
        flush.fill_(float(k))
        starts[k].record(stream)
        s.step(U, 1)
        ends[k].record(stream)
    torch.cuda.synchronize()
    if clk:
        clk.mark_end()
        clk.__exit__(None, None, None)
    s.check()
    per_step = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    timed_steps.last_per_step = per_step
    s.profile(True)
    s.profile_read(reset=True)
    for k in range(steps):
        flush.fill_(float(k))
        s.step(U, 1)
    torch.cuda.synchronize()
    prof = s.profile_read(reset=True)
    s.profile(False)
    s.check()
    return sum(per_step), prof, clk


def one_call_ms(s, U, steps, flush, stream):
    """ms per step of one fluid_step call of `steps` steps (the way a run advances), after one
    warm-up call; L2 flushed once before the timed call (the working set of a step exceeds L2)."""
    import torch
    s.step(U, steps)
    s.check()
    flush.fill_(1.0)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    s.step(U, steps)
    b.record(stream)
    torch.cuda.synchronize()
    s.check()
    return a.elapsed_time(b) / steps


def graph_step_ms(s, U, reps, stream):
    """Median ms of one RK3 step replayed from a CUDA graph that captured one single-step
    fluid_step call, over `reps` timed replays after ten untimed ones.  No L2 flush between
    replays: the arrays a step touches (state, stage state, right-hand side, primitives,
    gradients; about 0.5 GB on TGV 128^3) exceed the 126 MB L2."""
    import torch
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        s.step(U, 1)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode="relaxed"):
        s.step(U, 1)
    for _ in range(10):
        g.replay()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        g.replay()
        b.record(stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    s.check()
    del g
    return statistics.median(ts)


def slab_case(base, ws):
    """The workload extended ws times along z (its z-periodic state repeats), to be split into ws
    z-slabs of the workload's own size."""
    n, lo, hi = base["n"], base["lo"], base["hi"]
    return dict(base, n=(n[0], n[1], n[2] * ws), hi=(hi[0], hi[1], lo[2] + (hi[2] - lo[2]) * ws),
                name=base["name"] + "_zslabs%d" % ws)


def run_decomposed(args, ws, rank, local):
    """N > 1: one solve split into z-slabs, one per rank, NCCL halo exchange per RK3 stage."""
    import torch
    import torch.distributed as dist

    from paper_2406_19494_gb300 import build, decomp

    dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    base = WORKLOADS[args.workload]()
    case = slab_case(base, ws)
    blk = decomp.BlockSolver(case, (1, 1, ws), rank, decomp.TorchComm())
    s = blk.solver
    cen = [s.grid(a)[0][3:-3] for a in range(3)]
    W = np.pad(initial_prims(case, cen), [(0, 0)] + [(3, 3)] * 3, mode="edge")
    U0 = s.prim_to_cons(torch.from_numpy(W).cuda())
    s.autotune_faces(U0)
    ncell = base["n"][0] * base["n"][1] * base["n"][2]
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    U = U0.clone()
    clk = ClockSampler(local)
    clk.__enter__()
    blk.step(U, args.warmup)
    s.check()
    torch.cuda.synchronize()
    dist.barrier()
    clk.mark_start()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    for k in range(args.steps):
        flush.fill_(float(k))
        starts[k].record(stream)
        blk.step(U, 1)
        ends[k].record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    clk.mark_end()
    clk.__exit__(None, None, None)
    s.check()
    # the kernel profile from as many steps again, outside the timed region
    s.profile(True)
    s.profile_read(reset=True)
    for k in range(args.steps):
        flush.fill_(float(k))
        blk.step(U, 1)
    torch.cuda.synchronize()
    prof = s.profile_read(reset=True)
    s.profile(False)
    s.check()
    dist.barrier()
    per_step = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    total_ms = max_over_ranks(sum(per_step), "cuda")
    launches = sum(n for _, n in prof.values())
    # end to end: the rank's slab from pinned host memory, one step, back to the host
    Uh = U0.cpu().pin_memory()
    Uout = torch.empty_like(Uh).pin_memory()
    Ue = torch.empty_like(U0)
    e_ms = []
    for k in range(4):
        flush.fill_(float(k))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        Ue.copy_(Uh, non_blocking=True)
        blk.step(Ue, 1)
        Uout.copy_(Ue, non_blocking=True)
        b.record(stream)
        torch.cuda.synchronize()
        if k > 0:
            e_ms.append(a.elapsed_time(b))
    e2e_ms = max_over_ranks(sum(e_ms) / len(e_ms), "cuda")
    face_ms = sum(v[0] for k, v in prof.items() if k.startswith("face_"))
    face_calls = 3 * 3 * args.steps
    t_face = face_ms / face_calls * 1e-3 if face_ms > 0 else None
    peak64 = 152 * 2 * 2 * 2.07e9 / 1e12
    achieved = accounting.cell_axis_flops(3, case["weno"], case["visc"]) * ncell / t_face / 1e12 if t_face else None
    nbytes = Uh.numel() * 8
    result = {
        "metric": METRIC, "value": whole_job_rate(ncell, args.steps, ws, total_ms), "unit": UNIT,
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "ms_per_step_median": statistics.median(per_step), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(describe(args.workload, base), grid=list(case["n"]),
                       parallelism="z-slabs x%d: one %dx%dx%d slab per GPU, NCCL halo exchange (3 layers) "
                                   "before every RK3 stage, dt min-reduced" % ((ws,) + tuple(base["n"]))),
        "e2e": {"value": ncell * ws / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": nbytes,
                "d2h_bytes_per_step": nbytes},
        "gpu_launches": launches,
        "roofline": {"bound": "alu", "kernel": "k_face (x, y, z) with its seam kernel, FP64", "achieved": achieved,
                     "peak": peak64, "unit": "TFLOP/s", "frac": achieved / peak64 if achieved else None,
                     "traffic": None},
        "kernels_ms_per_step": {k: v[0] / args.steps for k, v in prof.items() if v[1]},
        "clocks": clk.summary(),
    }
    if rank == 0:
        print(json.dumps(result), flush=True)
    dist.destroy_process_group()


def run_fluid(args):
    import torch
    import torch.distributed as dist

    from paper_2406_19494_gb300 import build
    from paper_2406_19494_gb300.solver import Solver

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        return run_decomposed(args, ws, rank, local)
    build.build()
    case = WORKLOADS[args.workload]()
    s = Solver(case)
    cen = [s.grid(a)[0][3:-3] for a in range(3)]
    W = np.pad(initial_prims(case, cen), [(0, 0)] + [(3, 3)] * 3, mode="edge")
    Wd = torch.from_numpy(W).cuda()
    U0 = s.prim_to_cons(Wd)
    del Wd
    # launch shapes of the face kernels timed once on the initial state (results do not depend on
    # them), before any timed region
    s.autotune_faces(U0)
    ncell = case["n"][0] * case["n"][1] * case["n"][2]
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    # ---- timed region (FP64 path): K steps, barrier + synchronize on both sides ----------------
    U = U0.clone()
    total_ms, prof, clk = timed_steps(s, U, args.steps, args.warmup, flush, stream, clock_gpu=local)
    median_ms = statistics.median(timed_steps.last_per_step)
    launches = sum(n for _, n in prof.values())

    # ---- the mixed FP32-flux / FP64-state path on the same workload ------------------------------
    sm = Solver(case, precision="mixed")
    if args.mixed_tiles == "bulk":
        sm.tune_faces(0, 1)
    Um = U0.clone()
    mixed_ms, mprof, _ = timed_steps(sm, Um, args.steps, args.warmup, flush, stream)
    mixed_ms = max_over_ranks(mixed_ms, "cuda")
    mixed_err = mixed_vs_fp64(s, sm, U, Um, case, args.warmup + 2 * args.steps)
    if not args.no_mixed_errors and args.workload == "tgv128":
        mixed_err["stated_workloads"] = mixed_errors_stated()
    one_call = None
    if ws == 1:
        Uc = U0.clone()
        one_call = {"fp64_ms_per_step": one_call_ms(s, Uc, args.steps, flush, stream)}
        Uc.copy_(U0)
        one_call["mixed_ms_per_step"] = one_call_ms(sm, Uc, args.steps, flush, stream)
        one_call["note"] = ("K steps in one fluid_step call after a warm-up call of K; L2 flushed "
                            "once before the call, the working set of a step (~0.5 GB) exceeds L2")
        Uc.copy_(U0)
        graph = {"fp64_ms_per_step": graph_step_ms(s, Uc, 50, stream)}
        Uc.copy_(U0)
        graph["mixed_ms_per_step"] = graph_step_ms(sm, Uc, 50, stream)
        graph["note"] = ("median of 50 replays of a CUDA graph holding one single-step fluid_step call, "
                         "after 10 untimed replays; inputs larger than L2, no flush")
        one_call["graph"] = graph
        del Uc

    # ---- the paper's channel scheme (TENO6-A + sixth-order central, FP64) ------------------------
    teno = measure_teno(flush, stream, args) if not args.no_teno and ws == 1 else None

    # ---- adjoint / forward ratio (the metric's third part) -------------------------------------
    adjoint = measure_adjoint(flush, stream) if not args.no_adjoint else None

    serving = None
    if not args.no_serving:
        reqs = serving_requests()
        serving = {"fp64": measure_serving(reqs, "fp64", whole_job_rate(ncell, args.steps, 1, total_ms)),
                   "mixed": measure_serving(reqs, "mixed", whole_job_rate(ncell, args.steps, 1, mixed_ms))}
        del reqs
    e2 = measure_e2() if args.e2 else None

    # ---- end-to-end through the C ABI with host buffers ---------------------------------------
    Uh = U0.cpu().pin_memory()
    Uout = torch.empty_like(Uh).pin_memory()
    Ue = torch.empty_like(U0)
    nbytes = Uh.numel() * 8
    e_ms = []
    for k in range(max(2, min(args.steps, 5)) + 1):
        flush.fill_(float(k))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        Ue.copy_(Uh, non_blocking=True)
        s.step(Ue, 1)
        Uout.copy_(Ue, non_blocking=True)
        b.record(stream)
        torch.cuda.synchronize()
        if k > 0:
            e_ms.append(a.elapsed_time(b))
    e2e_ms = sum(e_ms) / len(e_ms)
    e2e_ms = max_over_ranks(e2e_ms, "cuda")

    # ---- rooflines of the dominant kernel class (the face kernels) ----------------------------
    def face_time(p, calls):
        """seconds per face-kernel call (one axis of one stage: the face kernel with its seam kernel)"""
        ms = sum(v[0] for k, v in p.items() if k.startswith("face_"))
        return (ms / calls * 1e-3) if calls and ms > 0 else None

    face_calls = len(case["n"]) * 3 * args.steps

    fp64_probe = ctypes_peak(s, 0)
    fp32_probe = ctypes_peak(s, 1)
    # peaks from unit counts and the maximum SM clock: FP64 152 SMs x 2 FMA/clk x 2 flops, FP32
    # 152 SMs x 128 lanes x 2 flops, at 2.07 GHz; HBM from the measured copy bandwidth
    peak64 = 152 * 2 * 2 * 2.07e9 / 1e12
    peak32 = 152 * 128 * 2 * 2.07e9 / 1e12
    hbm = measured_hbm_gbs()
    t_face = face_time(prof, face_calls)
    per_launch_flops = accounting.cell_axis_flops(3, case["weno"], case["visc"]) * ncell
    achieved = per_launch_flops / t_face / 1e12 if t_face else None
    tm_face = face_time(mprof, face_calls)
    m64 = accounting.mixed_cell_axis_flops64() * ncell / tm_face / 1e12
    m32 = accounting.mixed_cell_axis_flops32(case["weno"], case["visc"]) * ncell / tm_face / 1e12
    mbytes = accounting.mixed_face_bytes() * ncell / tm_face / 1e9

    value = whole_job_rate(ncell, args.steps, ws, total_ms)
    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "ms_per_step_median": median_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(describe(args.workload, case), parallelism="1 GPU"),
        "e2e": {"value": ncell * ws / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": nbytes,
                "d2h_bytes_per_step": nbytes},
        "gpu_launches": launches,
        "roofline": {"bound": "alu", "kernel": "k_face (x, y, z) with its seam kernel, FP64", "achieved": achieved, "peak": peak64,
                     "unit": "TFLOP/s", "frac": achieved / peak64 if achieved else None,
                     "traffic": face_traffic(ncell),
                     "traffic_note": "bytes per launch: ncu dram__bytes_read.sum + dram__bytes_write.sum of the x, y and z face launches of this workload (mean), null when the kernel sources changed since that capture",
                     "peak_source": "FP64 units x max SM clock (152 SMs x 2 FMA/clk x 2 flops x 2.07 GHz); "
                                    "measured by the FMA probe as fp64_fma_probe_tflops",
                     "fp64_fma_probe_tflops": fp64_probe / 1e3 if fp64_probe else None,
                     "flops_per_cell_axis": accounting.cell_axis_flops(3, case["weno"], case["visc"]),
                     "flops_basis": "algorithmic: the oracle's operations on counting scalars, per cell and axis",
                     "flops_per_cell_update": accounting.cell_update_flops(3, case["weno"], case["visc"]),
                     "flops_executed_per_cell_axis": accounting.EXECUTED["k_face"],
                     "achieved_executed": (accounting.EXECUTED["k_face"] * ncell / t_face / 1e12) if t_face else None,
                     "frac_executed": (accounting.EXECUTED["k_face"] * ncell / t_face / 1e12 / peak64) if t_face else None},
        "kernels_ms_per_step": {k: v[0] / args.steps for k, v in prof.items() if v[1]},
        "mixed": {
            "value": whole_job_rate(ncell, args.steps, ws, mixed_ms), "unit": UNIT,
            "ms_per_step": mixed_ms / args.steps, "speedup_vs_fp64": total_ms / mixed_ms,
            "dtype": "f32 fluxes / f64 state", "tiles": args.mixed_tiles,
            "error_vs_fp64": mixed_err,
            "kernels_ms_per_step": {k: v[0] / args.steps for k, v in mprof.items() if v[1]},
            "roofline_step": mixed_step_roofline(mixed_ms / args.steps, ncell),
            "roofline_face": {
                "fp64": {"achieved": m64, "peak": peak64, "unit": "TFLOP/s", "frac": m64 / peak64},
                "fp32": {"achieved": m32, "peak": peak32, "unit": "TFLOP/s", "frac": m32 / peak32,
                         "fp32_fma_probe_tflops": fp32_probe / 1e3 if fp32_probe else None},
                "hbm": {"achieved": mbytes, "peak": hbm, "unit": "GB/s", "frac": mbytes / hbm},
                "flops64_per_cell_axis": accounting.mixed_cell_axis_flops64(),
                "flops32_per_cell_axis": accounting.mixed_cell_axis_flops32(case["weno"], case["visc"]),
                "bytes_per_cell_axis": accounting.mixed_face_bytes()},
        },
        "teno6a": teno,
        "adjoint": adjoint,
        "serving": serving,
        "e2_boundary_layer": e2,
        "clocks": clk.summary(),
        "steps_in_one_call": one_call,
        "pid_s": {"per_cell": total_ms * 1e-3 / args.steps / ncell,
                  "per_dof": total_ms * 1e-3 / args.steps / (5 * ncell)},
    }
    if not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(args, case, samples=1)
    print(json.dumps(result), flush=True)


def mixed_vs_fp64(s64, s32, U64, U32, case, steps):
    """Differences between the FP64 and the mixed solutions after the same `steps` RK3 steps from
    the same state (both timed runs): the state per variable (max |dU| / max |U|), the kinetic
    energy and its rate of change (the TGV dissipation rate), with the rate from each solver's own
    right-hand side.  Plain host arithmetic on copies; diagnostics, not part of the solver."""
    import torch
    inner = (slice(None),) + tuple(slice(3, 3 + case["n"][a]) for a in (2, 1, 0))
    a = U64.cpu().numpy()[inner]
    b = U32.cpu().numpy()[inner]
    ra = s64.rhs(U64).cpu().numpy()[inner]
    rb = s32.rhs(U32).cpu().numpy()[inner]
    torch.cuda.synchronize()

    def ke_and_rate(u, r):
        m2 = u[1] ** 2 + u[2] ** 2 + u[3] ** 2
        ke = 0.5 * m2 / u[0]
        # d/dt (|m|^2 / 2 rho) = (m . dm/dt) / rho - |m|^2 / (2 rho^2) drho/dt
        rate = (u[1] * r[1] + u[2] * r[2] + u[3] * r[3]) / u[0] - 0.5 * m2 / u[0] ** 2 * r[0]
        return float(ke.sum()), float(rate.sum())
    ke_a, rate_a = ke_and_rate(a, ra)
    ke_b, rate_b = ke_and_rate(b, rb)
    scale = np.max(np.abs(a.reshape(5, -1)), axis=1)
    scale = np.where(scale > 0, scale, 1.0)
    return {"steps": steps,
            "state_max_rel": [float(v) for v in np.max(np.abs((a - b).reshape(5, -1)), axis=1) / scale],
            "kinetic_energy_rel": abs(ke_b - ke_a) / abs(ke_a),
            "kinetic_energy_rate_rel": abs(rate_b - rate_a) / abs(rate_a)}


def mixed_errors_stated(tgv_steps=1000, channel_steps=50, bl_steps=200):
    """Mixed precision against FP64 on the stated workloads, from the same initial states with the
    same frozen time step (the FP64 CFL step of the initial state), so both compare at the same
    times.  TGV 128^3 over its 1000 steps: the kinetic energy and its dissipation rate (from each
    solver's own right-hand side) every 100 steps; channel 192x128x128: the wall heat flux and wall
    shear of both walls (fluid_wall_fluxes) after channel_steps; porous boundary layer 512x128: the
    same on its porous wall after bl_steps.  Host diagnostics on copies."""
    import torch
    from paper_2406_19494_gb300.solver import Solver

    def setup(case, prims_of, extra=None):
        s = Solver(case)
        cen = [s.grid(a)[0] for a in range(3)]
        h = [3 if a < case["ndim"] else 0 for a in range(3)]
        cen = [cen[a][h[a]:len(cen[a]) - h[a]] for a in range(3)]
        W = prims_of(case, cen)
        pad = [(0, 0)] + [(h[a], h[a]) for a in (2, 1, 0)]
        U0 = s.prim_to_cons(torch.from_numpy(np.ascontiguousarray(np.pad(W, pad, mode="edge"))).cuda())
        dt = float(s.compute_dt(U0).item())
        out = {}
        for prec in ("fp64", "mixed"):
            sp = Solver(dict(case, dt_fixed=dt), precision=prec)
            if extra:
                extra(sp)
            out[prec] = sp
        return out, U0, dt

    def rel(a, b):
        return abs(a - b) / abs(b) if b != 0 else abs(a - b)

    res = {}
    # Taylor-Green 128^3
    case = workloads.tgv_case(128)
    sv, U0, dt = setup(case, lambda c, cen: workloads.tgv_prims(c, *cen))
    inner = (slice(None),) + tuple(slice(3, 3 + case["n"][a]) for a in (2, 1, 0))
    vol = (2 * math.pi / 128) ** 3
    U = {p: U0.clone() for p in sv}
    samples = []
    for k in range(0, tgv_steps + 1, 100):
        if k:
            for p in sv:
                sv[p].step(U[p], 100)
        ke, eps = {}, {}
        for p in sv:
            u = U[p].cpu().numpy()[inner]
            r = sv[p].rhs(U[p]).cpu().numpy()[inner]
            m2 = u[1] ** 2 + u[2] ** 2 + u[3] ** 2
            ke[p] = float((0.5 * m2 / u[0]).sum()) * vol
            eps[p] = -float(((u[1] * r[1] + u[2] * r[2] + u[3] * r[3]) / u[0] - 0.5 * m2 / u[0] ** 2 * r[0]).sum()) * vol
        samples.append({"step": k, "t": k * dt, "ke_rel": rel(ke["mixed"], ke["fp64"]),
                        "dissipation_rate_rel": rel(eps["mixed"], eps["fp64"]),
                        "dissipation_rate_fp64": eps["fp64"]})
    res["tgv128_1000_steps"] = {
        "dt": dt, "samples": samples,
        "max_dissipation_rate_rel": max(x["dissipation_rate_rel"] for x in samples),
        "max_ke_rel": max(x["ke_rel"] for x in samples)}
    del U, sv, U0
    torch.cuda.empty_cache()
    # channel 192x128x128: both walls
    case = workloads.channel_case(192, 128, 128)
    sv, U0, dt = setup(case, lambda c, cen: workloads.channel_prims(c, *cen, seed=0))
    walls = {}
    for p in sv:
        U = U0.clone()
        sv[p].step(U, channel_steps)
        walls[p] = [tuple(x.cpu().numpy() for x in sv[p].wall_fluxes(U, 1, sd)) for sd in (0, 1)]
    out = {"steps": channel_steps, "dt": dt}
    for sd in (0, 1):
        q64, t64 = walls["fp64"][sd]
        q32, t32 = walls["mixed"][sd]
        out["wall%d" % sd] = {"mean_heat_flux_rel": rel(q32.mean(), q64.mean()),
                              "mean_wall_shear_rel": rel(t32.mean(), t64.mean()),
                              "max_heat_flux_err_over_max": float(np.max(np.abs(q32 - q64)) / np.max(np.abs(q64))),
                              "max_wall_shear_err_over_max": float(np.max(np.abs(t32 - t64)) / np.max(np.abs(t64)))}
    res["channel192_walls"] = out
    del sv, U0
    torch.cuda.empty_cache()
    # porous boundary layer 512x128
    case = workloads.porous_bl_case(512, 128)
    phi = torch.from_numpy(workloads.porous_phi(case, seed=0)).cuda()

    def bl_extra(sp):
        yc = sp.grid(1)[0]
        sp.set_inflow(0, 0, torch.from_numpy(workloads.porous_bl_inflow(case, yc)).cuda())
        sp.set_wall_params(phi)

    sv, U0, dt = setup(case, lambda c, cen: workloads.porous_bl_prims(c, cen[0], cen[1]), bl_extra)
    fx = {}
    for p in sv:
        U = U0.clone()
        sv[p].step(U, bl_steps)
        fx[p] = tuple(x.cpu().numpy() for x in sv[p].wall_fluxes(U, 1, 0))
    res["porous_bl512_wall"] = {
        "steps": bl_steps, "dt": dt,
        "integrated_heat_flux_rel": rel(float(fx["mixed"][0].sum()), float(fx["fp64"][0].sum())),
        "mean_wall_shear_rel": rel(float(fx["mixed"][1].mean()), float(fx["fp64"][1].mean())),
        "max_heat_flux_err_over_max": float(np.max(np.abs(fx["mixed"][0] - fx["fp64"][0])) / np.max(np.abs(fx["fp64"][0]))),
        "max_wall_shear_err_over_max": float(np.max(np.abs(fx["mixed"][1] - fx["fp64"][1])) / np.max(np.abs(fx["fp64"][1])))}
    return res


def measure_teno(flush, stream, args, steps=5):
    """The scheme of the paper's channel computation (TENO6-A with the interpolation limiter, HLLC,
    sixth-order central dissipative fluxes; FP64) on the channel workload, 192 x 128 x 128 cells
    (96 x 64 x 64 with the small --workload tgv64): cell-updates/s per RK3 step and the roofline of
    its face kernels."""
    import torch
    from paper_2406_19494_gb300.solver import Solver
    n = (96, 64, 64) if args.workload == "tgv64" else (192, 128, 128)
    c = dict(workloads.channel_case(*n), weno="teno6a", visc_order=6)
    s = Solver(c)
    cen = [s.grid(a)[0][3:-3] for a in range(3)]
    W = np.pad(workloads.channel_prims(c, *cen, seed=0), [(0, 0)] + [(3, 3)] * 3, mode="edge")
    U = s.prim_to_cons(torch.from_numpy(W).cuda())
    s.autotune_faces(U)
    ncell = c["n"][0] * c["n"][1] * c["n"][2]
    ms, prof, _ = timed_steps(s, U, steps, max(3, args.warmup), flush, stream)
    f = {k: v for k, v in prof.items() if k.startswith("face_")}
    t_face = sum(v[0] for v in f.values()) / (len(c["n"]) * 3 * steps) * 1e-3
    # the oracle's definition forms its smoothness measures as full quadratic forms (each
    # symmetric pair twice), so the executed count is the meaningful one for this kernel
    per_axis_oracle = accounting.cell_axis_flops(3, "teno6a", c["visc"], 6)
    per_axis = accounting.EXECUTED["k_face_teno"]
    achieved = per_axis * ncell / t_face / 1e12
    peak64 = 152 * 2 * 2 * 2.07e9 / 1e12
    return {"workload": "channel %dx%dx%d, TENO6-A + interpolation limiter + HLLC + 6th-order central" % n,
            "value": ncell * steps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps, "steps": steps,
            "dtype": "f64", "kernels_ms_per_step": {k: v[0] / steps for k, v in prof.items() if v[1]},
            "roofline_face": {"bound": "alu", "achieved": achieved, "peak": peak64, "unit": "TFLOP/s",
                              "frac": achieved / peak64, "flops_per_cell_axis": per_axis,
                              "flops_basis": "executed (ncu: 2 DFMA + DADD + DMUL per cell and axis)",
                              "flops_per_cell_axis_oracle_counted": per_axis_oracle}}


def measure_adjoint(flush, stream, steps=5, warmup=3, grad_steps=400, K=20):
    """Adjoint/forward time ratio on the porous boundary layer (512 x 128, Ma 6, frozen dt, FP64):
    one RK3 step vs one adjoint step (with its stage recomputation, and with stored stages), and
    the end-to-end gradient dJ/dphi of the wall heat flux after `grad_steps` steps with checkpoints
    every K steps."""
    import torch
    from paper_2406_19494_gb300.adjoint import wall_heat_loss
    from paper_2406_19494_gb300.solver import Solver
    c = workloads.porous_bl_case(512, 128)
    probe = Solver(c)
    xc, _ = probe.grid(0)
    yc, _ = probe.grid(1)
    W = np.pad(workloads.porous_bl_prims(c, xc[3:-3], yc[3:-3]), [(0, 0), (0, 0), (3, 3), (3, 3)], mode="edge")
    U0 = probe.prim_to_cons(torch.from_numpy(W).cuda())
    dtd = probe.compute_dt(U0).item()
    del probe
    c = dict(c, dt_fixed=0.5 * dtd)
    s = Solver(c, adjoint=True)
    phi = torch.from_numpy(workloads.porous_phi(c, seed=0)).cuda()
    s.set_wall_params(phi)
    s.set_inflow(0, 0, torch.from_numpy(workloads.porous_bl_inflow(c, yc)).cuda())
    ev = lambda: torch.cuda.Event(enable_timing=True)

    def timed(fn):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        tot = 0.0
        for k in range(steps):
            flush.fill_(float(k))
            a, b = ev(), ev()
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            tot += a.elapsed_time(b)
        return tot / steps

    U = U0.clone()
    fwd = timed(lambda: s.step(U, 1))
    Un = U0.clone()
    U1, U2 = torch.zeros_like(U0), torch.zeros_like(U0)
    s.step_stages(Un.clone(), U1, U2)
    lam = torch.zeros_like(U0)
    gphi = torch.zeros_like(phi)
    adj = timed(lambda: s.adjoint_step(Un, lam, gphi))
    adj_stored = timed(lambda: s.adjoint_step(Un, lam, gphi, U1, U2))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    p = phi.clone().requires_grad_(True)
    J = wall_heat_loss(p, s, U0, grad_steps, K, 1, 0)
    J.backward()
    torch.cuda.synchronize()
    t_grad = time.perf_counter() - t0
    del s, U, Un, U1, U2, lam
    # the same ratios on a 3-D grid that fills the GPU (TGV 96^3, periodic, frozen dt)
    c3 = workloads.tgv_case(96)
    probe = Solver(c3)
    cen = [probe.grid(a)[0][3:-3] for a in range(3)]
    W3 = np.pad(initial_prims(c3, cen), [(0, 0)] + [(3, 3)] * 3, mode="edge")
    V0 = probe.prim_to_cons(torch.from_numpy(W3).cuda())
    c3 = dict(c3, dt_fixed=0.5 * probe.compute_dt(V0).item())
    del probe
    s3 = Solver(c3, adjoint=True)
    V = V0.clone()
    fwd3 = timed(lambda: s3.step(V, 1))
    V1, V2 = torch.zeros_like(V0), torch.zeros_like(V0)
    s3.step_stages(V0.clone(), V1, V2)
    mu3 = torch.zeros_like(V0)
    adj3 = timed(lambda: s3.adjoint_step(V0, mu3))
    adj3_stored = timed(lambda: s3.adjoint_step(V0, mu3, None, V1, V2))
    del s3, V, V0, V1, V2, mu3
    return {"workload": "porous boundary layer 512x128, Ma 6, 256 porous wall cells, frozen dt, FP64",
            "forward_ms_per_step": fwd, "adjoint_ms_per_step": adj, "adjoint_stored_stages_ms_per_step": adj_stored,
            "adjoint_forward_ratio": adj / fwd, "adjoint_forward_ratio_stored_stages": adj_stored / fwd,
            "gradient": {"steps": grad_steps, "checkpoint_every": K, "wall_s": t_grad, "J": J.item(),
                         "grad_norm_inf": float(p.grad.abs().max()),
                         "note": "the gradient's backward sweep runs the stored-stage adjoint step"},
            "tgv96_3d": {"forward_ms_per_step": fwd3, "adjoint_ms_per_step": adj3,
                         "adjoint_stored_stages_ms_per_step": adj3_stored,
                         "adjoint_forward_ratio": adj3 / fwd3,
                         "adjoint_forward_ratio_stored_stages": adj3_stored / fwd3}}


SERVING_STEP_SCALE = 100     # the stream's 100..2000 steps per request, divided by this


def serving_requests(count=512, seed=0):
    """The serving stream as stated (512 requests: 70 % 2-D isentropic vortices / four-quadrant
    Riemann problems on 64^2..1024^2, 30 % 3-D Taylor-Green vortices on 32^3..160^3, grids
    log-uniform), with its 100..2000 steps per request divided by SERVING_STEP_SCALE so that both
    precisions and both arms fit the benchmark's time; initial states on the host (padded,
    conservative).  Arrival times are drawn later, per arm, from the offered load."""
    import torch
    from paper_2406_19494_gb300.solver import Solver
    stream = workloads.serving_stream(count, seed=seed, n2d=(64, 1024), n3d=(32, 160), steps=(100, 2000))
    solvers = {}

    def solver_of(case):
        key = (case["name"], tuple(case["n"]))
        if key not in solvers:
            solvers[key] = Solver(case)
        return solvers[key]

    def centres_of(case):
        s = solver_of(case)
        out = [s.grid(a)[0] for a in range(3)]
        h = [3 if a < case["ndim"] else 0 for a in range(3)]
        return [out[a][h[a]:len(out[a]) - h[a]] for a in range(3)]

    reqs = []
    for r in stream:
        case, W = workloads.serving_case_and_prims(r, centres_of)
        pad = [(0, 0)] + [(3 if a < case["ndim"] else 0,) * 2 for a in (2, 1, 0)]
        Wd = torch.from_numpy(np.ascontiguousarray(np.pad(W, pad, mode="edge"))).cuda()
        U = solver_of(case).prim_to_cons(Wd).cpu().numpy()
        del Wd
        r = dict(r, nsteps=max(1, int(round(r["nsteps"] / SERVING_STEP_SCALE))))
        reqs.append((r, case, U, case["n"][0] * case["n"][1] * case["n"][2]))
    for s in solvers.values():
        s.close()
    torch.cuda.empty_cache()
    return reqs


def measure_serving(reqs, precision, rate_cu, load=1.5, seed=0):
    """Serving loop on the request stream `reqs` in one precision.  Arrivals: Poisson with the
    offered load `load` x rate_cu (cell-updates/s, the precision's measured one-solve rate), so
    requests keep arriving while others run.  Continuous batching (batched buckets, graphs per
    bucket, 150 GB budget) against one solve per launch: the same requests in arrival order, one at
    a time, each starting when it has arrived and the previous one has finished, with its solver
    created before the timed run (host -> device copy, fluid_step, device -> host copy).
    Latency = finish - arrival; throughput = interior cell updates / makespan."""
    import torch
    from paper_2406_19494_gb300.serve import Server
    from paper_2406_19494_gb300.solver import Solver
    total_cu = sum(r["nsteps"] * cells for r, _, _, cells in reqs)
    rate_hz = len(reqs) * load * rate_cu / total_cu
    u = workloads.uniform01(seed + 4242, len(reqs))
    arrivals = np.cumsum(-np.log1p(-u) / rate_hz)

    def pct(v, q):
        v = sorted(v)
        return v[min(len(v) - 1, int(round(q * (len(v) - 1))))]

    # continuous batching
    srv = Server(budget_bytes=150e9, max_active=128, chunk_steps=5, graphs=True, autotune=True, batch=True)
    t0 = time.perf_counter()
    tickets = []
    for (r, case, U0, _), ta in zip(reqs, arrivals):
        wait = ta - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        tickets.append(srv.submit(case, U0, r["nsteps"], precision=precision))
    lat, last = [], 0.0
    for t in tickets:
        res, _ = srv.poll(t, timeout_ms=900000)
        lat.append(res["finish_s"] - res["submit_s"])
        last = max(last, res["finish_s"])
    st = srv.stats()
    srv.close()
    makespan = last
    # one solve per launch, solvers (one per grid shape) created before the timed run
    solvers = {}
    for r, case, U0, _ in reqs:
        key = (case["name"], tuple(case["n"]))
        if key not in solvers:
            solvers[key] = Solver(case, precision=precision)
    lat1 = []
    t0 = time.perf_counter()
    for (r, case, U0, _), ta in zip(reqs, arrivals):
        now = time.perf_counter() - t0
        if now < ta:
            time.sleep(ta - now)
        s = solvers[(case["name"], tuple(case["n"]))]
        s.set_time(0.0)
        U = torch.from_numpy(U0).cuda()
        s.step(U, r["nsteps"])
        U.cpu()
        lat1.append(time.perf_counter() - t0 - ta)
    makespan1 = time.perf_counter() - t0
    for s in solvers.values():
        s.close()
    torch.cuda.empty_cache()
    n2 = sum(1 for r, *_ in reqs if r["kind"] != "tgv")
    return {"workload": "%d requests (%d 2-D vortex / Riemann on 64^2..1024^2, %d 3-D TGV on 32^3..160^3, "
                        "log-uniform grids), steps 100..2000 divided by %d, Poisson arrivals at %.2f/s "
                        "(offered load %.1f x the measured one-solve rate)"
                        % (len(reqs), n2, len(reqs) - n2, SERVING_STEP_SCALE, rate_hz, load),
            "precision": precision, "cell_updates": total_cu,
            "continuous_batching": {"p50_s": pct(lat, 0.5), "p99_s": pct(lat, 0.99), "makespan_s": makespan,
                                    "cell_updates_per_s": total_cu / makespan, "peak_hbm_bytes": st["peak_bytes"]},
            "one_solve_per_launch": {"p50_s": pct(lat1, 0.5), "p99_s": pct(lat1, 0.99), "makespan_s": makespan1,
                                     "cell_updates_per_s": total_cu / makespan1}}


def measure_e2(t_end=5.0):
    """Section 3.2's laminar boundary-layer validation (FP64): from the self-similar field to
    t_end (five flow-throughs reach the steady state), the outlet profile against the similarity
    solution over eta."""
    import torch
    from paper_2406_19494_gb300.solver import Solver
    c = workloads.e2_case()
    sim = workloads.e2_similarity(c)
    s = Solver(c)
    xc, _ = s.grid(0)
    yc, dy = s.grid(1)
    W = workloads.similarity_field(c, sim, xc[3:-3], yc[3:-3])
    Wp = np.pad(W, [(0, 0), (0, 0), (3, 3), (3, 3)], mode="edge")
    U = s.prim_to_cons(torch.from_numpy(np.ascontiguousarray(Wp)).cuda())
    s.set_inflow(0, 0, torch.from_numpy(workloads.e2_inflow(c, sim, yc)).cuda())
    t0 = time.perf_counter()
    t, steps = 0.0, 0
    while t < t_end:
        s.step(U, 4000, t_end)
        steps += 4000
        t, _ = s.time()
    s.check()
    wall = time.perf_counter() - t0
    Uh = U.cpu().numpy()
    rho = Uh[0, 0, 3:-3, -4]
    u = Uh[1, 0, 3:-3, -4] / rho
    v = Uh[2, 0, 3:-3, -4] / rho
    T = (c["gamma"] - 1.0) * (Uh[4, 0, 3:-3, -4] - 0.5 * rho * (u * u + v * v)) / (rho * c["R"])
    d = dy[3:-3]
    eta = (np.cumsum(rho * d) - 0.5 * rho * d) / math.sqrt(2.0 * xc[-4] * c["mu_ref"])
    fp = np.interp(eta, sim["eta"], sim["fp"], right=1.0)
    g = np.interp(eta, sim["eta"], sim["g"], right=1.0)
    sel = eta <= 8.0
    return {"case": "Ma 2.25 laminar flat-plate boundary layer, 300x200, adiabatic wall, similarity inlet, FP64",
            "t_end": t_end, "steps": steps, "wall_s": wall, "x_outlet": float(xc[-4]),
            "max_abs_err_u_over_ue": float(np.max(np.abs(u - fp)[sel])),
            "max_abs_err_T_over_Te": float(np.max(np.abs(T - g)[sel])),
            "rms_err_u": float(np.sqrt(np.mean((u - fp)[sel] ** 2))),
            "rms_err_T": float(np.sqrt(np.mean((T - g)[sel] ** 2))),
            "T_wall": float(T[0]), "T_wall_similarity": float(sim["g"][0]), "cells_eta_le_8": int(sel.sum())}


def measured_hbm_gbs():
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return 6800.0        # fallback copy bandwidth of an earlier GB300 measurement


def face_traffic(ncell):
    """DRAM bytes per face-kernel launch from the committed ncu summary, scaled by cells; None if the
    kernel sources changed since the counters were taken."""
    import hashlib
    try:
        info = json.load(open(os.path.join(ROOT, "profiles", "k_face_traffic.json")))
    except (OSError, ValueError):
        return None
    csrc = os.path.join(ROOT, "paper_2406_19494_gb300", "csrc")
    src = b"".join(open(os.path.join(csrc, f), "rb").read()
                   for f in ("kernels_fp64.cu", "fluid_internal.cuh", "flux_math.cuh"))
    if hashlib.sha256(src).hexdigest()[:16] != info.get("source_sha256_16"):
        return None
    per = sum(info["dram_bytes_per_launch"]) / len(info["dram_bytes_per_launch"])
    return per * ncell / info["cells"]


def mixed_step_roofline(ms_per_step, ncell):
    """Whole-step roofline of the mixed path from the committed ncu counters of one single-step
    call on TGV 128^3 (profiles/mixed_step_counters.json: every launch of the step with its FP64-pipe
    thread instructions, DRAM bytes and issued warp instructions), scaled per cell.  Three floors:
    the FP64 pipe (152 SMs x 2 lanes per clock), instruction issue (152 SMs x 4 schedulers x one
    warp instruction per clock), both at the maximum SM clock, and HBM at the measured copy
    bandwidth.  None when the kernel sources changed since the capture."""
    import hashlib
    try:
        info = json.load(open(os.path.join(ROOT, "profiles", "mixed_step_counters.json")))
    except (OSError, ValueError):
        return None
    csrc = os.path.join(ROOT, "paper_2406_19494_gb300", "csrc")
    src = b"".join(open(os.path.join(csrc, f), "rb").read()
                   for f in ("kernels_mixed.cu", "kernels_fp64.cu", "fluid_internal.cuh", "flux_math.cuh",
                             "fast_math.cuh"))
    if hashlib.sha256(src).hexdigest()[:16] != info.get("source_sha256_16"):
        return None
    scale = ncell / info["cells"]
    clk = 2.07e9
    tot = {k: sum(l[k] for l in info["launches"]) * scale
           for k in ("fp64_thread_inst", "dram_bytes", "warp_inst")}
    floors = {"fp64_pipe": tot["fp64_thread_inst"] / (152 * 2 * clk) * 1e3,
              "issue": tot["warp_inst"] / (152 * 4 * clk) * 1e3,
              "hbm": tot["dram_bytes"] / (measured_hbm_gbs() * 1e9) * 1e3}
    bound = max(floors, key=floors.get)
    return {"bound": bound, "floor_ms": floors[bound], "ms_per_step": ms_per_step,
            "frac": floors[bound] / ms_per_step, "floors_ms": floors,
            "per_cell_update": {"fp64_thread_inst": tot["fp64_thread_inst"] / ncell,
                                "dram_bytes": tot["dram_bytes"] / ncell,
                                "thread_inst": tot["warp_inst"] * 32 / ncell},
            "basis": "ncu counters of every launch of one single-step call (profiles/mixed_step_counters.json)"}


def ctypes_peak(s, kind):
    import ctypes
    import torch
    g = ctypes.c_double()
    st = s.lib.fluid_measure_peak(kind, ctypes.byref(g), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return g.value if st == 0 else None


# ------------------------------------------------------------------------------------------------
# CPU oracle on a bounded sample (the reference arm of this benchmark)
# ------------------------------------------------------------------------------------------------
SLAB = 8   # interior z-planes of the sample


def _oracle_sample(case_dict, k=0):
    """The oracle's view of z-slab k (SLAB interior planes with their halos, cut from the filled
    whole-domain state, wrapping around the periodic z axis), as an already filled block with the
    slab's own z extent."""
    from oracle import ns_fv as nf
    case = nf.Case(case_dict)
    grid = nf.Grid(case)
    cen = [grid.axes[a].xc[3:-3] for a in range(3)]
    W = np.pad(initial_prims(case_dict, cen), [(0, 0)] + [(3, 3)] * 3, mode="edge")
    U = nf.fill_halos(nf.prim_to_cons(W, case), case, grid)
    nz = case.n[2]
    z0 = (k * SLAB) % nz
    idx = [(z0 + j) % nz + 3 for j in range(-3, SLAB + 3)]
    lo, hi = case_dict["lo"][2], case_dict["hi"][2]
    dz = (hi - lo) / nz
    sub = dict(case_dict, n=(case.n[0], case.n[1], SLAB), lo=case_dict["lo"][:2] + (lo + z0 * dz,),
               hi=case_dict["hi"][:2] + (lo + (z0 + SLAB) * dz,))
    sc = nf.Case(sub)
    sg = nf.Grid(sc)
    Us = np.ascontiguousarray(U[:, idx])
    return nf, sc, sg, Us


def _oracle_slab_worker(k, case_dict, reps, warm, barrier, queue):
    """One process of the all-core oracle timing: its own slab, `warm` then `reps` steps' work
    (three right-hand sides each) after every process has built its slab; reports wall times."""
    nf, sc, sg, Us = _oracle_sample(case_dict, k)
    for _ in range(warm):
        nf.rhs_filled(Us, sc, sg)
    barrier.wait()
    t0 = time.time()
    for _ in range(reps):
        for _stage in range(3):
            nf.rhs_filled(Us, sc, sg)
    queue.put((t0, time.time(), sc.n[0] * sc.n[1] * sc.n[2]))


def oracle_all_cores(case_dict, reps, warm=1, cores=None):
    """The oracle on every host core: one process per core (started with spawn), each advancing
    its own z-slab; (cell-updates/s over the makespan, cores, cells per step, seconds per step)."""
    import multiprocessing as mp
    cores = cores or os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    barrier, queue = ctx.Barrier(cores), ctx.Queue()
    procs = [ctx.Process(target=_oracle_slab_worker, args=(k, case_dict, reps, warm, barrier, queue))
             for k in range(cores)]
    for p in procs:
        p.start()
    res = [queue.get() for _ in procs]
    for p in procs:
        p.join()
    span = max(r[1] for r in res) - min(r[0] for r in res)
    cells = sum(r[2] for r in res)
    return cells * reps / span, cores, cells, span / reps


def host_cpu():
    """The host's logical CPU count and model (from /proc/cpuinfo where it names one)."""
    model = None
    try:
        for line in open("/proc/cpuinfo"):
            key, _, val = line.partition(":")
            if key.strip() in ("model name", "Model", "Hardware") and val.strip():
                model = val.strip()
                break
    except OSError:
        pass
    import platform
    return {"host_cpus": os.cpu_count(), "host_cpu": model or platform.machine()}


def cpu_baseline(args, case_dict, samples=1):
    """The oracle on every host core (the reported value) and on one (beside it)."""
    nf, sc, sg, Us = _oracle_sample(case_dict)
    cells = sc.n[0] * sc.n[1] * sc.n[2]
    t0 = time.perf_counter()
    for _ in range(samples):
        for _stage in range(3):
            nf.rhs_filled(Us, sc, sg)
    dt = (time.perf_counter() - t0) / samples
    value, cores, cells_all, s_step = oracle_all_cores(case_dict, reps=samples)
    return dict({"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                 "sample": "3 oracle right-hand sides (one RK3 step's work) per process, one process per "
                           "host core, each on its own %dx%dx%d z-slab of the same state (%d cells in "
                           "all); numpy, spawned processes" % (sc.n[0], sc.n[1], SLAB, cells_all),
                 "single_core": {"value": cells / dt, "cores": 1,
                                 "sample": "the same work on one %dx%dx%d slab, one thread"
                                           % (sc.n[0], sc.n[1], sc.n[2])}}, **host_cpu())


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    case = WORKLOADS[args.workload]()
    value, cores, cells, s_step = oracle_all_cores(case, reps=args.steps, warm=args.warmup)
    total = s_step * args.steps
    sample = ("each step: 3 oracle right-hand sides (one RK3 step's work) per process, one process per "
              "host core, each on its own %dx%dx%d z-slab of the %s state (%d cells in all); numpy"
              % (case["n"][0], case["n"][1], SLAB, args.workload, cells))
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": describe(args.workload, case), "impl": "reference",
           "cpu_baseline": dict({"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
                                **host_cpu()),
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="fluid", choices=("fluid", "reference"))
    ap.add_argument("--workload", default="tgv128", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint/forward measurement")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving-loop measurement")
    ap.add_argument("--no-teno", action="store_true", help="skip the TENO6-A channel-scheme measurement")
    ap.add_argument("--no-mixed-errors", action="store_true",
                    help="skip the mixed-vs-FP64 errors on the stated workloads (TGV 1000 steps, walls)")
    ap.add_argument("--mixed-tiles", default="plain", choices=("plain", "bulk"),
                    help="the mixed path's y / z face tiles: plain loads (default) or rows staged by bulk copies")
    ap.add_argument("--e2", action="store_true",
                    help="also run the Ma 2.25 boundary-layer validation to steady state (about 3 minutes)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "fluid":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_fluid(args)


if __name__ == "__main__":
    main()
