#!/usr/bin/env python3
"""Throughput of the multipatch scalar-wave hot path on GB300.

Metric: grid-point RK4 stage-updates/s = (live points summed over patches) x 4
substages x steps / device time, ghost fills and cover flags included.
Workload: global 256^3 on [-1,1]^3 plus four orbiting local 128^3 patches,
eight Gaussian pulses, 6-point Lagrange, FP64 (paper_2002_00088_gb300.workloads
.orbiting_gauss).  The state (~1.8 GB) is far larger than L2, so no flush is
needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--precision 64|32]

--motion spinning runs the rotating-patch workload instead
(workloads.spinning_gauss: global 256^3 plus four local 96^3 cubes at 2x
spinning in place about seeded axes, the rotating local patch of Sec. 3.2).

--precision 32 runs the binary32 precision workload instead
(workloads.plane_gauss: periodic global 512^3 plus a static local 256^3 at 2x,
plane wave k = (2,3,5) pi plus a Gaussian pulse).  Its line adds "accuracy":
the binary32 error against the closed form after the run, and the FP64 path's
time and error on the same workload and steps.

--surrogate runs the learned-surrogate configuration instead
(workloads.surrogate_layout: periodic global 128^3, two orbiting local 64^3
patches at 2x): the network is trained on 2,000 trajectories of the method,
then 400 steps of the hybrid (one network call advances the global four steps,
the local patches stay on the method) are timed against the plain method.

With --gpus N > 1 (under torch.distributed.run) every rank advances an
independent replica on its own GPU ("replicas only": the method needs no
exchange between instances); value is the sum over ranks.  --impl reference
times the plain FP64 CPU oracle on the host cores on a bounded sample of the
same workload (the paper publishes no timings to compare with).
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "grid-point RK4 stage-updates/s"
UNIT = "stage-updates/s"
FALLBACK_HBM_GBS = 6800.0
# algorithmic bytes of one live point in one fused RHS+stage launch, averaged
# over the four substages: S1 48 B, S2 80 B, S3 80 B, S4 48 B (FP64)
BYTES_PER_POINT_STAGE = 64  # (32 B in binary32)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scale", type=int, default=1, help="divide the workload resolution (testing only)")
    ap.add_argument("--e2e-steps", type=int, default=None,
                    help="end-to-end leg: timed steps (default: --steps; the first input copy and the last "
                         "result copy are not overlapped, so short legs understate the rate)")
    ap.add_argument("--cpu-sample-scale", type=int, default=1,
                    help="cpu_baseline: the workload at this resolution divisor")
    ap.add_argument("--cpu-sample-steps", type=int, default=10, help="cpu_baseline: timed oracle steps")
    ap.add_argument("--ref-sample-scale", type=int, default=2,
                    help="--impl reference: resolution divisor of the oracle sample taken per step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch", type=int, default=0,
                    help="time N independent instances of uneven sizes (workloads.batch_instances) advanced with "
                         "batched launches, beside the same instances stepped one after the other")
    ap.add_argument("--max-global", type=int, default=192, help="--batch: largest global patch edge")
    ap.add_argument("--static", action="store_true", help="--batch: local patches do not move (graph replay)")
    ap.add_argument("--shells", action="store_true",
                    help="--batch: every second instance holds a spherical shell instead of local cubes")
    ap.add_argument("--motion", default="orbiting", choices=["orbiting", "spinning"],
                    help="orbiting: translating local patches on circular orbits (default); spinning: the "
                         "rotating-patch workload")
    ap.add_argument("--surrogate", action="store_true",
                    help="the learned surrogate: train it on the method's trajectories, then time the hybrid "
                         "(surrogate global, local patches on the method) against the plain method")
    ap.add_argument("--trajectories", type=int, default=2000, help="--surrogate: training trajectories")
    ap.add_argument("--network", action="store_true",
                    help="the surrogate network's forward alone (four 3x3x3 conv layers at 128^3, seeded random "
                         "BF16 input), per layer, against the measured bf16 peak")
    ap.add_argument("--tol", type=float, default=1e-4, help="--surrogate: residual tolerance of a call")
    ap.add_argument("--precision", type=int, default=64, choices=[64, 32],
                    help="64: the FP64 workload (default); 32: the binary32 precision workload, with its error "
                         "against the closed form and the FP64 path on the same workload")
    args = ap.parse_args()
    if args.e2e_steps is None:
        args.e2e_steps = args.steps
    return args


def dist_info():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def whole_job(seconds, units, world, device="cpu"):
    """Whole-job throughput of independent replicas: the units of every rank
    divided by the slowest rank's time (a max over ranks; no data-path
    collective).  Returns (max seconds, summed units, units per second)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(seconds), float(units)], dtype=torch.float64, device=device)
        mx = t.clone()
        dist.all_reduce(mx, op=dist.ReduceOp.MAX)
        sm = t.clone()
        dist.all_reduce(sm, op=dist.ReduceOp.SUM)
        seconds, units = float(mx[0]), float(sm[1])
    return seconds, units, units / seconds


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            with open(path) as f:
                d = json.load(f)
            for k in ("hbm_gbs", "hbm_GBs", "hbm"):
                if k in d:
                    return float(d[k]), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.out = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.flush()
        rows = []
        with open(self.out.name) as f:
            for ln in f:
                parts = [p.strip() for p in ln.split(",")]
                if len(parts) == 7:
                    rows.append(parts)
        os.unlink(self.out.name)
        if not rows:
            return None
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[3 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": float(rows[0][1]) if rows[0][1].replace(".", "").isdigit() else None,
                "reasons": reasons, "samples": len(rows)}


RHS_SOURCES = ("mpw_rhs.cu", "mpw_fixed.cuh", "mpw_rhs_args.cuh", "mpw_tma.cuh")
RHS32_SOURCES = ("mpw_rhs32.cu", "mpw_rhs_args.cuh", "mpw_tma.cuh")


def kernel_source_hash(f32=False):
    """Hash of the sources that define the fused RHS + stage kernel."""
    h = hashlib.sha256()
    for name in (RHS32_SOURCES if f32 else RHS_SOURCES):
        with open(os.path.join(ROOT, "paper_2002_00088_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(f32=False, workload=None):
    """DRAM bytes per launch of the RHS kernel from the committed ncu summary,
    if it was taken on the current kernel sources and on this workload."""
    path = os.path.join(ROOT, "profiles", "rhs32_stage_traffic.json" if f32 else "rhs_stage_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    if d.get("kernel_source_hash") != kernel_source_hash(f32):
        return None
    if workload is not None and d.get("workload") != workload:
        return None
    return d.get("traffic_bytes_per_launch")


def precision_report(args, w, sim, mpw, stream, device):
    """Binary32 run: its error against the closed form at the current time and
    the FP64 path on the same workload and number of steps (time and error).
    The closed form is evaluated by the library's own FP64 kernel in a third
    context; errors are max |difference| over the live cells of all patches
    relative to the largest |exact value| of the field."""
    import torch
    steps = args.warmup + args.steps
    t = sim.time

    def make(precision):
        s = mpw.Multipatch(w.interp_points, w.ko_eps, device=device, stream=stream, precision=precision)
        for p in w.patches:
            s.create_patch(p.kind, p.n, p.lo, p.hi, p.outer_bc, p.motion, p.motion_params, p.topology)
        s.set_analytic(w.analytic_kind, w.analytic_params, w.analytic_count)
        return s

    def fields(s):
        out = []
        for q, p in enumerate(w.patches):
            a = torch.empty((p.n[2], p.n[1], p.n[0]), dtype=torch.float64, device=device)
            b = torch.empty_like(a)
            s.get_fields(q, out=(a, b))
            out.append((a, b))
        return out

    exact_sim = make(64)
    exact_sim.fill_analytic(t)
    exact = fields(exact_sim)
    del exact_sim

    def errors(run):
        res = []
        for f in range(2):
            scale = max(float(x[f].abs().max()) for x in exact)
            e = 0.0
            for a, b in zip(run, exact):
                d = (a[f] - b[f]).abs()
                e = max(e, float(torch.nan_to_num(d, nan=0.0).max()))
            res.append(e / scale)
        return res

    e32 = errors(fields(sim))
    s64 = make(64)
    s64.fill_analytic(0.0)
    s64.step(w.dt, args.warmup)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    s64.step(w.dt, args.steps)
    b.record(stream)
    torch.cuda.synchronize()
    ms64 = a.elapsed_time(b)
    e64 = errors(fields(s64))
    live = s64.live_points()
    del s64
    torch.cuda.empty_cache()
    return {"time": t, "steps": steps,
            "f32_error_vs_closed_form": {"psi": e32[0], "pi": e32[1]},
            "f64_error_vs_closed_form": {"psi": e64[0], "pi": e64[1]},
            "f64_value": live * 4 * args.steps / (ms64 * 1e-3), "f64_ms_per_step": ms64 / args.steps}


def fp64_workload(args):
    from paper_2002_00088_gb300 import workloads as wl
    return wl.spinning_gauss if args.motion == "spinning" else wl.orbiting_gauss


def cpu_baseline(args, threads):
    """The oracle as it stands, on the host cores, on a bounded sample."""
    from oracle import pyoracle as po
    from paper_2002_00088_gb300 import workloads as wl
    # the precision workload is 6x larger: its oracle sample runs at half resolution
    make = wl.plane_gauss if args.precision == 32 else fp64_workload(args)
    w = make(scale=max(args.scale, args.cpu_sample_scale, 2 if args.precision == 32 else 1))
    o = po.Oracle(w.interp_points, w.ko_eps, 4, threads=threads)
    for p in w.patches:
        o.add_patch(p.kind, p.n, p.lo, p.hi, p.outer_bc, p.motion, p.motion_params, p.topology)
    o.set_analytic(w.analytic_kind, w.analytic_params, w.analytic_count)
    o.fill_analytic(0.0)
    o.step(w.dt, 1)  # first step: flags from scratch, allocation warm-up
    live = o.live_points()
    t0 = time.perf_counter()
    o.step(w.dt, args.cpu_sample_steps)
    el = time.perf_counter() - t0
    return {"value": live * 4 * args.cpu_sample_steps / el, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{args.cpu_sample_steps} step(s) of {w.name} after one untimed step, {live} live points, "
                      f"{el:.2f} s, binary64"}


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return 0
    from oracle import pyoracle as po
    from paper_2002_00088_gb300 import workloads as wl
    threads = os.cpu_count() or 1
    full = fp64_workload(args)(scale=args.scale)
    w = fp64_workload(args)(scale=max(args.scale, args.ref_sample_scale))
    o = po.Oracle(w.interp_points, w.ko_eps, 4, threads=threads)
    for p in w.patches:
        o.add_patch(p.kind, p.n, p.lo, p.hi, p.outer_bc, p.motion, p.motion_params, p.topology)
    o.set_analytic(w.analytic_kind, w.analytic_params, w.analytic_count)
    o.fill_analytic(0.0)
    o.step(w.dt, args.warmup)
    live = o.live_points()
    t0 = time.perf_counter()
    o.step(w.dt, args.steps)
    el = time.perf_counter() - t0
    value = live * 4 * args.steps / el
    sample = (f"each step: one oracle step of {w.name} (the workload at 1/{max(args.scale, args.ref_sample_scale)}"
              f" resolution per axis), {live} live points")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded closed-form Gaussian pulses)",
            "config": {"workload": full.name, "sample": w.name},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch

    rank, world, local = dist_info()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    from paper_2002_00088_gb300.build import build_library
    build_library()
    from paper_2002_00088_gb300 import mpw
    from paper_2002_00088_gb300 import workloads as wl

    f32 = args.precision == 32
    w = wl.plane_gauss(scale=args.scale) if f32 else fp64_workload(args)(scale=args.scale)
    stream = torch.cuda.current_stream(local)
    sim = mpw.Multipatch(w.interp_points, w.ko_eps, device=local, stream=stream, precision=args.precision)
    for p in w.patches:
        sim.create_patch(p.kind, p.n, p.lo, p.hi, p.outer_bc, p.motion, p.motion_params, p.topology)
    sim.set_analytic(w.analytic_kind, w.analytic_params, w.analytic_count)
    sim.fill_analytic(0.0)  # inputs generated in HBM
    sim.step(w.dt, args.warmup)
    live = sim.live_points()

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    # ---- device-timed region: exactly K steps, inputs resident in HBM
    sampler = ClockSampler(local)
    sampler.start()
    sim.profile(True)
    sim.profile_read()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    start.record(stream)
    sim.step(w.dt, args.steps)
    end.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = start.elapsed_time(end)
    prof = sim.profile_read()
    sim.profile(False)
    clocks = sampler.stop()
    sec, _, value = whole_job(ms * 1e-3, live * 4 * args.steps, world, "cuda")
    ms = sec * 1e3
    accuracy = precision_report(args, w, sim, mpw, stream, local) if f32 else None

    # ---- end-to-end through the C ABI with host buffers: every step copies
    # its input in from pinned host memory and its result back out, with the
    # asynchronous calls so that the copies (copy engines, two streams of the
    # library's) overlap the neighbouring steps' compute
    shapes = [(p.n[2], p.n[1], p.n[0]) for p in w.patches]
    host = [(torch.empty(s, dtype=torch.float64, pin_memory=True).numpy(),
             torch.empty(s, dtype=torch.float64, pin_memory=True).numpy()) for s in shapes]
    for q in range(len(shapes)):
        sim.get_fields(q)  # warm the staging path
    hq = [sim.get_fields(q) for q in range(len(shapes))]
    for q in range(len(shapes)):
        host[q][0][...] = np.nan_to_num(hq[q][0])
        host[q][1][...] = np.nan_to_num(hq[q][1])
    bytes_in = sum(2 * 8 * int(np.prod(s)) for s in shapes)
    outs = [[(torch.empty(s, dtype=torch.float64, pin_memory=True).numpy(),
              torch.empty(s, dtype=torch.float64, pin_memory=True).numpy()) for s in shapes] for _ in range(2)]
    for q in range(len(shapes)):  # warm the staging buffers
        sim.set_fields_async(q, host[q][0], host[q][1])
        sim.get_fields_async(q, outs[0][q][0], outs[0][q][1])
    sim.sync()
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(args.e2e_steps):
        for q in range(len(shapes)):
            sim.set_fields_async(q, host[q][0], host[q][1])
        sim.step_async(w.dt, 1)
        for q in range(len(shapes)):
            sim.get_fields_async(q, outs[k % 2][q][0], outs[k % 2][q][1])
    sim.sync()
    torch.cuda.synchronize()
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e_s, _, e2e_value = whole_job(e2e_s, live * 4 * args.e2e_steps, world, "cuda")

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0

    rhs_ms, rhs_n = prof["rhs"]
    fill_ms, fill_n = prof["fill"]
    flags_ms, flags_n = prof["flags"]
    rhs_avg_ms = rhs_ms / max(rhs_n, 1)
    peak, peak_kind = measured_peaks()
    bytes_pt = BYTES_PER_POINT_STAGE // 2 if f32 else BYTES_PER_POINT_STAGE
    achieved = live * bytes_pt / (rhs_avg_ms * 1e-3) / 1e9
    traffic = recorded_traffic(f32, w.name)
    esize = 4 if f32 else 8
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if f32 else "f64",
        "data": "synthetic (seeded closed-form plane wave + Gaussian pulse)" if f32 else
                "synthetic (seeded closed-form Gaussian pulses)",
        "config": {"workload": w.name, "live_points": live, "interp_points": w.interp_points,
                   "dt": w.dt, "parallelism": "replicas" if world > 1 else "single",
                   "l2": "state of %.2f GB, larger than L2; no flush" % (
                       sum(8 * esize * (p.n[0] + 6) * (p.n[1] + 6) * (p.n[2] + 6) for p in w.patches) / 1e9)},
        "roofline": {"bound": "hbm", "kernel": "rhs_stage (fused RHS + RK4 stage%s)" % (", binary32" if f32 else ""),
                     "achieved": achieved,
                     "peak": peak, "peak_source": f"{peak_kind} HBM GB/s", "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "avg_launch_ms": rhs_avg_ms,
                     "algorithmic_bytes_per_launch": live * bytes_pt},
        "kernel_time_share": {"rhs_stage": rhs_ms / ms, "ghost_fill": fill_ms / ms, "cover_flags": flags_ms / ms},
        "gpu_launches": int(rhs_n + fill_n + flags_n),
        "clocks": clocks,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": bytes_in, "d2h_bytes_per_step": bytes_in,
                "steps": args.e2e_steps},
    }
    if accuracy is not None:
        line["accuracy"] = accuracy
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args, os.cpu_count() or 1)
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_batch(args):
    """Batched instances: value = live points of all instances x 4 x steps /
    device time of the batched steps; "sequential" times the same instances
    stepped one after the other with mpw_step."""
    import torch
    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    from paper_2002_00088_gb300.build import build_library
    build_library()
    from paper_2002_00088_gb300 import mpw
    from paper_2002_00088_gb300 import workloads as wl
    ws = wl.batch_instances(count=args.batch, steps=args.warmup + args.steps + 4, max_global=args.max_global,
                            moving=not args.static, shells=args.shells)
    stream = torch.cuda.current_stream(local)

    def make():
        sims = []
        for w in ws:
            g = mpw.Multipatch(w.interp_points, w.ko_eps, device=local, stream=stream, precision=args.precision)
            for p in w.patches:
                g.create_patch(p.kind, p.n, p.lo, p.hi, p.outer_bc, p.motion, p.motion_params, p.topology)
            g.set_analytic(w.analytic_kind, w.analytic_params, w.analytic_count)
            g.fill_analytic(0.0)
            sims.append(g)
        return sims

    dts = [w.dt for w in ws]
    sims = make()
    live = sum(g.live_points() for g in sims)
    b = mpw.Batch(sims)
    b.step(dts, args.warmup + 4)  # warm-up, including the four chunk-depth trials
    zc, zc_ms, n0, g0 = b.tuning()
    for g in sims:
        g.profile_read()  # clears the per-instance launch counters
    sampler = ClockSampler(local)
    sampler.start()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    start.record(stream)
    b.step(dts, args.steps)
    end.record(stream)
    torch.cuda.synchronize()
    ms = start.elapsed_time(end)
    clocks = sampler.stop()
    graph_steps = b.tuning()[3] - g0
    # batched launches (flags included when batched) plus the instances' own
    # flags launches when they are not
    launches = b.tuning()[2] - n0 + sum(g.profile_read()["flags"][1] for g in sims)
    del b, sims
    torch.cuda.empty_cache()
    # the same instances, one mpw_step after the other
    seq = make()
    for g, dt in zip(seq, dts):
        g.step(dt, args.warmup)
    torch.cuda.synchronize()
    start.record(stream)
    for _ in range(args.steps):
        for g, dt in zip(seq, dts):
            g.step(dt, 1)
    end.record(stream)
    torch.cuda.synchronize()
    ms_seq = start.elapsed_time(end)
    line = {
        "metric": METRIC, "value": live * 4 * args.steps / (ms * 1e-3), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision == 32 else "f64",
        "data": "synthetic (seeded closed-form Gaussian pulses)",
        "config": {"workload": f"batch of {len(ws)} instances (globals 64^3-{args.max_global}^3, 1-8 "
                               f"{'static' if args.static else 'moving'} locals each"
                               f"{'; every second instance one ' + ('static' if args.static else 'spinning') + ' spherical shell r in [0.1, 0.5]' if args.shells else ''})",
                   "instances": len(ws), "live_points": live, "parallelism": "single",
                   "rhs_chunk_depth": zc, "tuning_rhs_ms": zc_ms, "graph_replayed_steps": graph_steps},
        "sequential": {"value": live * 4 * args.steps / (ms_seq * 1e-3), "ms_per_step": ms_seq / args.steps},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    return 0


SUR_SIGMA = 1e-4


def surrogate_cpu_baseline(w, params, threads):
    """The oracle's surrogate call (features, network, update; numpy FP64 with
    the device's bfloat16 roundings) on a bounded sample volume."""
    import numpy as np
    from oracle import surrogate as so
    n = (32, 16, 16)
    h = 2.0 / w.patches[0].n[0]
    r = np.random.default_rng(7)
    psi = r.standard_normal((1, n[2], n[1], n[0]))
    pi = r.standard_normal((1, n[2], n[1], n[0])) * 20
    t0 = time.perf_counter()
    x, s = so.features(psi, pi, w.dt, h)
    _, y = so.net_forward(x, params)
    so.apply(psi, pi, s, y, w.dt, h, SUR_SIGMA)
    el = time.perf_counter() - t0
    pts = n[0] * n[1] * n[2]
    return {"value": pts * 16 / el, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"one surrogate call (4 steps x 4 substages) on a periodic {n[0]}x{n[1]}x{n[2]} volume, "
                      f"{el:.2f} s, numpy FP64 with bfloat16 roundings"}


def run_surrogate(args):
    """Learned surrogate: train on the method's trajectories (periodic global
    128^3), then the hybrid (one call advances the global four steps, two
    moving local 64^3 patches on the method) against the plain method on the
    same layout, and the plain global-only run the surrogate learned from."""
    import numpy as np
    import torch
    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    from paper_2002_00088_gb300.build import build_library
    build_library()
    from paper_2002_00088_gb300 import mpw
    from paper_2002_00088_gb300 import surrogate as S
    from paper_2002_00088_gb300 import workloads as wl
    stream = torch.cuda.current_stream(local)
    steps = max(4, args.steps // 4 * 4)
    calls = steps // 4
    w = wl.surrogate_layout(scale=args.scale, steps=steps)
    n = w.patches[0].n[0]
    h = 2.0 / n
    ev = lambda: torch.cuda.Event(enable_timing=True)
    # training, every step on the device (trajectories, features, targets, forward, backward, Adam)
    src = S.Trajectories(n, w.dt, device=local)
    sur = S.Surrogate(w.dt, h, SUR_SIGMA, device=local, stream=stream, params=wl.surrogate_init(1))
    t0 = time.perf_counter()
    losses = S.train(sur, src, trajectories=args.trajectories, batch=2, lr=2e-3, lr_end=1e-4)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    # what the network gains: one call against the method's four steps on held-out trajectories
    off = S.Surrogate(w.dt, h, SUR_SIGMA, device=local, stream=stream, params=np.zeros(sur.count, np.float32))
    gain = {"trained": 0.0, "network_off": 0.0}
    for k in range(8):
        u0 = [torch.empty((n, n, n), dtype=torch.float64, device="cuda") for _ in range(2)]
        u1 = [torch.empty((n, n, n), dtype=torch.float64, device="cuda") for _ in range(2)]
        src.pair(80000 + k, u0, u1)
        sc = max(float(u1[0].abs().max()), 4 * w.dt * float(u1[1].abs().max()))
        for name, s_ in (("trained", sur), ("network_off", off)):
            p1, q1 = s_.predict(u0[0], u0[1])
            e = max(float((p1 - u1[0]).abs().max()), 4 * w.dt * float((q1 - u1[1]).abs().max())) / sc
            gain[name] = max(gain[name], e)

    def make(npatch):
        g = mpw.Multipatch(w.interp_points, w.ko_eps, device=local, stream=stream)
        for p in w.patches[:npatch]:
            g.create_patch(p.kind, p.n, p.lo, p.hi, p.outer_bc, p.motion, p.motion_params, p.topology)
        g.set_analytic(w.analytic_kind, w.analytic_params, w.analytic_count)
        g.fill_analytic(0.0)
        return g

    # warm-up on a throwaway copy, then the timed hybrid run
    warm = make(3)
    S.step_hybrid(warm, sur, w.dt, max(args.warmup, 1), args.tol)
    del warm
    hyb = make(3)
    live = hyb.live_points()
    sampler = ClockSampler(local)
    sampler.start()
    a, b = ev(), ev()
    torch.cuda.synchronize()
    a.record(stream)
    accepted, max_res = S.step_hybrid(hyb, sur, w.dt, calls, args.tol)
    b.record(stream)
    torch.cuda.synchronize()
    ms_h = a.elapsed_time(b)
    clocks = sampler.stop()
    plain = make(3)
    plain.step(w.dt, args.warmup)
    plain = make(3)
    torch.cuda.synchronize()
    a.record(stream)
    plain.step(w.dt, steps)
    b.record(stream)
    torch.cuda.synchronize()
    ms_p = a.elapsed_time(b)
    solo = make(1)
    solo.step(w.dt, steps)

    def errors(x, y, patches):
        out = []
        for f in range(2):
            got = [x.get_fields(q)[f] for q in patches]
            want = [y.get_fields(q)[f] for q in patches]
            scale = max(np.nanmax(np.abs(v)) for v in want)
            out.append(float(max(np.nanmax(np.abs(g - v)) for g, v in zip(got, want)) / scale))
        return {"psi": out[0], "pi": out[1]}

    err_mp = errors(hyb, plain, range(3))
    err_solo = errors(hyb, solo, [0])
    # each run against the closed form (free space) at 200 steps, before the
    # pulses reach the faces of the periodic global and wrap around (after
    # that the closed form no longer describes the periodic problem): the
    # global on the cells the plain multipatch run keeps live, the local
    # patches whole, relative to the largest closed-form value on the global
    early = min(steps, 200) // 4
    hyb, plain, solo = make(3), make(3), make(1)
    S.step_hybrid(hyb, sur, w.dt, early, args.tol)
    plain.step(w.dt, 4 * early)
    solo.step(w.dt, 4 * early)
    exact3, exact1 = make(3), make(1)
    exact3.fill_analytic(plain.time)
    exact1.fill_analytic(plain.time)
    live_cells = (plain.get_flags() & 3) == 0

    def vs_exact(run, ex, patches):
        out = {}
        for f, nm in enumerate(("psi", "pi")):
            scale = np.nanmax(np.abs(ex.get_fields(0)[f]))
            e = {}
            for q in patches:
                d = np.abs(run.get_fields(q)[f] - ex.get_fields(q)[f])
                e["global" if q == 0 else f"local{q}"] = float(np.nanmax(d[live_cells] if q == 0 else d) / scale)
            out[nm] = e
        return out

    err_exact = {"steps": 4 * early, "hybrid": vs_exact(hyb, exact3, range(3)),
                 "plain_multipatch": vs_exact(plain, exact3, range(3)),
                 "plain_global_only": vs_exact(solo, exact1, [0])}
    # the network's forward throughput (tensor-core bound), CUDA events
    x = torch.zeros((1, n, n, n, 8), dtype=torch.bfloat16, device="cuda")
    for _ in range(3):
        sur.forward(x)
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(10):
        sur.forward(x)
    b.record(stream)
    torch.cuda.synchronize()
    fwd_ms = a.elapsed_time(b) / 10
    flops = n ** 3 * 2 * 27 * (7 * 32 + 32 * 32 * 2 + 32 * 2)
    peak = None
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peak = float(json.load(f)["bf16_tflops"])
        peak_src = "measured bf16 TFLOP/s (burst)"
    except Exception:
        peak, peak_src = 1900.0, "fallback bf16 TFLOP/s"
    achieved = flops / (fwd_ms * 1e-3) / 1e12
    line = {
        "metric": METRIC, "value": live * 4 * steps / (ms_h * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": steps,
        "warmup": args.warmup, "ms_per_step": ms_h / steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64+bf16", "data": "synthetic (seeded Gaussian pulses; trained on the method's "
                                                           "own trajectories)",
        "config": {"workload": w.name, "live_points": live, "calls": calls, "tol": args.tol, "sigma": SUR_SIGMA,
                   "trajectories": args.trajectories, "parallelism": "single",
                   "l2": "state larger than L2 (global 128^3 x 8 dense FP64 arrays per call); no flush"},
        "plain": {"value": live * 4 * steps / (ms_p * 1e-3), "ms_per_step": ms_p / steps},
        "speedup_vs_plain": ms_p / ms_h,
        "accepted_calls": accepted, "max_residual": max_res,
        "error_vs_plain_multipatch": err_mp, "error_vs_plain_global_only": err_solo,
        "error_vs_closed_form": err_exact,
        "one_call_error": gain, "training": {"seconds": train_s, "first_loss": float(np.mean(losses[:20])),
                                             "last_loss": float(np.mean(losses[-20:]))},
        "roofline": {"bound": "tensor",
                     "kernel": ("k_conv3_tc, k_conv3_tc_yx (network forward, tcgen05 BF16 with FP32 TMEM "
                                "accumulators)" if n == 128
                                else "k_conv3 (network forward, mma.sync BF16/FP32)"),
                     "achieved": achieved, "peak": peak, "peak_source": peak_src, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None, "avg_launch_ms": fwd_ms / 4},
        # per accepted call: cover flags and revival 2, the Local-to-Global fill
        # 1, the dead-cell fill 1, the pack 1, the global's exponent scan 1,
        # features 7 (maximum, scale, three Laplacians, per-sample products,
        # features), network 4, update 1, check 2 (Laplacian, residual), per
        # step the Hermite stage states 1 and 4 x (fill + RHS), cover flags on
        # steps 2-4 (3), the unpack 1: 60; the first call has no revival and
        # scans the exponents of all three patches (+1)
        "gpu_launches": calls * 60 + 1,
        "clocks": clocks,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = surrogate_cpu_baseline(w, wl.surrogate_init(1), os.cpu_count() or 1)
    print(json.dumps(line), flush=True)
    return 0


def run_network(args):
    """The surrogate network's forward (8 -> 32 -> 32 -> 32 -> 8 channels,
    3x3x3 taps, periodic) on one 128^3 volume: per-layer CUDA-event times
    over --steps forwards after --warmup ones."""
    import torch
    from paper_2002_00088_gb300.build import build_library
    build_library()
    from paper_2002_00088_gb300 import surrogate as S
    n = 128
    torch.cuda.set_device(0)
    g = torch.Generator(device="cuda").manual_seed(5)
    x = torch.randn((1, n, n, n, 8), device="cuda", generator=g).to(torch.bfloat16)
    layers = [(8, 32), (32, 32), (32, 32), (32, 8)]
    acts = [x] + [torch.empty((1, n, n, n, co), dtype=torch.bfloat16, device="cuda") for _, co in layers[:-1]]
    ws = [(torch.randn((co, 27, ci), device="cuda", generator=g) / (27 * ci) ** 0.5).to(torch.bfloat16)
          for ci, co in layers]
    bs = [torch.randn(co, device="cuda", generator=g) * 0.1 for _, co in layers]
    ev = lambda: torch.cuda.Event(enable_timing=True)
    per = [0.0] * len(layers)

    def forward(record):
        for l, (ci, co) in enumerate(layers):
            if record:
                a, b = ev(), ev()
                a.record()
            last = l == len(layers) - 1
            y, _ = S.conv3_forward(acts[l], ws[l], bs[l], relu=not last)
            if not last:
                acts[l + 1] = y
            if record:
                b.record()
                events.append((l, a, b))

    events = []
    for _ in range(max(args.warmup, 1)):
        forward(False)
    torch.cuda.synchronize()
    a, b = ev(), ev()
    a.record()
    for _ in range(args.steps):
        forward(True)
    b.record()
    torch.cuda.synchronize()
    for l, e0, e1 in events:
        per[l] += e0.elapsed_time(e1) / args.steps
    ms = a.elapsed_time(b) / args.steps
    flops = [2 * 27 * ci * co * n ** 3 for ci, co in layers]
    pk = None
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk, src = float(json.load(f)["bf16_tflops"]), "measured bf16 TFLOP/s (burst)"
    except Exception:
        pk, src = 1900.0, "fallback bf16 TFLOP/s"
    tf = sum(flops) / (ms * 1e-3) / 1e12
    line = {"metric": "network forward TFLOP/s", "value": tf, "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "dtype": "bf16 in, f32 accumulate",
            "data": "synthetic (seeded normal input and weights)",
            "config": {"workload": "surrogate network 8-32-32-32-8, 3x3x3, periodic 128^3, batch 1",
                       "kernel": "k_conv3_tc (8 -> 32, 32 -> 32), k_conv3_tc_yx (32 -> 8)"},
            "layers": [{"cin": ci, "cout": co, "ms": per[l], "tflops": flops[l] / (per[l] * 1e-3) / 1e12}
                       for l, (ci, co) in enumerate(layers)],
            "roofline": {"bound": "tensor", "achieved": tf, "peak": pk, "peak_source": src, "unit": "TFLOP/s",
                         "frac": tf / pk}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.network:
        return run_network(args)
    if args.batch:
        return run_batch(args)
    if args.surrogate:
        return run_surrogate(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
