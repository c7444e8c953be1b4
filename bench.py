"""Benchmark of the kinetic DG step on GB300.

A step is one application of S(dt) = R_omega o T_CN(dt) to the whole state:
the K = 3 subdomain-iterated downwind DG transport of every population plus
the fused over-relaxation, i.e. one launch of the fused step kernel.

Workload (default): 2D compressible Euler, isentropic vortex on [0,10]^2,
256 x 256 cells, DG degree 2 (3 x 3 Gauss-Lobatto nodes), D2Q4 (16
populations per node), dt = 5 x the explicit DG limit, 8 x 8 subdomains,
FP32 kinetic state: 9,437,184 kinetic DOF (37.7 MB).  The state is smaller
than L2, so L2 is flushed before every timed step -- a 256 MB write, then a
256 MB read so that the written lines are back in HBM -- and only the step
kernel itself is inside the CUDA-event window.

Metric: kinetic-DOF updates per second (one kinetic DOF = one nodal value of
one population advanced by one full step).

`--impl reference` times the FP64 CPU oracle (the test reference of this
repository) on the same workload and metric on the host cores.
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

METRIC = "kinetic-DOF updates/s"
UNIT = "DOF-updates/s"
ALGO_BYTES_PER_DOF = {"f32": 8, "f64": 16}   # read f^n once + write f^{n+1} once
# FP64 on GB300 runs at a small fraction of the FP32 rate: the FP64 path is
# bound by FP64 arithmetic.  Peak from the unit counts: 152 SMs x 2 FP64 FMA
# per clock (4 flop) x 2.07 GHz maximum SM clock.
FP64_PEAK_TFLOPS = 152 * 4 * 2.07e9 / 1e12


def flops_per_dof(dim, degree, m, nvel, maxwell=False):
    """FP64 floating-point operations of one step per kinetic DOF, counted from
    the axis-velocity scheme as the kernels evaluate it (an FMA is 2 flop):
    sweep per cell line of NP nodes: NP rows of (P - I) u (2 NP) plus g t (2),
    the outflow trace (1) and f^{n+1} = u + 2 delta (2 per node); block
    summary per cell line: outflow row (2 NP) and gain (2); relaxation per
    node: the moment sums, Euler pressure and fluxes, and two Maxwellian
    updates per (axis, variable); for Maxwell the conductivity factor on E and
    both Maxwellians (before and after it) per (axis, variable); the
    look-back is below 1 flop per DOF."""
    NP = degree + 1
    sweep = (NP * (2 * NP + 2) + 1 + 2 * NP) / NP
    summary = (2 * NP + 2) / NP
    npop = nvel * m
    if maxwell:
        relax = m * (nvel - 1) + 3 + dim * m * 14
    elif m == 1:
        relax = (nvel - 1) + dim * (1 + 2 + 2 * 4)
    else:
        relax = m * (nvel - 1) + (1 + 2 * dim + 4) + dim * (1 + 2 * dim + 3 + m * 8)
    return sweep + summary + relax / npop + 1.0
# DRAM bytes (read + write) of one step launch from an ncu capture of the same
# kernel and workload (profiles/step_kernel_fixed_vortex2d_256x256_p2.md,
# profiles/step_kernel_fixed_vortex2d_512x512_p3.md); stores still in L2 at
# kernel end are not counted by the capture.
NCU_TRAFFIC = {("vortex2d", "f32"): 39.760384e6 + 0.0704e6,
               ("vortex2d-512-p3", "f32"): 279.491328e6 + 217.914624e6}


def host_cpu():
    """The host CPU the oracle baseline ran on: model (or part id on Arm
    hosts without a model name) and the number of online cores."""
    import platform
    model = None
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu part") and ":" in line:
                    model = line.split(":", 1)[1].strip()
                    if key == "model name":
                        break
    except OSError:
        pass
    return {"model": model or platform.processor() or platform.machine(), "online_cores": os.cpu_count()}


def replica_aggregate(local_ms, steps, units_per_rank, device="cuda"):
    """Whole-job figures of N independent replicas: the slowest rank's timed
    region (max over ranks, after a barrier) and the units all ranks
    processed per second over it.  Single process: the local figures."""
    import torch
    import torch.distributed as dist
    ws = dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1
    max_ms = float(local_ms)
    if ws > 1:
        dist.barrier()
        t = torch.tensor([float(local_ms)], device=device, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        max_ms = float(t.item())
    ms_per_step = max_ms / steps
    return ms_per_step, ws * units_per_rank / (ms_per_step * 1e-3)


def make_workload(name):
    import workloads
    if name == "vortex2d":
        w = workloads.vortex2d(seed=0)
        desc = "vortex2d-euler-256x256-p2-D2Q4-8x8sub-K3"
    elif name == "densitywave3d":
        w = workloads.densitywave3d(seed=0)
        desc = "densitywave3d-euler-128^3-p1-D3Q6-16^3sub-K3"
    elif name == "advection1d":
        w = workloads.advection1d(seed=0, n=256, tiles=4)
        desc = "advection1d-256-p1-D1Q2-4sub-K3"
    elif name == "vortex2d-d2q3":
        w = workloads.vortex2d(seed=0, velset=1)
        desc = "vortex2d-euler-256x256-p2-D2Q3-8x8sub-K3"
    elif name == "densitywave3d-d3q4":
        w = workloads.densitywave3d(seed=0, velset=1)
        desc = "densitywave3d-euler-128^3-p1-D3Q4-16^3sub-K3"
    elif name == "vortex2d-512-p3":
        w = workloads.with_(workloads.vortex2d(seed=0, n=512, degree=3), tiles=(16, 16))
        desc = "vortex2d-euler-512x512-p3-D2Q4-16x16sub-K3"
    elif name == "maxwell3d-dirichlet":
        # every face a domain boundary with the homogeneous Dirichlet state
        # (zero field), as in the paper's body-model run
        w = workloads.with_(workloads.maxwell3d(seed=0, n=128, degree=1, tiles=16, sigma=1.0),
                            inflow=(1, 1, 1), Wb=np.zeros((3, 2, 6)))
        desc = "maxwell3d-128^3-p1-D3Q6-16^3sub-K3-sigma1-dirichlet0"
    elif name == "maxwell3d":
        w = workloads.maxwell3d(seed=0, n=128, degree=1, tiles=16, sigma=1.0)
        desc = "maxwell3d-128^3-p1-D3Q6-16^3sub-K3-sigma1"
    else:
        raise SystemExit(f"unknown workload {name}")
    return w, desc


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None
        self.thread = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            t0 = time.time()
            while not self.rows and time.time() - t0 < 5.0:    # wait until sampling is live
                time.sleep(0.02)
        except Exception:
            self.proc = None
        self.window = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append((time.perf_counter(), [x.strip() for x in line.split(",")]))

    def mark(self, t_begin, t_end):
        self.window = (t_begin, t_end)

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.thread.join(timeout=2)

    def summary(self):
        rows = self.rows
        if self.window is not None:
            a, b = self.window
            inside = [r for t, r in rows if a <= t <= b + 0.06]
            rows = inside
        else:
            rows = [r for _, r in rows]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        self_rows = rows
        sm = [float(r[1]) for r in self_rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for _, r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self_rows:
            for i, nm in enumerate(names):
                if len(r) > 5 + i and r[5 + i].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self_rows)}


def measured_peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def cpu_oracle_rate(w, budget_s=12.0, max_steps=50):
    """The oracle as it stands, single thread, timed on a bounded sample:
    whole steps of the same workload from the same initial state."""
    import oracle
    P = oracle.Problem(**w.oracle_kwargs())
    f = oracle.init(P, w.W0)
    steps = 0
    t0 = time.perf_counter()
    while steps < max_steps:
        oracle.step(P, f, 1)
        steps += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return w.kinetic_dofs * steps / dt, steps, dt


def reference_sample(w, name, steps, warmup, budget_s=100.0):
    """A bounded sample of the workload for the oracle arm: the same problem
    (same degree, velocity set, subdomain extent, time step and initial-data
    recipe) on a mesh small enough that warmup + steps oracle steps fit the
    time budget.  The oracle's cost per kinetic DOF does not depend on the
    mesh size, so the DOF-update rate of the sample is that of the workload."""
    import oracle
    import workloads
    if name != "vortex2d":
        return w, "full workload"
    sub = w.n[0] // w.tiles[0]               # subdomain extent (32 cells)
    probe = workloads.vortex2d(seed=0, n=sub, tiles=1)
    P = oracle.Problem(**probe.oracle_kwargs())
    f = oracle.init(P, probe.W0)
    t0 = time.perf_counter()
    oracle.step(P, f, 2)
    per_dof = (time.perf_counter() - t0) / (2 * probe.kinetic_dofs)
    n = w.n[0]
    while n > sub and per_dof * (steps + warmup) * (w.kinetic_dofs * (n / w.n[0]) ** 2) > budget_s:
        n //= 2
    if n == w.n[0]:
        return w, "full workload"
    s = workloads.vortex2d(seed=0, n=n, tiles=n // sub)
    return s, f"{n}x{n} cells of the same recipe ({n // sub}x{n // sub} subdomains of {sub}^2 cells)"


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    w, desc = make_workload(args.workload)
    import oracle
    s, sample = reference_sample(w, args.workload, args.steps, args.warmup)
    P = oracle.Problem(**s.oracle_kwargs())
    f = oracle.init(P, s.W0)
    for _ in range(args.warmup):
        oracle.step(P, f, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.step(P, f, 1)
    el = time.perf_counter() - t0
    value = s.kinetic_dofs * args.steps / el
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": desc, "kinetic_dofs": w.kinetic_dofs, "parallelism": "cpu-1thread"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"each step: one full step of {sample}", "host": host_cpu()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    import paper_2212_11010_gb300 as kin
    from paper_2212_11010_gb300 import build as kbuild

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    if not kbuild.up_to_date():
        if rank == 0:
            kbuild.build()
        if ws > 1:
            dist.barrier()
    kin.load_library()
    dev = torch.cuda.current_device()

    w, desc = make_workload(args.workload)
    prec = args.precision or w.precision
    kprec = kin.KIN_FP32 if prec == "f32" else kin.KIN_FP64
    stream = torch.cuda.Stream()
    ctx = kin.Context.from_workload(w, precision=kprec, torch_alloc=True, stream=stream.cuda_stream)
    W0 = np.ascontiguousarray(w.W0.reshape(-1))
    ctx.set_state(W0)
    dofs = w.kinetic_dofs
    esize = 4 if prec == "f32" else 8

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    clean = torch.ones(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    sink = torch.empty(1, dtype=torch.float32, device="cuda")

    def flush_l2():
        # write a buffer larger than L2, then read another one: the write
        # evicts the state; the read makes the write's dirty lines go back to
        # HBM before the timed step, so the step pays only for its own traffic
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
            torch.sum(clean, dim=0, keepdim=True, out=sink)

    # warm-up
    for _ in range(args.warmup):
        flush_l2()
        ctx.step(1)
    stream.synchronize()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev) as clk:
        t0 = time.perf_counter()
        for i in range(args.steps):
            flush_l2()
            starts[i].record(stream)
            ctx.step(1)
            ends[i].record(stream)
        stream.synchronize()
        wall = time.perf_counter() - t0
    torch.cuda.synchronize()
    times = [s.elapsed_time(e) for s, e in zip(starts, ends)]   # ms
    local_ms = float(np.sum(times))
    ms_per_step, value = replica_aggregate(local_ms, args.steps, dofs)

    # the same step through the public C ABI with host buffers: pinned host
    # f -> kin_set_kinetic -> kin_step(1) -> kin_get_kinetic -> pinned host
    fh = torch.empty(ctx.info.kinetic_values, dtype=torch.float32 if prec == "f32" else torch.float64,
                     pin_memory=True)
    kin.kin_get_kinetic(ctx.ctx, fh.numpy())
    e2e_steps = max(3, min(args.steps, 20))
    for _ in range(2):
        kin.kin_set_kinetic(ctx.ctx, fh.numpy())
        ctx.step(1)
        kin.kin_get_kinetic(ctx.ctx, fh.numpy())
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        kin.kin_set_kinetic(ctx.ctx, fh.numpy())
        ctx.step(1)
        kin.kin_get_kinetic(ctx.ctx, fh.numpy())
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    fbytes = ctx.info.kinetic_values * esize

    peak, peak_kind = measured_peak_hbm()
    algo_bytes = ALGO_BYTES_PER_DOF[prec] * dofs
    achieved = algo_bytes / (ms_per_step * 1e-3) / 1e9
    if prec == "f64" and w.velset == 0:
        fpd = flops_per_dof(w.dim, w.degree, w.m, 2 * w.dim, maxwell=w.system == 2)  # Maxwell system id
        tflops = fpd * dofs / (ms_per_step * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": tflops, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": tflops / FP64_PEAK_TFLOPS, "traffic": None, "peak_kind": "derived-fp64-units",
                "flops_per_dof": fpd, "hbm_GBs": achieved, "hbm_frac": achieved / peak}
    else:
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": NCU_TRAFFIC.get((args.workload, prec)),
                "peak_kind": peak_kind, "algorithmic_bytes_per_launch": algo_bytes}
    # launches of ours per step: one fused step kernel for the axis sets; the
    # d + 1 sets take a trace pass, K sweeps and a relaxation pass
    launches_per_step = 1 if w.velset == 0 else 2 + w.iters
    clocks = clk.summary()

    # result sanity (not timed): finite state
    Wf = ctx.get_state()
    finite = bool(np.isfinite(Wf).all())

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": prec, "data": "synthetic",
            "config": {"workload": desc, "kinetic_dofs": dofs, "state_bytes": fbytes,
                       "l2": "flushed before every timed step (256 MB write, then 256 MB read so the "
                             "written lines are back in HBM before the step; untimed)",
                       "block": list(ctx.info.block), "grid": ctx.info.grid,
                       "smem_bytes": ctx.info.smem_bytes,
                       "parallelism": f"replicas{ws}" if ws > 1 else "single-gpu"},
            "roofline": roof,
            "e2e": {"value": dofs / e2e_s, "unit": UNIT, "h2d_bytes_per_step": fbytes,
                    "d2h_bytes_per_step": fbytes},
            "gpu_launches": args.steps * launches_per_step,
            "clocks": clocks,
            "wall_s_timed_region": wall,
            "state_finite": finite,
        }
        if ws == 1 and not args.no_cpu_baseline:
            rate, nst, el = cpu_oracle_rate(w)
            line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                                    "sample": f"{nst} full steps of {desc} in {el:.1f} s", "host": host_cpu()}
        print(json.dumps(line), flush=True)
    ctx.close()
    if ws > 1:
        dist.destroy_process_group()


def _events_time(stream, fn, steps):
    import torch
    s = torch.cuda.Event(enable_timing=True)
    e = torch.cuda.Event(enable_timing=True)
    s.record(stream)
    for _ in range(steps):
        fn()
    e.record(stream)
    e.synchronize()
    return s.elapsed_time(e) / 1e3


def run_batched(args):
    """64 uneven 2D Euler / D2Q4 instances (n in {64,128,256,512}, p in
    {1,2,3}, vortex or density wave, dt multiple in [2,8]) stepped together in
    FP32 (one launch per degree per step, CUDA graphs), against the same
    instances in FP64 stepped one instance at a time.  The state (3.4 GB FP32)
    exceeds L2, so no flush is needed between steps."""
    import torch
    import workloads
    import paper_2212_11010_gb300 as kin
    from paper_2212_11010_gb300 import build as kbuild
    ws, rank, _ = dist_env()
    torch.cuda.set_device(0)
    if not kbuild.up_to_date():
        kbuild.build()
    kin.load_library()
    mix = workloads.batched_mix(seed=0, count=64)
    dofs = sum(w.kinetic_dofs for w in mix)
    stream = torch.cuda.Stream()
    ctxs = []
    for w in mix:
        c = kin.Context.from_workload(w, precision=kin.KIN_FP32, torch_alloc=True, stream=stream.cuda_stream)
        c.set_state(np.ascontiguousarray(w.W0.reshape(-1)))
        ctxs.append(c)
    batch = kin.Batch(ctxs, stream=stream.cuda_stream)
    batch.step(args.warmup)
    batch.sync()
    with ClockSampler(0) as clk:
        t0 = time.perf_counter()
        el = _events_time(stream, lambda: batch.step(args.steps), 1)   # K steps in one call
        clk.mark(t0, time.perf_counter())
    batch.sync()
    value = dofs * args.steps / el
    launches_per_step = len({(c.info.degree, c.info.specialised) for c in ctxs})
    batch.close()
    for c in ctxs:
        c.close()
    # plain FP64 path: the same instances one at a time
    ctx64 = []
    for w in mix:
        c = kin.Context.from_workload(w, precision=kin.KIN_FP64, torch_alloc=True, stream=stream.cuda_stream)
        c.set_state(np.ascontiguousarray(w.W0.reshape(-1)))
        ctx64.append(c)
    k64 = max(1, min(args.steps, 5))

    def one_at_a_time():
        for c in ctx64:
            c.step(1)
    one_at_a_time()
    stream.synchronize()
    el64 = _events_time(stream, one_at_a_time, k64)
    value64 = dofs * k64 / el64
    for c in ctx64:
        c.close()
    peak, peak_kind = measured_peak_hbm()
    ms = 1e3 * el / args.steps
    achieved = 8 * dofs / (ms * 1e-3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "batched-64x-euler2d-D2Q4-n64..512-p1..3-32cell-subdomains-K3",
                   "instances": len(mix), "kinetic_dofs": dofs, "state_bytes": 4 * dofs,
                   "l2": "state 3.4 GB exceeds L2; no flush", "launches_per_step": launches_per_step},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None, "peak_kind": peak_kind},
        "plain_fp64": {"value": value64, "unit": UNIT, "ms_per_step": 1e3 * el64 / k64,
                       "path": "each instance stepped alone, FP64"},
        "batched_over_plain_fp64": value / value64,
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


def run_serving(args):
    """Seeded Poisson stream (200 requests/s) of 2D Euler / D2Q4 requests, mesh
    64^2..1024^2 (log-uniform over powers of two), degree 1..3, 50..500
    steps, FP32 state resident on the device, admitted under a 150 GB budget;
    continuous batching (paper_2212_11010_gb300.serve)."""
    import torch
    import workloads
    import paper_2212_11010_gb300 as kin
    from paper_2212_11010_gb300 import build as kbuild
    from paper_2212_11010_gb300 import serve
    torch.cuda.set_device(0)
    if not kbuild.up_to_date():
        kbuild.build()
    kin.load_library()
    reqs = workloads.serving_stream(seed=0, count=args.requests, rate=200.0)
    for r in reqs:
        r.seed = 0            # one initial field per (kind, n, degree): client data, prepared up front
    for r in reqs:
        workloads.request_workload(r)
    # the clients' initial fields arrive in page-locked host memory, so that
    # their host-to-device copies run at the link's rate
    pinned = []
    for w in workloads._request_cache.values():
        t = torch.empty(w.W0.size, dtype=torch.float64, pin_memory=True)
        t.numpy()[:] = w.W0.reshape(-1)
        pinned.append(t)
        w.W0 = t.numpy().reshape(w.W0.shape)
    # warm-up: one small request through the server (module load, graph set-up paths)
    warm = workloads.serving_stream(seed=9, count=2, rate=1000.0, sizes=(64,), steps=(5, 5))
    serve.Server(budget_bytes=150e9).run(warm, workloads.request_workload)
    torch.cuda.synchronize()
    with ClockSampler(0) as clk:
        t0 = time.perf_counter()
        server = serve.Server(budget_bytes=150e9, chunk_steps=25, keep_results=False)
        recs = server.run(reqs, workloads.request_workload)
        clk.mark(t0, time.perf_counter())
    st = serve.summarize(recs, server.device_busy_s)
    peak, peak_kind = measured_peak_hbm()
    dev_gbs = 8 * st["dof_updates_per_device_s"] / 1e9
    line = {
        "metric": METRIC, "value": st["dof_updates_per_s"], "unit": UNIT, "n_gpus": 1,
        "steps": None, "warmup": 1, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "serving-poisson200-euler2d-D2Q4-n64..1024-p1..3-steps50..500",
                   "requests": st["requests"], "hbm_budget_bytes": 150e9, "chunk_steps": 25},
        "latency": {"p50_s": st["p50_s"], "p99_s": st["p99_s"], "mean_s": st["mean_s"],
                    "makespan_s": st["makespan_s"],
                    "note": "offered load exceeds the device's throughput; latency includes queueing"},
        "device": {"busy_s": st["device_busy_s"], "dof_updates_per_busy_s": st["dof_updates_per_device_s"],
                   "hbm_GBs_while_busy": dev_gbs, "hbm_frac_while_busy": dev_gbs / peak, "peak": peak,
                   "peak_kind": peak_kind,
                   "note": "CUDA-event time of the chunks on the server's stream; value is over the makespan"},
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="vortex2d",
                    choices=["vortex2d", "densitywave3d", "advection1d", "batched", "serving",
                             "vortex2d-d2q3", "densitywave3d-d3q4", "maxwell3d", "vortex2d-512-p3",
                             "maxwell3d-dirichlet"])
    ap.add_argument("--requests", type=int, default=48)
    ap.add_argument("--precision", default=None, choices=[None, "f32", "f64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "serving":
        run_serving(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
