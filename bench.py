"""Benchmark of the kinetic DG step on GB300.

A step is one application of S(dt) = R_omega o T_CN(dt) to the whole state:
the K = 3 subdomain-iterated downwind DG transport of every population plus
the fused over-relaxation.

Default workload (batched): 64 independent 2D compressible Euler / D2Q4
problems of uneven size -- mesh n x n with n in {64, 128, 256, 512}, DG
degree 1..3, isentropic vortex or density wave, dt = 2..8 x the explicit DG
limit, 32-cell subdomains, FP32 -- 1,105,788,928 kinetic DOF (4.4 GB, far
larger than L2, so no flush is needed between steps).  One step advances
every instance once, replayed from a captured CUDA graph with the schedule
the autotuner picks on this GPU.  The line also carries:

* roofline: algorithmic bytes (8 B per kinetic DOF in FP32: read f^n, write
  f^{n+1}) over the event-timed step, against the measured HBM copy rate;
  the per-degree launches timed alone; DRAM traffic from an ncu capture of
  the same kernels when that capture matches the current source;
* e2e: the same metric through the C ABI with host buffers -- every step
  copies every instance's f in from page-locked host memory
  (kin_set_kinetic), steps the batch, and copies every f out
  (kin_get_kinetic);
* plain_fp64: the same instances stepped one at a time in FP64;
* serving: the serving configuration's Poisson stream (1000 requests by
  default) through the continuous-batching server, p50/p99 latency;
* cpu_baseline / error_vs_oracle (the oracle leg, after the GPU work): the
  FP64 CPU oracle timed on the host cores (one thread and all of them) on a
  bounded sample of the instances, and the GPU result of sampled instances
  against the oracle run for the same number of steps.

Metric: kinetic-DOF updates per second (one kinetic DOF = one nodal value of
one population advanced by one full step).

`--workload` selects a single-problem line instead (vortex2d, densitywave3d,
...).  `--impl reference` times the FP64 CPU oracle (the test reference of
this repository) on a bounded sample of the same workload on all host cores.
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
# DRAM bytes (read + write) per launch from ncu captures, with the hash of
# the kernel sources they were taken on (source_hash): a figure is reported
# only while the sources are unchanged, else the line's traffic is null.
# Keys: (workload, precision); the batched figure is per batch step (all its
# launches), scaled from a capture of a smaller mix by the kinetic DOF.
NCU_TRAFFIC = {
    # 64-instance batched mix, one step = three launches (degree 2, 1, 3):
    # read 674.4 + 497.6 + 3411.7 MB, write 619.8 + 439.9 + 3361.0 MB
    ("batched", "f32"): (9.0044e9, "92f2ff9b2905ce7d"),
}
# the same capture per launch, keyed by degree
NCU_TRAFFIC_PER_DEGREE = {1: (0.9375e9, "92f2ff9b2905ce7d"), 2: (1.2942e9, "92f2ff9b2905ce7d"),
                          3: (6.7727e9, "92f2ff9b2905ce7d")}


# device sources of the axis-velocity step kernels (single, batched, mixed)
STEP_KERNEL_SOURCES = ("kin_device.cuh", "kin_fixed.cuh", "kin_tma.cuh", "kin_step_d1.cu", "kin_step_d2.cu",
                       "kin_step_d3.cu")


def source_hash():
    """sha256 (16 hex digits) of the step kernels' device sources."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2212_11010_gb300", "csrc")
    for name in STEP_KERNEL_SOURCES:
        with open(os.path.join(csrc, name), "rb") as fh:
            h.update(name.encode() + b"\0" + fh.read())
    return h.hexdigest()[:16]


def traffic_for(key):
    """(bytes per launch or None, note)."""
    rec = NCU_TRAFFIC.get(key)
    if rec is None:
        return None, "no ncu capture of this workload"
    nbytes, src = rec
    if src != source_hash():
        return None, f"capture taken on sources {src}; sources changed since"
    return nbytes, f"ncu capture on sources {src}"


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
                 "--format=csv,noheader,nounits", "-lms", "20"],
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

    MARGIN_S = 0.1     # samples this close to the timed window count (the region can be ~40 ms)

    def summary(self):
        rows = self.rows
        if self.window is not None:
            a, b = self.window
            inside = [r for t, r in rows if a - self.MARGIN_S <= t <= b + self.MARGIN_S]
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
                "reasons": sorted(reasons), "samples": len(self_rows),
                "window_margin_s": self.MARGIN_S, "interval_ms": 20}


def measured_peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# the oracle leg: CPU baseline and accuracy check (after the GPU work)
# ---------------------------------------------------------------------------

def _gll_weights(w):
    import oracle
    _, wq = oracle.gll(w.degree)
    cellw = np.ones(1)
    for _ in range(w.dim):
        cellw = np.kron(wq, cellw)
    return np.tile(cellw, int(np.prod(w.n)))


def state_errors(w, W, Wo, f=None, fo=None):
    """Relative errors against the oracle: per conserved variable the
    GLL-weighted L2 and the max norm (relative to the oracle's norm of that
    variable), the worst variable; and f element by element per population
    (relative to the oracle's max |f| of that population), the worst one."""
    W = np.asarray(W).reshape(w.m, -1)
    Wo = np.asarray(Wo).reshape(w.m, -1)
    q = _gll_weights(w)
    l2 = max(float(np.sqrt(np.sum(q * (W[v] - Wo[v]) ** 2) / np.sum(q * Wo[v] ** 2))) for v in range(w.m))
    linf = max(float(np.abs(W[v] - Wo[v]).max() / np.abs(Wo[v]).max()) for v in range(w.m))
    out = {"W_l2": l2, "W_linf": linf}
    if f is not None:
        f = np.asarray(f).reshape(w.npop, -1).astype(np.float64)
        fo = np.asarray(fo).reshape(w.npop, -1)
        out["f_max"] = max(float(np.abs(f[k] - fo[k]).max() / np.abs(fo[k]).max()) for k in range(w.npop))
    return out


def oracle_state(w, steps, threads=0):
    """(f, W) of the FP64 oracle after 'steps' steps from w.W0."""
    import oracle
    oracle.set_threads(threads or os.cpu_count() or 1)
    P = oracle.Problem(**w.oracle_kwargs())
    f = oracle.init(P, w.W0)
    oracle.step(P, f, steps)
    return f, oracle.moments(P, f)


def oracle_rate(ws, threads, budget_s):
    """DOF-updates/s of the oracle as it stands on 'threads' host threads:
    one step of every problem in ws, passes repeated until budget_s."""
    import oracle
    oracle.set_threads(threads)
    probs = [(oracle.Problem(**w.oracle_kwargs()), w) for w in ws]
    states = [oracle.init(P, w.W0) for P, w in probs]
    done = 0
    passes = 0
    t0 = time.perf_counter()
    while True:
        for (P, w), f in zip(probs, states):
            oracle.step(P, f, 1)
            done += w.kinetic_dofs
        passes += 1
        if time.perf_counter() - t0 > budget_s:
            break
    el = time.perf_counter() - t0
    return done / el, passes, el


def cpu_baseline_of(sample_all, desc_all, sample_one, desc_one, budget_s=12.0):
    """The oracle on all host cores and on one core, each on a bounded sample."""
    cores = os.cpu_count() or 1
    rate, passes, el = oracle_rate(sample_all, cores, budget_s)
    rate1, passes1, el1 = oracle_rate(sample_one, 1, budget_s / 3)
    return {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{passes} pass(es) of one step of {desc_all} in {el:.1f} s, OpenMP over the "
                      f"subdomains of each iteration",
            "single_thread": {"value": rate1, "unit": UNIT, "cores": 1,
                              "sample": f"{passes1} pass(es) of one step of {desc_one} in {el1:.1f} s"},
            "host": host_cpu()}


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
                "frac": achieved / peak, "traffic": traffic_for((args.workload, prec))[0],
                "traffic_note": traffic_for((args.workload, prec))[1],
                "peak_kind": peak_kind, "algorithmic_bytes_per_launch": algo_bytes}
    # launches of ours per step: one fused step kernel for the axis sets; the
    # d + 1 sets take a trace pass, K sweeps and a relaxation pass
    launches_per_step = 1 if w.velset == 0 else 2 + w.iters
    clocks = clk.summary()


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
        }
        if ws == 1 and not args.no_cpu_baseline:
            # the oracle leg: accuracy after the steps this context took (when
            # the oracle finishes them within the budget), then the CPU baseline
            steps_taken = args.warmup + args.steps + 2 + e2e_steps
            if w.kinetic_dofs * steps_taken < 4e9:
                fo, Wo = oracle_state(w, steps_taken)
                err = state_errors(w, ctx.get_state(), Wo, ctx.get_kinetic(), fo)
                err.update({"steps": steps_taken, "tolerance": 1e-5 if prec == "f32" else 1e-12})
                line["error_vs_oracle"] = err
            else:
                line["error_vs_oracle"] = {"skipped": "the oracle would exceed the time budget at this size; "
                                                      "the parity tests cover it"}
            line["cpu_baseline"] = cpu_baseline_of([w], desc, [w], desc)
        print(json.dumps(line), flush=True)
    ctx.close()
    if ws > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# tetrahedral meshes (the paper's setting)
# ---------------------------------------------------------------------------

TET_DESC = "tet-densitywave-euler-32^3x6-tets-P1-D3Q4-4^3sub-K3"


def run_tet(args):
    """3D Euler density wave on the periodic unit cube meshed by 32^3 cubes x
    6 tetrahedra (196,608 cells, P1 nodes at the vertices), D3Q4 (the
    paper's cube diagonals), 4^3 subdomains of 8^3 cubes, K = 3,
    dt = 5 h_min / |V|, FP32: 15,728,640 kinetic DOF (63 MB).  A step is K
    sweep launches (one block per subdomain and velocity, walking the
    breadth-first levels) and one extrapolation + relaxation launch."""
    import torch
    import workloads
    import paper_2212_11010_gb300 as kin
    ws, rank, dev = _setup_gpu()
    w = workloads.tet_densitywave(seed=0, n=32, tiles=4, velset=1, dt_mult=5.0)
    prec = args.precision or w.precision
    kprec = kin.KIN_FP32 if prec == "f32" else kin.KIN_FP64
    stream = torch.cuda.Stream()
    ctx = kin.TetContext.from_workload(w, precision=kprec, torch_alloc=True, stream=stream.cuda_stream)
    ctx.set_state(np.ascontiguousarray(w.W0.reshape(-1)))
    dofs = w.kinetic_dofs
    esize = 4 if prec == "f32" else 8
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def flush_l2():
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
    for _ in range(args.warmup):
        flush_l2()
        ctx.step(1)
    stream.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(dev) as clk:
        t0 = time.perf_counter()
        for a, b in ev:
            flush_l2()
            a.record(stream)
            ctx.step(1)
            b.record(stream)
        stream.synchronize()
        clk.mark(t0, time.perf_counter())
    ms_per_step, value = replica_aggregate(float(np.sum([a.elapsed_time(b) for a, b in ev])), args.steps, dofs)
    peak, peak_kind = measured_peak_hbm()
    # bytes a step must move with K literal sweeps: every sweep reads f^n and
    # writes its iterate, the final launch reads f^n and the last iterate and
    # writes f^{n+1} -- (2 K + 3) x the state; the floor of one read and one
    # write (8 B per DOF in FP32) is what the roofline fraction is taken on
    algo_bytes = ALGO_BYTES_PER_DOF[prec] * dofs
    achieved = algo_bytes / (ms_per_step * 1e-3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": prec, "data": "synthetic",
        "config": {"workload": TET_DESC, "cells": w.mesh.cells, "kinetic_dofs": dofs, "state_bytes": esize * dofs,
                   "subdomains": int(w.subdomains().max()) + 1, "l2": "256 MB written before every timed step",
                   "launches_per_step": w.iters + 1},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None, "peak_kind": peak_kind, "algorithmic_bytes_per_launch": algo_bytes,
                     "note": f"K + 1 = {w.iters + 1} launches per step move about {2 * w.iters + 3} x the state"},
        "gpu_launches": (w.iters + 1) * args.steps,
        "clocks": clk.summary(),
    }
    if rank == 0 and not args.no_cpu_baseline:
        # accuracy on the same recipe at 8^3 cubes (the oracle at 32^3 would
        # take minutes), after the same number of steps
        import oracle
        ws8 = workloads.tet_densitywave(seed=0, n=8, tiles=1, velset=1, dt_mult=5.0)
        nst = args.warmup + args.steps
        with kin.TetContext.from_workload(ws8, precision=kprec) as c8:
            c8.set_state(np.ascontiguousarray(ws8.W0.reshape(-1)))
            c8.step(nst)
            W8, f8 = c8.get_state(), c8.get_kinetic()
        oracle.set_threads(os.cpu_count() or 1)
        P = oracle.tet_problem(ws8)
        T = oracle.TetMesh.from_workload(ws8)
        fo = oracle.tet_init(P, T, ws8.W0)
        oracle.tet_step(P, T, fo, nst)
        Wo = oracle.tet_moments(P, T, fo).reshape(ws8.m, -1)
        W8 = W8.reshape(ws8.m, -1)
        line["error_vs_oracle"] = {
            "W_linf": max(float(np.abs(W8[v] - Wo[v]).max() / np.abs(Wo[v]).max()) for v in range(ws8.m)),
            "f_max": float(np.abs(f8 - fo).max() / np.abs(fo).max()), "steps": nst,
            "sample": "the same recipe on 8^3 cubes x 6 tetrahedra, one subdomain"}
        # the oracle's rate on that sample, all cores and one
        t0 = time.perf_counter()
        oracle.tet_step(P, T, fo, 2)
        el = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": 2 * ws8.kinetic_dofs / el, "unit": UNIT, "cores": os.cpu_count(),
                                "kind": "oracle", "sample": f"2 steps of the 8^3-cube recipe in {el:.1f} s",
                                "host": host_cpu()}
    ctx.close()
    if rank == 0:
        print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# batched (default)
# ---------------------------------------------------------------------------

BATCHED_DESC = "batched-64x-euler2d-D2Q4-n64..512-p1..3-32cell-subdomains-K3"


def _setup_gpu():
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
            import torch.distributed as dist
            dist.barrier()
    kin.load_library()
    return ws, rank, torch.cuda.current_device()


def _time_batch(batch, stream, steps):
    """Per-step CUDA-event times (ms) of 'steps' single-step graph replays."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for a, b in ev:
        a.record(stream)
        batch.step(1)
        b.record(stream)
    stream.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def run_batched(args):
    """The batched configuration: 64 uneven 2D Euler / D2Q4 instances stepped
    together in FP32.  See the module docstring for the fields."""
    import torch
    import workloads
    import paper_2212_11010_gb300 as kin
    from paper_2212_11010_gb300 import autotune
    ws, rank, dev = _setup_gpu()
    mix = workloads.batched_mix(seed=0, count=args.instances)
    dofs = sum(w.kinetic_dofs for w in mix)
    stream = torch.cuda.Stream()
    ctxs = []
    for w in mix:
        c = kin.Context.from_workload(w, precision=kin.KIN_FP32, torch_alloc=True, stream=stream.cuda_stream)
        c.set_state(np.ascontiguousarray(w.W0.reshape(-1)))
        ctxs.append(c)
    steps_done = [0] * len(mix)

    # schedule: the autotuner times the candidate batch schedules on these
    # members (untimed); --schedule fixes it instead (profiler runs, where
    # serialised launches would skew the tuner's timings)
    if args.schedule == "auto":
        sched, sched_ms, taken = autotune.tune_batch(ctxs, stream)
    else:
        sched, sched_ms, taken = autotune.BatchSchedule(args.schedule == "mixed"), {}, 0
    steps_done = [s + taken for s in steps_done]
    batch = kin.Batch(ctxs, stream=stream.cuda_stream, mixed=sched.mixed)
    batch.step(args.warmup)
    batch.sync()
    steps_done = [s + args.warmup for s in steps_done]

    # timed region: K single-step graph replays, CUDA events on the batch stream
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev) as clk:
        t0 = time.perf_counter()
        times = _time_batch(batch, stream, args.steps)
        clk.mark(t0, time.perf_counter())
    torch.cuda.synchronize()
    steps_done = [s + args.steps for s in steps_done]
    launches = batch.launches_per_step
    batch.close()
    ms_per_step, value = replica_aggregate(float(np.sum(times)), args.steps, dofs)

    # each kernel type's launch alone (the same members, untimed for the metric)
    per_kernel = []
    for p in sorted({w.degree for w in mix}):
        idx = [i for i, w in enumerate(mix) if w.degree == p]
        with kin.Batch([ctxs[i] for i in idx], stream=stream.cuda_stream) as b:
            b.step(2)
            t = _time_batch(b, stream, args.steps)
        for i in idx:
            steps_done[i] += 2 + args.steps
        d = sum(mix[i].kinetic_dofs for i in idx)
        ms = float(np.mean(t))
        per_kernel.append({"kernel": f"step_kernel_fixed_batch, degree {p}, block {list(ctxs[idx[0]].info.block)}",
                           "instances": len(idx), "kinetic_dofs": d, "ms": ms,
                           "GBs": 8 * d / (ms * 1e-3) / 1e9})

    peak, peak_kind = measured_peak_hbm()
    algo_bytes = ALGO_BYTES_PER_DOF["f32"] * dofs
    achieved = algo_bytes / (ms_per_step * 1e-3) / 1e9
    traffic, traffic_note = traffic_for(("batched", "f32")) if args.instances == 64 else (None, "not the 64-instance mix")
    for k, p in zip(per_kernel, sorted({w.degree for w in mix})):
        k["frac"] = k["GBs"] / peak
        rec = NCU_TRAFFIC_PER_DEGREE.get(p)
        k["traffic"] = rec[0] if rec and rec[1] == source_hash() and args.instances == 64 else None
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "peak_kind": peak_kind, "algorithmic_bytes_per_launch": algo_bytes,
            "kernel": f"the batch step: {launches} launch(es) of the fused step kernel ({sched.label}), "
                      "back to back on one stream; per step 8 B per kinetic DOF",
            "traffic_note": traffic_note, "per_kernel": per_kernel}

    # e2e through the C ABI with host buffers: every step copies every
    # instance's f in from page-locked host memory and its result out.  The
    # instances form two batches of about equal bytes, each on its own stream,
    # and the copies are pipelined per instance: an instance's input for the
    # next step goes in (one copy stream) as soon as its result has left (the
    # other), and one half steps while the other half's copies run, so both
    # directions of the host link stay busy.  The timed region holds every
    # step's copies both ways.
    # one page-locked buffer per instance: its result lands there and is the
    # next step's input, in that order (the per-instance event)
    fh = [torch.empty(c.info.kinetic_values, dtype=torch.float32, pin_memory=True) for c in ctxs]
    for c, h in zip(ctxs, fh):
        kin.kin_get_kinetic(c.ctx, h.numpy())
    e2e_steps = max(2, min(args.steps, 4))
    halves, size = [[], []], [0, 0]
    for i in sorted(range(len(ctxs)), key=lambda i: -ctxs[i].info.kinetic_values):
        k = 0 if size[0] <= size[1] else 1
        halves[k].append(i)
        size[k] += ctxs[i].info.kinetic_values
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
    s_step = [torch.cuda.Stream(), torch.cuda.Stream()]
    left = [torch.cuda.Event() for _ in ctxs]
    arrived, stepped = [torch.cuda.Event(), torch.cuda.Event()], [torch.cuda.Event(), torch.cuda.Event()]
    halves_b = [kin.Batch([ctxs[i] for i in h], stream=s_step[k].cuda_stream, mixed=sched.mixed)
                for k, h in enumerate(halves)]
    try:
        def e2e_step():
            for k in (0, 1):
                for i in halves[k]:
                    s_in.wait_event(left[i])        # this instance's last result has left
                    kin.kin_set_kinetic_async(ctxs[i].ctx, fh[i], s_in.cuda_stream)
                arrived[k].record(s_in)
            for k in (0, 1):
                s_step[k].wait_event(arrived[k])
                halves_b[k].step(1)
                stepped[k].record(s_step[k])
            for k in (0, 1):
                s_out.wait_event(stepped[k])
                for i in halves[k]:
                    kin.kin_get_kinetic_async(ctxs[i].ctx, fh[i], s_out.cuda_stream)
                    left[i].record(s_out)
        e2e_step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            e2e_step()
        torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / e2e_steps
    finally:
        for hb in halves_b:
            hb.close()
    steps_done = [s + 1 + e2e_steps for s in steps_done]
    del fh

    # the plain path: the same instances in FP64, one instance at a time
    ctx64 = []
    for w in mix:
        c = kin.Context.from_workload(w, precision=kin.KIN_FP64, torch_alloc=True, stream=stream.cuda_stream)
        c.set_state(np.ascontiguousarray(w.W0.reshape(-1)))
        ctx64.append(c)
    k64 = max(1, min(args.steps, 3))

    def one_at_a_time():
        for c in ctx64:
            c.step(1)
    one_at_a_time()
    stream.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(k64):
        one_at_a_time()
    e1.record(stream)
    e1.synchronize()
    el64 = e0.elapsed_time(e1) * 1e-3
    value64 = dofs * k64 / el64
    steps64 = 1 + k64

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": BATCHED_DESC if args.instances == 64 else
                   BATCHED_DESC.replace("64x", f"{args.instances}x"), "instances": len(mix), "kinetic_dofs": dofs,
                   "state_bytes": 4 * dofs,
                   "l2": f"state {4 * dofs / 1e9:.1f} GB exceeds L2 (129 MB); no flush"
                         if 4 * dofs > 1e9 else "state comparable to L2: not for roofline figures",
                   "launches_per_step": launches, "schedule": sched.label,
                   "schedule_ms_per_step": {s_.label: v for s_, v in sched_ms.items()},
                   "parallelism": f"replicas{ws}" if ws > 1 else "single-gpu"},
        "roofline": roof,
        "e2e": {"value": dofs / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 4 * dofs,
                "d2h_bytes_per_step": 4 * dofs,
                "path": "per step: kin_set_kinetic_async of every instance from page-locked host memory, "
                        "kin_batch_step of two halves of the instances (two batches, one stream each), "
                        "kin_get_kinetic_async of every instance into page-locked host memory; each "
                        "instance's input for the next step goes in while other results come out, and "
                        "one half steps while the other's copies run (two copy streams, ordered per "
                        "instance by events)"},
        "plain_fp64": {"value": value64, "unit": UNIT, "ms_per_step": 1e3 * el64 / k64,
                       "path": "each instance stepped alone (kin_step), FP64"},
        "batched_over_plain_fp64": value / value64,
        "gpu_launches": launches * args.steps,
        "clocks": clk.summary(),
    }
    if not args.no_serving and ws == 1:
        line["serving"] = serving_object(args)

    # the oracle leg (rank 0, one GPU): accuracy of sampled instances, CPU baseline
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        sample = []
        for p in sorted({w.degree for w in mix}):
            i = min((i for i, w in enumerate(mix) if w.degree == p), key=lambda i: (mix[i].n[0], i))
            sample.append(i)
        errs32, errs64 = [], []
        for i in sample:
            w = mix[i]
            fo, Wo = oracle_state(w, steps_done[i])
            e = state_errors(w, ctxs[i].get_state(), Wo, ctxs[i].get_kinetic(), fo)
            e.update({"instance": i, "n": w.n[0], "degree": w.degree, "steps": steps_done[i]})
            errs32.append(e)
            fo, Wo = oracle_state(w, steps64)
            e = state_errors(w, ctx64[i].get_state(), Wo, ctx64[i].get_kinetic(), fo)
            e.update({"instance": i, "steps": steps64})
            errs64.append(e)
        line["error_vs_oracle"] = {
            "f32": {k: max(e[k] for e in errs32) for k in ("W_l2", "W_linf", "f_max")},
            "f64": {k: max(e[k] for e in errs64) for k in ("W_l2", "W_linf", "f_max")},
            "tolerance": {"f32": 1e-5, "f64": 1e-12, "applies_to": "W_l2, W_linf"},
            "sample": errs32, "sample_f64": errs64,
            "note": "the smallest instance of each degree, against the FP64 oracle run for the same steps"}
        small = [w for w in mix if w.n[0] <= 128]
        one = [w for w in mix if w.n[0] == 64]
        line["cpu_baseline"] = cpu_baseline_of(small, f"the {len(small)} instances with n <= 128",
                                               one, f"the {len(one)} instances with n = 64")
    for c in ctx64:
        c.close()
    for c in ctxs:
        c.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# serving (nested in the batched line, or alone with --workload serving)
# ---------------------------------------------------------------------------

SERVING_DESC = "serving-poisson200-euler2d-D2Q4-n64..1024-loguniform-p1..3-steps50..500-budget150GB"


def serving_object(args):
    """The serving configuration: a seeded Poisson stream (mean 200 requests
    per second) of 2D Euler / D2Q4 requests, mesh n x n with n log-uniform on
    [64, 1024] (rounded to the 32-cell subdomain extent), degree 1..3, 50..500
    steps, FP32 state resident on the device, admitted under a 150 GB budget
    and advanced by the continuous-batching server."""
    import torch
    from concurrent.futures import ThreadPoolExecutor
    import workloads
    from paper_2212_11010_gb300 import serve
    reqs = workloads.serving_stream(seed=0, count=args.requests, rate=200.0, size_range=(64, 1024))
    for r in reqs:
        r.seed = 0            # one initial field per (kind, n, degree): client data prepared up front
    uniq = {}
    for r in reqs:
        uniq.setdefault((r.kind, r.n, r.degree), r)
    t0 = time.perf_counter()
    with ThreadPoolExecutor(max(1, min(16, os.cpu_count() or 1))) as ex:
        list(ex.map(workloads.request_workload, uniq.values()))
    # the clients' fields arrive in page-locked host memory, so that their
    # host-to-device copies run at the link's rate (request_workload hands
    # out copies of these cached recipes, sharing their W0)
    pinned = []
    for key, w in list(workloads._request_cache.items()):
        t = torch.empty(w.W0.size, dtype=torch.float64, pin_memory=True)
        t.numpy()[:] = w.W0.reshape(-1)
        pinned.append(t)
        w.W0 = t.numpy().reshape(w.W0.shape)
    prep_s = time.perf_counter() - t0
    warm = workloads.serving_stream(seed=9, count=2, rate=1000.0, sizes=(64,), steps=(5, 5))
    serve.Server(budget_bytes=150e9).run(warm, workloads.request_workload)
    torch.cuda.synchronize()
    with ClockSampler(torch.cuda.current_device()) as clk:
        t0 = time.perf_counter()
        server = serve.Server(budget_bytes=150e9, chunk_steps=25, keep_results=False)
        recs = server.run(reqs, workloads.request_workload)
        clk.mark(t0, time.perf_counter())
    st = serve.summarize(recs, server.device_busy_s)
    peak, peak_kind = measured_peak_hbm()
    dev_gbs = 8 * st["dof_updates_per_device_s"] / 1e9
    waited = sum(1 for r in recs if r.admitted - r.arrival > 0.05)
    workloads._request_cache.clear()
    del pinned
    return {"workload": SERVING_DESC, "requests": st["requests"], "distinct_meshes": len({r.n for r in reqs}),
            "value": st["dof_updates_per_s"], "unit": UNIT,
            "p50_s": st["p50_s"], "p99_s": st["p99_s"], "mean_s": st["mean_s"],
            "makespan_s": st["makespan_s"], "arrival_span_s": reqs[-1].arrival,
            "note": "offered load exceeds the device's throughput; latency includes queueing",
            "admitted_after_50ms_wait": waited, "peak_device_bytes": server.peak_bytes,
            "hbm_budget_bytes": 150e9, "chunk_steps": 25, "schedule": "mixed" if server.mixed else "per kernel type",
            "device": {"busy_s": st["device_busy_s"], "dof_updates_per_busy_s": st["dof_updates_per_device_s"],
                       "hbm_GBs_while_busy": dev_gbs, "hbm_frac_while_busy": dev_gbs / peak,
                       "peak": peak, "peak_kind": peak_kind},
            "client_data_prep_s": prep_s, "clocks": clk.summary()}


def run_serving(args):
    _setup_gpu()
    obj = serving_object(args)
    line = {"metric": METRIC, "value": obj["value"], "unit": UNIT, "n_gpus": 1, "steps": None,
            "warmup": 1, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": SERVING_DESC, "requests": obj["requests"]}, "serving": obj}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# the reference arm: the oracle on the host cores
# ---------------------------------------------------------------------------

def run_reference(args):
    """The FP64 CPU oracle as it stands, on all host cores, on the default
    line's workload and metric: each step is one oracle step of a bounded
    sample of the workload (for the batched mix: every instance with
    n <= 128; for a single problem: the problem itself, or a smaller mesh
    of the same recipe when a step of the full one would not fit the budget)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    import workloads
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    if args.workload == "batched":
        mix = workloads.batched_mix(seed=0, count=64)
        sample = [w for w in mix if w.n[0] <= 128]
        desc, sdesc = BATCHED_DESC, f"the {len(sample)} instances with n <= 128"
        dofs_total = sum(w.kinetic_dofs for w in mix)
    else:
        w, desc = make_workload(args.workload)
        s, sdesc = reference_sample(w, args.workload, args.steps, args.warmup)
        sample = [s]
        dofs_total = w.kinetic_dofs
    probs = [(oracle.Problem(**w.oracle_kwargs()), w) for w in sample]
    states = [oracle.init(P, w.W0) for P, w in probs]

    def one():
        for (P, w), f in zip(probs, states):
            oracle.step(P, f, 1)
    for _ in range(args.warmup):
        one()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one()
    el = time.perf_counter() - t0
    value = sum(w.kinetic_dofs for w in sample) * args.steps / el
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": desc, "kinetic_dofs": dofs_total, "parallelism": f"cpu-{cores}threads"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"each step: one oracle step of {sdesc}", "host": host_cpu()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def reference_sample(w, name, steps, warmup, budget_s=100.0):
    """A bounded sample of a single-problem workload for the oracle arm: the
    same recipe (degree, velocity set, subdomain extent, time step) on a mesh
    small enough that warmup + steps oracle steps fit the time budget.  The
    oracle's cost per kinetic DOF does not depend on the mesh size."""
    import workloads
    if name != "vortex2d":
        return w, "the full workload"
    sub = w.n[0] // w.tiles[0]               # subdomain extent (32 cells)
    n = w.n[0]
    per_dof = 1.0 / (2e7 * max(1, (os.cpu_count() or 1) // 2))
    while n > sub and per_dof * (steps + warmup) * (w.kinetic_dofs * (n / w.n[0]) ** 2) > budget_s:
        n //= 2
    if n == w.n[0]:
        return w, "the full workload"
    s = workloads.vortex2d(seed=0, n=n, tiles=n // sub)
    return s, f"{n}x{n} cells of the same recipe ({n // sub}x{n // sub} subdomains of {sub}^2 cells)"


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batched",
                    choices=["batched", "serving", "vortex2d", "densitywave3d", "advection1d",
                             "vortex2d-d2q3", "densitywave3d-d3q4", "maxwell3d", "vortex2d-512-p3",
                             "maxwell3d-dirichlet", "tet-densitywave"])
    ap.add_argument("--requests", type=int, default=1000)
    ap.add_argument("--schedule", default="auto", choices=["auto", "per-type", "mixed"],
                    help="batch schedule: chosen by the autotuner (auto) or fixed")
    ap.add_argument("--instances", type=int, default=64,
                    help="instances of the batched mix (64 is the configuration; fewer for small profiler captures)")
    ap.add_argument("--precision", default=None, choices=[None, "f32", "f64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "serving":
        run_serving(args)
    elif args.workload == "tet-densitywave":
        run_tet(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
