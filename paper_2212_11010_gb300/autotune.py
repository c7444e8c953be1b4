"""Autotuner for the launch schedules of kinetic DG problems.

A schedule changes how a step is executed, never what it computes beyond
round-off.  The subdomain tiling is not a schedule: it defines which
iterate of the subdomain iteration (Sec. 5.1, eq. ibvp) the step returns, so
it is part of the problem and the tuner never changes it.

* ``tune(w)``: one problem -- cell-block extents, threads per block,
  shared-memory stages.  Builds a temporary context per candidate through
  the public C ABI and times a few steps with CUDA events (L2 flushed between
  steps when the state would fit in it).
* ``tune_batch(contexts)``: a batch of problems -- one persistent launch per
  kernel type, or one mixed-degree launch for all 2D members.  Times each
  candidate on the actual members with graph-replayed steps.

Results are cached per (GPU name, problem or batch shape), in memory and
optionally in a JSON file.
"""
from __future__ import annotations

import json
import os
from dataclasses import dataclass

import numpy as np

from . import KIN_FP32, KIN_FP64, Context, KinError


@dataclass(frozen=True)
class Schedule:
    block: tuple
    threads: int = 0
    stages: int = 0

    def kwargs(self):
        return {"block": self.block, "threads": self.threads, "stages": self.stages}


def _divisors(n):
    return [d for d in range(1, n + 1) if n % d == 0]


def candidates(w, precision, max_count: int = 24):
    """Block shapes that divide the subdomain extents (longest rows first),
    each with the default thread count, plus a few thread counts for the
    default shape."""
    L = [w.n[a] // w.tiles[a] for a in range(w.dim)]
    esize = 4 if precision == KIN_FP32 else 8
    nn = (w.degree + 1) ** w.dim
    out = [Schedule(tuple([0] * w.dim))]
    shapes = []
    for b0 in _divisors(L[0]):
        for b1 in (_divisors(L[1]) if w.dim > 1 else [1]):
            for b2 in (_divisors(L[2]) if w.dim > 2 else [1]):
                cells = b0 * b1 * b2
                smem = w.npop * cells * nn * esize
                if smem > 100 * 1024 or smem < 4 * 1024 or (b0 * nn * esize) % 16:
                    continue
                shapes.append((b0, b1, b2)[:w.dim])
    shapes.sort(key=lambda s: (-s[0], -int(np.prod(s))))
    for s in shapes[:max_count]:
        out.append(Schedule(s))
    for th in (128, 192, 256):
        out.append(Schedule(tuple([0] * w.dim), threads=th))
    return out


def _time(ctx, steps, flush):
    import torch
    times = []
    for _ in range(steps):
        if flush is not None:
            flush.fill_(1.0)
        torch.cuda.synchronize()
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record()
        ctx.step(1)
        e.record()
        e.synchronize()
        times.append(s.elapsed_time(e))
    return float(np.median(times))


_cache = {}


def _key(w, precision):
    import torch
    return json.dumps([torch.cuda.get_device_name(), w.dim, list(w.n), w.degree, w.system,
                       list(w.tiles), w.iters, int(precision)])


def tune(w, precision=None, steps: int = 8, cache_file: str = None, cands=None):
    """Fastest schedule for workload w; returns (Schedule, {schedule: ms})."""
    import torch
    prec = precision if precision is not None else (KIN_FP32 if w.precision == "f32" else KIN_FP64)
    key = _key(w, prec)
    if cache_file and os.path.exists(cache_file) and not _cache:
        try:
            with open(cache_file) as fh:
                for k, v in json.load(fh).items():
                    _cache[k] = Schedule(tuple(v["block"]), v["threads"], v["stages"])
        except (OSError, ValueError, KeyError):
            pass
    if key in _cache:
        return _cache[key], {}
    state_bytes = w.kinetic_dofs * (4 if prec == KIN_FP32 else 8)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda") \
        if state_bytes < 200e6 else None
    W0 = np.ascontiguousarray(w.W0.reshape(-1))
    timings = {}
    for cand in (cands or candidates(w, prec)):
        try:
            with Context.from_workload(w, precision=prec, **cand.kwargs()) as ctx:
                ctx.set_state(W0)
                ctx.step(2)
                timings[cand] = _time(ctx, steps, flush)
        except KinError:
            continue
    best = min(timings, key=timings.get)
    _cache[key] = best
    if cache_file:
        data = {k: {"block": list(v.block), "threads": v.threads, "stages": v.stages}
                for k, v in _cache.items()}
        with open(cache_file, "w") as fh:
            json.dump(data, fh, indent=1)
    return best, timings


@dataclass(frozen=True)
class BatchSchedule:
    mixed: bool = False      # one mixed-degree launch (KIN_BATCH_MIXED) instead of one per kernel type

    @property
    def label(self):
        return "one mixed-degree launch per step" if self.mixed else "one launch per kernel type per step"


_batch_cache = {}


def _batch_key(contexts):
    import torch
    shape = sorted((c.info.dim, c.info.degree, c.info.m, int(c.info.cells), c.info.precision,
                    tuple(c.info.block)) for c in contexts)
    return json.dumps([torch.cuda.get_device_name(), shape])


def tune_batch(contexts, stream=None, steps: int = 6, reps: int = 2):
    """Fastest batch schedule for these contexts.  Every candidate batch is
    created over the same members, run for two untimed steps, then timed on
    ``reps`` runs of ``steps`` graph-replayed steps (best run kept).  The
    members' states advance by the steps taken; returns (schedule,
    {schedule: ms per step}, steps taken)."""
    import torch
    from . import Batch
    key = _batch_key(contexts)
    if key in _batch_cache:
        return _batch_cache[key], {}, 0
    st = stream if stream is not None else torch.cuda.current_stream()
    taken = 0
    timings = {}
    for cand in (BatchSchedule(False), BatchSchedule(True)):
        with Batch(contexts, stream=st.cuda_stream, mixed=cand.mixed) as b:
            if cand.mixed and b.mixed_members == 0:
                continue
            b.step(2)
            taken += 2
            best = float("inf")
            for _ in range(reps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(st)
                b.step(steps)
                e1.record(st)
                e1.synchronize()
                taken += steps
                best = min(best, e0.elapsed_time(e1) / steps)
            b.sync()
            timings[cand] = best
    choice = min(timings, key=timings.get)
    _batch_cache[key] = choice
    return choice, timings, taken


def batch_choice(default=BatchSchedule(False)):
    """The schedule the last tune_batch on this GPU chose (or the default):
    for batches whose membership changes too often to tune each one."""
    return next(reversed(_batch_cache.values()), default) if _batch_cache else default
