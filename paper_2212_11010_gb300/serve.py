"""Continuous-batching request loop over the C ABI.

Requests (one kinetic DG simulation each: mesh, degree, step count) arrive
over time.  The server keeps every admitted request's kinetic state resident
on the device, admits arrivals in order as long as the device-memory budget
allows, and advances all active requests together: each round is one
kin_batch_step over the active set (one launch per kernel type per step),
after which finished requests are read back and retired and newly arrived
ones join.  Latency of a request = completion time - arrival time.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from . import KIN_FP32, Batch, Context


@dataclass
class Served:
    rid: int
    arrival: float
    admitted: float = None
    finished: float = None
    steps: int = 0
    dofs: int = 0
    result: np.ndarray = field(default=None, repr=False)

    @property
    def latency(self):
        return self.finished - self.arrival


def state_bytes_estimate(w, esize=4) -> int:
    """Conservative device bytes of a request before its context exists:
    kinetic state, block summaries (at most half of it) and FP64 staging."""
    f = w.kinetic_dofs * esize
    return int(f * 1.5 + w.m * w.nodes * 8 + (1 << 20))


class Server:
    def __init__(self, budget_bytes: float = 150e9, chunk_steps: int = 25, torch_alloc: bool = True,
                 keep_results: bool = True, pinned_results: bool = True, mixed=None):
        self.budget = float(budget_bytes)
        # batch schedule: the autotuner's choice for this GPU unless given
        # (membership changes every few chunks, too often to tune each batch)
        if mixed is None:
            from .autotune import batch_choice
            mixed = batch_choice().mixed
        self.mixed = bool(mixed)
        self.chunk = int(chunk_steps)
        self.torch_alloc = torch_alloc
        self.keep_results = keep_results
        # results are read back into page-locked host buffers (reused by size
        # when the caller does not keep them), so the device-to-host copy runs
        # at the link's rate instead of through the driver's staging copies
        self.pinned_results = pinned_results
        self._pool = {}

    def _result_buffer(self, n):
        free = self._pool.setdefault(n, [])
        if free:
            return free.pop()
        import torch
        return torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()

    def _read_result(self, ctx):
        n = ctx.info.state_values
        if not self.pinned_results:
            return ctx.get_state()
        buf = self._result_buffer(n)
        ctx.get_state(buf)
        if self.keep_results:
            return buf                                  # handed to the caller
        self._pool[n].append(buf)
        return None

    def run(self, requests, workload_of, clock=time.perf_counter):
        """requests: objects with rid, arrival (s), steps; workload_of(r) -> Workload.
        Returns the Served records in request order.

        The loop keeps one chunk of steps queued behind the one that runs.
        Each round enqueues the next chunk for the active set, then waits
        for the previous chunk, reads back and retires the requests that
        finished with it and admits the requests that have arrived (context
        creation and initial state on a separate, high-priority stream), all
        while the new chunk runs.  A change of membership makes a new batch
        on the other of two run streams; it is ordered after the running
        chunk through its continuing members' events.  After the run,
        self.device_busy_s holds the device time covered by chunks."""
        import torch

        pending = deque(sorted(requests, key=lambda r: r.arrival))
        records = {r.rid: Served(r.rid, r.arrival) for r in requests}
        active = []            # [record, context, remaining steps, bytes]
        used = 0.0
        run_streams = (torch.cuda.Stream(), torch.cuda.Stream())
        which = 0              # run stream of the next batch
        try:
            lo, hi = torch.cuda.Stream.priority_range()
            adm_stream = torch.cuda.Stream(priority=min(lo, hi))     # the highest priority
        except (AttributeError, RuntimeError):
            adm_stream = torch.cuda.Stream()
        origin = torch.cuda.Event(enable_timing=True)
        origin.record(run_streams[0])
        chunks = []            # (start, end) events of every chunk
        self.peak_bytes = 0    # most device bytes held by admitted requests at once
        t0 = clock()

        def admit(now):
            nonlocal used
            new = []
            while pending and pending[0].arrival <= now:
                r = pending[0]
                w = workload_of(r)
                need = state_bytes_estimate(w)
                if used > 0 and used + need > self.budget:
                    break                                  # wait for memory to free up
                pending.popleft()
                ctx = Context.from_workload(w, precision=KIN_FP32, torch_alloc=self.torch_alloc,
                                            stream=adm_stream.cuda_stream)
                ctx.set_state(np.ascontiguousarray(w.W0.reshape(-1)))
                rec = records[r.rid]
                rec.admitted = clock() - t0
                rec.steps = r.steps
                rec.dofs = w.kinetic_dofs
                used += ctx.info.device_bytes
                self.peak_bytes = max(self.peak_bytes, used)
                new.append([rec, ctx, r.steps, ctx.info.device_bytes])
            return new

        def retire(done):
            nonlocal used
            for rec, ctx, _, nbytes in done:
                W = self._read_result(ctx)
                rec.finished = clock() - t0
                if self.keep_results:
                    rec.result = W
                ctx.close()
                used -= nbytes

        batch = None           # batch of the active set
        inflight = None        # (end event, finished entries, batch) of the chunk queued last
        while pending or active or inflight is not None:
            queued = None
            if active:
                if batch is None:
                    # membership changes every few chunks: direct launches, no graph capture
                    run = run_streams[which]
                    batch = Batch([a[1] for a in active], stream=run.cuda_stream, graphs=False,
                                  mixed=self.mixed)
                # chunks bound the wait of a pending request; with none
                # pending, a chunk runs up to the next finish
                k = min(a[2] for a in active)
                if pending:
                    k = min(k, self.chunk)
                ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                ev[0].record(run)
                batch.step(k)                              # asynchronous
                ev[1].record(run)
                chunks.append(ev)
                for a in active:
                    a[2] -= k
                queued = (ev[1], [a for a in active if a[2] == 0], batch)
                active = [a for a in active if a[2] > 0]
            if inflight is not None:
                inflight[0].synchronize()                  # the previous chunk; the queued one runs
                if inflight[2] is not batch:               # superseded: its stream is idle
                    # (a member's device error word is checked when its result is read)
                    inflight[2].close()                    # before its finished members go
                retire(inflight[1])
            new = admit(clock() - t0)
            if queued is not None and (queued[1] or new) and batch is queued[2]:
                batch = None                               # the next chunk needs a new batch
                which ^= 1
            active = active + new
            inflight = queued
            if not active and inflight is None and pending:
                time.sleep(max(0.0, pending[0].arrival - (clock() - t0)))
        if batch is not None:
            batch.close()
        torch.cuda.synchronize()
        # device time covered by chunks (the union of their intervals; the
        # rest of the makespan is host work between chunks, ramp-up and tail)
        spans = sorted((origin.elapsed_time(a), origin.elapsed_time(b)) for a, b in chunks)
        busy, end = 0.0, float("-inf")
        for a, b in spans:
            if b > end:
                busy += b - max(a, end)
                end = b
        self.device_busy_s = busy * 1e-3
        return [records[r.rid] for r in requests]


def summarize(records, device_busy_s=None):
    lat = np.array([r.latency for r in records])
    t_first = min(r.arrival for r in records)
    t_last = max(r.finished for r in records)
    work = sum(r.dofs * r.steps for r in records)
    return {"requests": len(records), "p50_s": float(np.percentile(lat, 50)),
            "p99_s": float(np.percentile(lat, 99)), "mean_s": float(lat.mean()),
            "makespan_s": t_last - t_first, "dof_updates": work,
            "dof_updates_per_s": work / (t_last - t_first),
            "device_busy_s": device_busy_s,
            "dof_updates_per_device_s": work / device_busy_s if device_busy_s else None}
