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

        Each round enqueues one chunk of steps for the active batch, admits
        the requests that have arrived meanwhile (context creation and
        initial state run on the new contexts' own streams while the chunk
        runs), then waits for the chunk, retires finished requests and folds
        the admitted ones into the next batch.  After the run,
        self.device_busy_s holds the device time spent inside chunks."""
        import torch
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        records = {r.rid: Served(r.rid, r.arrival) for r in requests}
        active = []            # [record, context, remaining steps, bytes]
        used = 0.0
        batch = None
        # the batch runs on the server's stream; new contexts are created and
        # loaded on a second stream, so admission overlaps the running chunk
        run_stream = torch.cuda.Stream()
        adm_stream = torch.cuda.Stream()
        chunks = []            # (start, end) events of every chunk on the run stream
        self.peak_bytes = 0    # most device bytes held by admitted requests at once
        t0 = clock()

        def admit(now):
            nonlocal used
            new = []
            while pending and pending[0].arrival <= now:
                r = pending[0]
                w = workload_of(r)
                need = state_bytes_estimate(w)
                if used + need > self.budget and (active or new):
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

        while pending or active:
            k = 0
            if active:
                if batch is None:
                    # membership changes every few chunks: direct launches, no graph capture
                    batch = Batch([a[1] for a in active], stream=run_stream.cuda_stream, graphs=False,
                                  mixed=self.mixed)
                k = min(self.chunk, min(a[2] for a in active))
                ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                ev[0].record(run_stream)
                batch.step(k)                              # asynchronous
                ev[1].record(run_stream)
                chunks.append(ev)
            new = admit(clock() - t0)                      # overlaps the chunk
            if not active and not new:
                if pending:
                    time.sleep(max(0.0, pending[0].arrival - (clock() - t0)))
                continue
            still = []
            if active:
                batch.sync()
                for a in active:
                    a[2] -= k
                    if a[2] == 0:
                        rec, ctx = a[0], a[1]
                        W = self._read_result(ctx)
                        rec.finished = clock() - t0
                        if self.keep_results:
                            rec.result = W
                        used -= a[3]
                    else:
                        still.append(a)
                if len(still) != len(active) or new:
                    batch.close()
                    batch = None
                for a in active:
                    if a[2] == 0:
                        a[1].close()
            elif new and batch is not None:
                batch.close()
                batch = None
            active = still + new
        if batch is not None:
            batch.close()
        torch.cuda.synchronize()
        # device time spent inside chunks (the rest of the makespan is host
        # work between chunks, ramp-up and tail)
        self.device_busy_s = sum(a.elapsed_time(b) for a, b in chunks) * 1e-3
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
