"""Host logic of the continuous-batching loop (serve.Server.run), on the CPU.

The contexts, batches, streams and events are fakes that keep the state the
library keeps (steps done per context, which batch last stepped it) and the
order the device would impose (a chunk completes only after the chunks of
other batches that its members were last stepped by).  The checks: every
request gets exactly its steps; the admitted bytes never exceed the budget;
a request can wait for memory; a batch is never stepped after it is closed
and never steps a member that another batch stepped since it was made; a
batch is closed before any of its members; a context is freed only after the
last chunk that stepped it is complete; and at most one chunk is queued
behind the one that runs."""
import types

import numpy as np
import pytest
import torch

from paper_2212_11010_gb300 import serve


class World:
    def __init__(self):
        self.chunks = []          # {"deps": [...], "done": bool, "stream": FakeStream}
        self.max_outstanding = 0
        self.batches = []


class FakeStream:
    world = None

    def __init__(self, *a, **kw):
        self.ops = []             # chunk indices in stream order
        self.cuda_stream = id(self)


def _complete(world, idx):
    ch = world.chunks[idx]
    if ch["done"]:
        return
    for d in ch["deps"]:
        _complete(world, d)
    # stream order: everything queued before it on its stream completes first
    for j in ch["stream"].ops:
        if j == idx:
            break
        _complete(world, j)
    ch["done"] = True


class FakeEvent:
    world = None

    def __init__(self, enable_timing=False):
        self.stream, self.upto = None, 0

    def record(self, stream=None):
        self.stream, self.upto = stream, len(stream.ops)

    def synchronize(self):
        for j in self.stream.ops[:self.upto]:
            _complete(self.world, j)

    def elapsed_time(self, other):
        return 0.0


class FakeContext:
    world = None

    def __init__(self, w):
        self.w = w
        self.steps = 0
        self.last_chunk = None
        self.closed = False
        self.info = types.SimpleNamespace(device_bytes=w.bytes, state_values=4)

    @classmethod
    def from_workload(cls, w, precision=None, torch_alloc=False, stream=None):
        return cls(w)

    def set_state(self, W):
        assert not self.closed

    def get_state(self, out=None):
        assert not self.closed
        # the library orders the read after the context's last batch step
        if self.last_chunk is not None:
            _complete(self.world, self.last_chunk)
        return np.full(4, float(self.steps))

    def close(self):
        assert not self.closed
        # freeing is safe only once nothing on the device uses the memory
        assert self.last_chunk is None or self.world.chunks[self.last_chunk]["done"]
        for b in self.world.batches:
            assert b.closed or self not in b.members, "a context closed while its batch is open"
        self.closed = True


class FakeBatch:
    world = None

    def __init__(self, contexts, stream=None, graphs=True, mixed=False):
        self.members = list(contexts)
        self.stream = stream_of[stream]
        self.expect = [c.steps for c in self.members]
        self.closed = False
        self.world.batches.append(self)

    def step(self, n=1):
        assert not self.closed
        world = self.world
        outstanding = sum(1 for ch in world.chunks if not ch["done"])
        world.max_outstanding = max(world.max_outstanding, outstanding)
        deps = []
        for c, e in zip(self.members, self.expect):
            assert not c.closed
            assert c.steps == e, "member stepped outside this batch"
            if c.last_chunk is not None:
                deps.append(c.last_chunk)
        idx = len(world.chunks)
        world.chunks.append({"deps": deps, "done": False, "stream": self.stream})
        self.stream.ops.append(idx)
        for i, c in enumerate(self.members):
            c.steps += n
            c.last_chunk = idx
            self.expect[i] += n

    def sync(self):
        for j in self.stream.ops:
            _complete(self.world, j)

    def close(self):
        assert not self.closed
        for c in self.members:
            assert not c.closed, "members must outlive their batch"
        self.sync()
        self.closed = True


stream_of = {}


@pytest.fixture
def world(monkeypatch):
    w = World()
    for cls in (FakeStream, FakeEvent, FakeContext, FakeBatch):
        monkeypatch.setattr(cls, "world", w)

    def make_stream(*a, **kw):
        s = FakeStream()
        stream_of[s.cuda_stream] = s
        return s

    monkeypatch.setattr(torch.cuda, "Stream", make_stream)
    monkeypatch.setattr(torch.cuda, "Event", FakeEvent)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a: [_complete(w, j) for j in range(len(w.chunks))])
    monkeypatch.setattr(serve, "Context", FakeContext)
    monkeypatch.setattr(serve, "Batch", FakeBatch)
    yield w
    stream_of.clear()


def _requests(seed, count, spread_s):
    rng = np.random.default_rng(seed)
    arrivals = np.sort(rng.uniform(0.0, spread_s, count))
    return [types.SimpleNamespace(rid=i, arrival=float(t), steps=int(rng.integers(3, 40)),
                                  size=int(rng.integers(1, 5)))
            for i, t in enumerate(arrivals)]


def _workload(r):
    dofs = 1000 * r.size
    w = types.SimpleNamespace(kinetic_dofs=dofs, m=4, nodes=dofs // 16, W0=np.zeros(4))
    w.bytes = serve.state_bytes_estimate(w)
    return w


@pytest.mark.parametrize("seed,count,chunk,budget_requests", [(0, 40, 7, 3), (1, 25, 10, 100), (2, 60, 4, 1)])
def test_serving_loop_bookkeeping(world, seed, count, chunk, budget_requests):
    reqs = _requests(seed, count, spread_s=0.02)
    need = [_workload(r).bytes for r in reqs]
    budget = budget_requests * max(need)
    server = serve.Server(budget_bytes=budget, chunk_steps=chunk, mixed=False, pinned_results=False)
    # a clock that advances 0.1 ms per reading: the interleaving of arrivals
    # and loop rounds is the same on every run
    now = [0.0]

    def clock():
        now[0] += 1e-4
        return now[0]

    recs = server.run(reqs, _workload, clock=clock)
    for r, rec in zip(reqs, recs):
        assert rec.finished is not None and rec.admitted is not None
        assert rec.admitted >= r.arrival - 1e-9
        assert np.all(rec.result == r.steps), (r.rid, rec.result, r.steps)
    assert 0 < server.peak_bytes <= budget
    assert all(b.closed for b in world.batches)
    assert all(ch["done"] for ch in world.chunks)
    # one chunk queued behind the running one, never more
    assert world.max_outstanding <= 1
    if budget_requests <= 3:
        # some request that had already arrived was admitted only once an
        # earlier one had finished and released its memory
        assert any(a.finished is not None and b.arrival < a.finished <= b.admitted
                   for a in recs for b in recs if a is not b)
