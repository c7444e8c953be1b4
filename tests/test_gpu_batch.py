"""Batches of independent problems: one launch per kernel type per step over
every member's tiles must give exactly the result of stepping each member
alone (same per-tile arithmetic), for uneven mesh sizes and degrees."""
import numpy as np
import pytest

import workloads
from tests.test_gpu_parity import TOL32, oracle_run, rel_errors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kin():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_11010_gb300 import build
    build.build()
    import paper_2212_11010_gb300 as kin
    kin.load_library()
    return kin


def _mix():
    # uneven 2D Euler problems (degrees 1..3, n 32..128, 32-cell subdomains),
    # plus members without a fixed-shape kernel (3D, FP64 p = 1, odd block)
    # and Maxwell members with and without one
    ws = [workloads.vortex2d(seed=1, n=64, degree=2, tiles=2, dt_mult=6.0),
          workloads.densitywave2d(seed=2, n=32, degree=1, tiles=1, dt_mult=3.0),
          workloads.vortex2d(seed=3, n=128, degree=3, tiles=4, dt_mult=7.0),
          workloads.vortex2d(seed=4, n=96, degree=2, tiles=3, dt_mult=2.0),
          workloads.densitywave2d(seed=5, n=64, degree=1, tiles=2, dt_mult=8.0),
          workloads.densitywave3d(seed=6, n=16, degree=1, tiles=2, dt_mult=5.0),
          workloads.vortex2d(seed=7, n=32, degree=1, tiles=1, dt_mult=4.0, precision="f64"),
          workloads.maxwell3d(seed=8, n=16, degree=1, tiles=2, dt_mult=6.0, sigma=2.0),
          workloads.maxwell3d(seed=9, n=8, degree=2, tiles=1, dt_mult=4.0, sigma=0.5)]
    blocks = [None, None, None, None, (16, 4), None, None, None, None]
    return ws, blocks


def _ctx(kin, w, block):
    kw = {} if block is None else {"block": block}
    c = kin.Context.from_workload(w, **kw)
    c.set_state(np.ascontiguousarray(w.W0.reshape(-1)))
    return c


def test_batch_equals_members_alone(kin):
    ws, blocks = _mix()
    alone = []
    for w, b in zip(ws, blocks):
        with _ctx(kin, w, b) as c:
            c.step(5)
            alone.append(c.get_kinetic())
    ctxs = [_ctx(kin, w, b) for w, b in zip(ws, blocks)]
    assert any(c.info.specialised == 0 for c in ctxs) and any(c.info.specialised for c in ctxs)
    with kin.Batch(ctxs) as batch:
        batch.step(2)
        batch.step(3)          # odd count: summary parity flips
        batch.sync()
    for c, want in zip(ctxs, alone):
        assert np.array_equal(c.get_kinetic(), want)
        assert kin.kin_query(c.ctx).steps_done == 5
    for c in ctxs:
        c.close()


def test_direct_batch_equals_graph_batch(kin):
    """Direct launches per step (no CUDA graphs) give the graph-replay result."""
    ws, blocks = _mix()
    res = []
    for graphs in (True, False):
        ctxs = [_ctx(kin, w, b) for w, b in zip(ws, blocks)]
        with kin.Batch(ctxs, graphs=graphs) as batch:
            batch.step(3)
            batch.step(2)
            batch.sync()
        res.append([c.get_kinetic() for c in ctxs])
        for c in ctxs:
            c.close()
    for a, b in zip(*res):
        assert np.array_equal(a, b)


def test_batch_members_with_different_parity_and_oracle(kin):
    ws, blocks = _mix()
    ws, blocks = ws[:3], blocks[:3]
    ctxs = [_ctx(kin, w, b) for w, b in zip(ws, blocks)]
    ctxs[1].step(1)            # one member starts a step ahead
    with kin.Batch(ctxs) as batch:
        batch.step(3)
        batch.sync()
    for i, (c, w) in enumerate(zip(ctxs, ws)):
        steps = 3 + (1 if i == 1 else 0)
        W = c.get_state()
        _, Wo = oracle_run(w, steps)
        l2, linf = rel_errors(w, W, Wo)
        assert l2 < TOL32 and linf < TOL32, (i, l2, linf)
        c.close()


def test_stepping_a_member_alone_invalidates_batch(kin):
    ws, blocks = _mix()
    ctxs = [_ctx(kin, w, b) for w, b in zip(ws[:2], blocks[:2])]
    batch = kin.Batch(ctxs)
    batch.step(1)
    ctxs[0].step(1)
    with pytest.raises(kin.KinError) as ei:
        batch.step(1)
    assert ei.value.status == kin.KIN_ESTATE
    batch.close()
    with pytest.raises(kin.KinError) as ei:
        kin.kin_batch_create([ctxs[0].ctx, ctxs[0].ctx])
    assert ei.value.status == kin.KIN_EINVAL
    for c in ctxs:
        c.close()


def test_set_kinetic_keeps_a_member_in_its_batch(kin):
    """Setting a member's kinetic state (checkpoint resume, or fresh client
    data) between batch steps keeps the batch valid: the state's block
    summaries are rebuilt in place, and the run equals the member alone."""
    ws, blocks = _mix()
    ws, blocks = ws[:2], blocks[:2]
    alone = []
    for w, b in zip(ws, blocks):
        with _ctx(kin, w, b) as c:
            c.step(5)
            alone.append(c.get_kinetic())
    ctxs = [_ctx(kin, w, b) for w, b in zip(ws, blocks)]
    with kin.Batch(ctxs) as batch:
        batch.step(2)
        batch.sync()
        for c in ctxs:
            c.set_kinetic(c.get_kinetic())     # host round trip of f
        batch.step(3)
        batch.sync()
    for c, want in zip(ctxs, alone):
        assert np.array_equal(c.get_kinetic(), want)
        c.close()


def test_mixed_degrees_share_one_launch(kin):
    """With the mixed schedule, 2D Euler FP32 members of degrees 1, 2, 3 and
    different mesh sizes, with the default cell blocks, advance in one launch
    per batch step; the result equals each member alone and the
    per-kernel-type batch, bitwise."""
    ws = [workloads.vortex2d(seed=11, n=64, degree=1, tiles=2, dt_mult=5.0),
          workloads.densitywave2d(seed=12, n=96, degree=2, tiles=3, dt_mult=3.0),
          workloads.vortex2d(seed=13, n=128, degree=3, tiles=4, dt_mult=6.0),
          workloads.densitywave2d(seed=14, n=32, degree=3, tiles=1, dt_mult=8.0),
          workloads.vortex2d(seed=15, n=32, degree=2, tiles=1, dt_mult=2.0)]
    alone = []
    for w in ws:
        with _ctx(kin, w, None) as c:
            c.step(5)
            alone.append(c.get_kinetic())
    res = {}
    for mixed in (True, False):
        ctxs = [_ctx(kin, w, None) for w in ws]
        with kin.Batch(ctxs, mixed=mixed) as batch:
            if mixed:
                assert batch.launches_per_step == 1 and batch.mixed_members == len(ws)
            else:
                assert batch.launches_per_step == 3 and batch.mixed_members == 0
            batch.step(2)
            batch.step(3)
            batch.sync()
        res[mixed] = [c.get_kinetic() for c in ctxs]
        for c in ctxs:
            c.close()
    for a, b, want in zip(res[True], res[False], alone):
        assert np.array_equal(a, want)
        assert np.array_equal(b, want)


def test_async_host_copies_pipeline_equals_synchronous(kin):
    # the pipelined host round trip of the e2e measurement (each member's
    # result copied out on one stream, its next input in on another, ordered
    # per member by an event) gives bitwise the synchronous round trip
    import torch
    ws, blocks = _mix()
    ws, blocks = ws[:5], blocks[:5]
    steps = 3

    def run(pipelined):
        ctxs = [_ctx(kin, w, b) for w, b in zip(ws, blocks)]
        dt = lambda c: torch.float32 if c.info.precision == kin.KIN_FP32 else torch.float64
        fh = [torch.empty(c.info.kinetic_values, dtype=dt(c), pin_memory=True) for c in ctxs]
        for c, h in zip(ctxs, fh):
            kin.kin_get_kinetic(c.ctx, h.numpy())
        stream = torch.cuda.Stream()
        with kin.Batch(ctxs, stream=stream.cuda_stream) as b:
            if pipelined:
                s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
                left = [torch.cuda.Event() for _ in ctxs]
                arrived, stepped = torch.cuda.Event(), torch.cuda.Event()
                for _ in range(steps):
                    for c, h, ev in zip(ctxs, fh, left):
                        s_in.wait_event(ev)
                        kin.kin_set_kinetic_async(c.ctx, h, s_in.cuda_stream)
                    arrived.record(s_in)
                    stream.wait_event(arrived)
                    b.step(1)
                    stepped.record(stream)
                    s_out.wait_event(stepped)
                    for c, h, ev in zip(ctxs, fh, left):
                        kin.kin_get_kinetic_async(c.ctx, h, s_out.cuda_stream)
                        ev.record(s_out)
                torch.cuda.synchronize()
            else:
                for _ in range(steps):
                    for c, h in zip(ctxs, fh):
                        kin.kin_set_kinetic(c.ctx, h.numpy())
                    b.step(1)
                    b.sync()
                    for c, h in zip(ctxs, fh):
                        kin.kin_get_kinetic(c.ctx, h.numpy())
        out = [h.numpy().copy() for h in fh]
        for c in ctxs:
            c.close()
        return out

    a, p = run(False), run(True)
    for x, y in zip(a, p):
        assert np.array_equal(x, y)
    with _ctx(kin, ws[0], blocks[0]) as c:
        with pytest.raises(ValueError):
            kin.kin_set_kinetic_async(c.ctx, np.zeros(c.info.kinetic_values, dtype=np.float32))
        h = torch.empty(3, dtype=torch.float32, pin_memory=True)
        with pytest.raises(kin.KinError) as ei:
            kin.kin_get_kinetic_async(c.ctx, h)
        assert ei.value.status == kin.KIN_EINVAL


def test_async_set_then_step_equals_synchronous(kin):
    # a context stepped alone after kin_set_kinetic_async computes the
    # deferred interface summaries itself: the same state as after the
    # synchronous kin_set_kinetic, bitwise; the defect diagnostic too
    import torch
    w = workloads.vortex2d(seed=11, n=64, degree=2, tiles=2, dt_mult=6.0)
    out = []
    for use_async in (False, True):
        with _ctx(kin, w, None) as c:
            c.step(2)
            h = torch.empty(c.info.kinetic_values, dtype=torch.float32, pin_memory=True)
            kin.kin_get_kinetic(c.ctx, h.numpy())
            if use_async:
                kin.kin_set_kinetic_async(c.ctx, h)
                torch.cuda.synchronize()
            else:
                kin.kin_set_kinetic(c.ctx, h.numpy())
            _, dfc, _ = c.diag()
            c.step(3)
            out.append((c.get_kinetic(), dfc))
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])


def test_lazy_ordering_across_batches_and_a_shared_stream(kin):
    """Members sharing one stream, stepped by a batch on one stream and then,
    with nothing synchronised, by a new batch of the same members on another:
    the second batch is ordered after the first through the members' events,
    and a member's own later calls (a step, a read) wait for the second."""
    import torch
    ws, blocks = _mix()
    ws, blocks = ws[:5], blocks[:5]
    alone = []
    for w, b in zip(ws, blocks):
        with _ctx(kin, w, b) as c:
            c.step(8)
            alone.append(c.get_kinetic())
    shared = torch.cuda.Stream()
    ctxs = []
    for w, b in zip(ws, blocks):
        kw = {} if b is None else {"block": b}
        c = kin.Context.from_workload(w, stream=shared.cuda_stream, **kw)
        c.set_state(np.ascontiguousarray(w.W0.reshape(-1)))
        ctxs.append(c)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    b1 = kin.Batch(ctxs, stream=s1.cuda_stream, graphs=False)
    b1.step(4)
    b2 = kin.Batch(ctxs, stream=s2.cuda_stream)
    b2.step(3)
    ctxs[0].step(1)                      # on the shared stream, after the second batch
    for i, (c, want) in enumerate(zip(ctxs, alone)):
        if i > 0:
            c.step(1)
        assert np.array_equal(c.get_kinetic(), want), i
        assert kin.kin_query(c.ctx).steps_done == 8
    b2.sync()
    b1.close()
    b2.close()
    for c in ctxs:
        c.close()
