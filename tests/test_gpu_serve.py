"""Continuous batching: requests arriving while others run are admitted as
memory allows, share kin_batch steps, and each result equals the same
request run alone (the batched arithmetic is the single-problem one)."""
import numpy as np
import pytest

import workloads

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


def test_served_results_equal_alone(kin):
    from paper_2212_11010_gb300 import serve
    reqs = workloads.serving_stream(seed=3, count=10, rate=4000.0, sizes=(32, 64), steps=(5, 30))
    need = [serve.state_bytes_estimate(workloads.request_workload(r)) for r in reqs]
    # a budget that holds the two largest requests but not all ten: the
    # arrivals (0.25 ms apart on average) come faster than requests finish, so
    # admission has to wait for memory to free up
    budget = 2.0 * max(need)
    assert sum(need) > budget
    server = serve.Server(budget_bytes=budget, chunk_steps=7)
    recs = server.run(reqs, workloads.request_workload)
    assert all(r.finished is not None and r.latency > 0 for r in recs)
    # the resident device bytes never exceeded the budget
    assert 0 < server.peak_bytes <= budget
    # some request that had already arrived was admitted only once an earlier
    # one had finished and released its memory
    waited = [b for b in recs
              if any(a.finished is not None and b.arrival < a.finished <= b.admitted for a in recs if a is not b)]
    assert waited, [(r.arrival, r.admitted, r.finished) for r in recs]
    for r, rec in zip(reqs, recs):
        w = workloads.request_workload(r)
        with kin.Context.from_workload(w, precision=kin.KIN_FP32) as ctx:
            ctx.set_state(np.ascontiguousarray(w.W0.reshape(-1)))
            ctx.step(r.steps)
            alone = ctx.get_state()
        assert np.array_equal(rec.result, alone), r.rid
    stats = serve.summarize(recs)
    assert stats["p99_s"] >= stats["p50_s"] > 0 and stats["dof_updates_per_s"] > 0


def test_requests_overlap_on_the_device(kin):
    # with a large budget several requests are in flight at once
    from paper_2212_11010_gb300 import serve
    reqs = workloads.serving_stream(seed=4, count=8, rate=2000.0, sizes=(64,), steps=(40, 60))
    recs = serve.Server(budget_bytes=1e9, chunk_steps=10).run(reqs, workloads.request_workload)
    spans = sorted((r.admitted, r.finished) for r in recs)
    overlaps = sum(1 for a, b in zip(spans, spans[1:]) if b[0] < a[1])
    assert overlaps >= 1
