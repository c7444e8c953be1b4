"""Multi-GPU runs are independent replicas (no data-path collective): the
bench's whole-job figures take the slowest rank's timed region and the units
of all ranks.  Checked here with two gloo ranks on the CPU."""
import importlib.util
import os
import socket

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=ws)
    try:
        # rank r was slower by r ms over 10 steps, each processing 1e6 units per step
        ms, value = _bench().replica_aggregate(20.0 + rank, 10, 1e6, device="cpu")
        out.put((rank, ms, value))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank_and_all_units():
    torch_mp = pytest.importorskip("torch.multiprocessing")
    ctx = torch_mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in res:
        assert ms == pytest.approx(2.1)                    # max(20, 21) ms / 10 steps
        assert value == pytest.approx(2 * 1e6 / 2.1e-3)    # both ranks' units over the slowest time


def test_single_process_is_local():
    ms, value = _bench().replica_aggregate(30.0, 10, 5e5, device="cpu")
    assert ms == pytest.approx(3.0) and value == pytest.approx(5e5 / 3e-3)
