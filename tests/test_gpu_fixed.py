"""GPU parity of the compile-time block-shape kernels: every compiled shape
against the FP64 oracle and against the generic kernel on the same block."""
import numpy as np
import pytest

import oracle
import workloads
from tests.test_gpu_parity import TOL32, TOL64, oracle_run, rel_errors

pytestmark = pytest.mark.gpu

# (dim, degree, precision, block) of every compiled fixed shape
SHAPES = [
    (2, 1, "f32", (16, 8)), (2, 1, "f32", (16, 16)), (2, 2, "f32", (8, 8)), (2, 3, "f32", (8, 4)),
    (2, 3, "f32", (8, 8)), (2, 2, "f64", (8, 8)),
    (3, 1, "f32", (8, 2, 2)), (3, 1, "f32", (4, 4, 2)), (3, 1, "f32", (8, 4, 2)), (3, 1, "f32", (4, 4, 4)),
    (3, 1, "f32", (4, 4, 2), "maxwell"), (3, 1, "f32", (8, 2, 2), "maxwell"),
    (3, 1, "f32", (4, 2, 2), "maxwell"), (3, 1, "f32", (8, 4, 2), "maxwell"), (3, 1, "f32", (4, 4, 4), "maxwell"),
]


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


def _problem(dim, degree, prec, block, system="euler"):
    if system == "maxwell":
        w = workloads.maxwell3d(seed=6, n=16, degree=degree, tiles=2, dt_mult=30.0, sigma=3.0, omega=1.8,
                                precision=prec)
        return workloads.with_(w, tiles=(2, 2, 2))
    if dim == 2:
        n = 2 * max(block) * 2
        w = workloads.vortex2d(seed=5, n=n, degree=degree, tiles=2, dt_mult=40.0, precision=prec)
        return workloads.with_(w, tiles=(2, 2))
    w = workloads.densitywave3d(seed=6, n=16, degree=degree, tiles=2, dt_mult=30.0, precision=prec)
    return workloads.with_(w, tiles=(2, 2, 2))


def _run(kin, w, block, steps, threads=0, stages=0):
    with kin.Context.from_workload(w, block=block, threads=threads, stages=stages) as ctx:
        ctx.set_state(np.ascontiguousarray(w.W0.reshape(-1)))
        ctx.step(steps)
        return ctx.get_state(), ctx.get_kinetic(), ctx.info


@pytest.mark.parametrize("shape", SHAPES, ids=[str(s) for s in SHAPES])
def test_fixed_shape_matches_oracle_and_generic(kin, shape):
    dim, degree, prec, block = shape[:4]
    w = _problem(*shape)
    steps = 4
    W, f, info = _run(kin, w, block, steps)
    assert info.specialised == 1 and tuple(info.block[:dim]) == tuple(block)
    _, Wo = oracle_run(w, steps)
    l2, linf = rel_errors(w, W, Wo)
    tol = TOL32 if prec == "f32" else TOL64
    assert l2 < tol and linf < tol, (l2, linf)
    # the generic kernel on the same block (a different thread count forces it).
    # The two evaluate the same formulas with different FMA contractions and
    # (in FP32) packed pair arithmetic, so they agree to a few dozen ulp after
    # four steps, not bit for bit.
    Wg, fg, infog = _run(kin, w, block, steps, threads=256 if info.threads != 256 else 128)
    assert infog.specialised == 0
    assert np.abs(f - fg).max() / np.abs(fg).max() < (5e-6 if prec == "f32" else 1e-14)


def test_default_block_uses_fixed_kernel_for_benchmarked_workload(kin):
    w = workloads.with_(workloads.vortex2d(seed=0), tiles=(8, 8))
    with kin.Context.from_workload(w) as ctx:
        assert ctx.info.specialised == 1
        assert tuple(ctx.info.block[:2]) == (8, 8)


TWO_BUFFER = [(2, 2, "f32", (8, 8)), (2, 1, "f32", (16, 8)), (3, 1, "f32", (4, 4, 2))]


@pytest.mark.parametrize("shape", TWO_BUFFER, ids=[str(s) for s in TWO_BUFFER])
def test_two_buffer_schedule_is_bitwise_identical(kin, shape):
    """The two-buffer schedule changes only when tiles are loaded, not what
    any thread computes: the state after several steps is bit for bit the
    one-buffer result."""
    dim, degree, prec, block = shape
    w = _problem(dim, degree, prec, block)
    _, f1, i1 = _run(kin, w, block, 3, stages=1)
    _, f2, i2 = _run(kin, w, block, 3, stages=2)
    assert (i1.stages, i2.stages) == (1, 2) and i1.specialised == 1 and i2.specialised == 1
    assert np.array_equal(f1, f2)
