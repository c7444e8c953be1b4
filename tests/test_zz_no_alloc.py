"""kin_step_noalloc: the step without device allocation.

Callers whose device memory belongs to their own allocator or to a fixed
memory plan cannot let the library call cudaMalloc; this entry point keeps
its scratch in a static device array instead.  The test calls it through the
C ABI twice in a row, on two different problems (so the second call runs on
scratch left over from the first), and checks each result against the
context-based entry points (kin_create / kin_set_kinetic / kin_step /
kin_get_kinetic) on the same input, within the parity tolerances of the
other GPU tests.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

TOL = {"f32": 1e-5, "f64": 1e-12}


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


def _with_context(kin, w, steps):
    with kin.Context.from_workload(w) as ctx:
        ctx.set_state(np.ascontiguousarray(w.W0.reshape(-1)))
        f0 = ctx.get_kinetic()
        ctx.set_kinetic(f0)
        ctx.step(steps)
        return f0, ctx.get_kinetic()


def _noalloc(kin, w, f0, steps):
    import torch
    prec = kin.KIN_FP32 if w.precision == "f32" else kin.KIN_FP64
    mesh, model, opts = kin.make_args(w.dim, w.n, w.lo, w.hi, w.system, w.lam, omega=w.omega,
                                      gamma=w.gamma, adv=w.adv, tiles=w.tiles, iters=w.iters,
                                      precision=prec)
    fd = torch.from_numpy(f0.copy()).cuda()
    torch.cuda.synchronize()
    kin.kin_step_noalloc(mesh, model, w.degree, w.dt, opts, fd, steps)
    torch.cuda.synchronize()
    return fd.cpu().numpy()


def test_noalloc_matches_context_entry_points_two_calls(kin):
    import torch
    problems = [
        (workloads.with_(workloads.vortex2d(seed=11, n=64, degree=2, tiles=2, dt_mult=20.0),
                         tiles=(2, 2)), 4),
        (workloads.densitywave3d(seed=12, n=16, degree=1, tiles=2, dt_mult=20.0, precision="f64"), 3),
    ]
    before = torch.cuda.memory_allocated()
    for w, steps in problems:
        f0, want = _with_context(kin, w, steps)
        got = _noalloc(kin, w, f0, steps)
        rel = np.abs(got - want).max() / np.abs(want).max()
        assert rel < TOL[w.precision], (w.name, rel)
    assert torch.cuda.memory_allocated() == before


def test_noalloc_rejects_problems_beyond_its_scratch(kin):
    import torch
    w = workloads.densitywave3d(seed=0, n=64, degree=1, tiles=8)
    mesh, model, opts = kin.make_args(w.dim, w.n, w.lo, w.hi, w.system, w.lam, tiles=w.tiles,
                                      precision=kin.KIN_FP32)
    f = torch.zeros(8, device="cuda")
    with pytest.raises(kin.KinError) as ei:
        kin.kin_step_noalloc(mesh, model, w.degree, w.dt, opts, f, 1)
    assert ei.value.status == kin.KIN_EINVAL
    assert "limited to" in str(ei.value)
