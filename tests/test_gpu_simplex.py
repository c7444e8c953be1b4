"""GPU parity for the paper's d + 1 velocity sets (D2Q3, Sec. 2.4; D3Q4,
Sec. 6.1.3): diagonal velocities, anti-diagonal wavefront sweeps and
corner-sharing subdomains, against the FP64 oracle."""
import numpy as np
import pytest

import oracle
import workloads
from tests.test_gpu_parity import TOL32, TOL64, oracle_run, rel_errors

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


CASES = [
    lambda prec: workloads.with_(workloads.densitywave2d(seed=1, n=16, degree=2, tiles=2, dt_mult=20.0,
                                                         velset=1, precision=prec), tiles=(2, 2)),
    lambda prec: workloads.with_(workloads.densitywave2d(seed=2, n=12, degree=1, tiles=1, dt_mult=30.0,
                                                         velset=1, precision=prec), tiles=(3, 2), iters=2),
    lambda prec: workloads.with_(workloads.densitywave2d(seed=3, n=8, degree=3, tiles=2, dt_mult=10.0,
                                                         velset=1, precision=prec), tiles=(2, 1), iters=1),
    lambda prec: workloads.with_(workloads.densitywave3d(seed=4, n=8, degree=1, tiles=2, dt_mult=20.0,
                                                         velset=1, precision=prec), tiles=(2, 2, 2)),
    lambda prec: workloads.with_(workloads.densitywave3d(seed=5, n=4, degree=2, tiles=1, dt_mult=10.0,
                                                         velset=1, precision=prec), tiles=(1, 2, 1)),
]


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_simplex_sets_match_oracle(kin, case, prec):
    w = CASES[case](prec)
    steps = 4
    with kin.Context.from_workload(w) as ctx:
        assert ctx.info.nvel == w.dim + 1
        ctx.set_state(np.ascontiguousarray(w.W0.reshape(-1)))
        ctx.step(steps)
        W = ctx.get_state()
        mass = ctx.diag()[0]
    _, Wo = oracle_run(w, steps)
    l2, linf = rel_errors(w, W, Wo)
    tol = TOL64 if prec == "f64" else TOL32
    assert l2 < tol and linf < tol, (l2, linf)
    P = oracle.Problem(**w.oracle_kwargs())
    mo = oracle.mass(P, Wo)
    np.testing.assert_allclose(mass, mo, rtol=tol * 10, atol=tol * 10)


# Launch shapes of the streaming sweep: many (variable, subdomain) problems
# per thread block (more problems than one resident wave of blocks), columns
# spread over several warps (the transverse exchange crosses warps), column
# counts that are not a multiple of 32, a 2D subdomain wider than it is high.
STREAM_CASES = [
    lambda prec: workloads.with_(workloads.densitywave3d(seed=6, n=16, degree=1, tiles=8, dt_mult=20.0,
                                                         velset=1, precision=prec), tiles=(8, 8, 8)),
    lambda prec: workloads.with_(workloads.densitywave3d(seed=7, n=16, degree=1, tiles=2, dt_mult=20.0,
                                                         velset=1, precision=prec), tiles=(2, 2, 2)),
    lambda prec: workloads.with_(workloads.densitywave3d(seed=8, n=24, degree=1, tiles=2, dt_mult=15.0,
                                                         velset=1, precision=prec), tiles=(2, 3, 4)),
    lambda prec: workloads.with_(workloads.densitywave2d(seed=9, n=128, degree=2, tiles=32, dt_mult=20.0,
                                                         velset=1, precision=prec), tiles=(32, 32)),
    lambda prec: workloads.with_(workloads.densitywave2d(seed=10, n=64, degree=2, tiles=1, dt_mult=20.0,
                                                         velset=1, precision=prec), tiles=(1, 2)),
    lambda prec: workloads.with_(workloads.densitywave2d(seed=11, n=48, degree=3, tiles=1, dt_mult=10.0,
                                                         velset=1, precision=prec), tiles=(3, 1), iters=2),
]


@pytest.mark.parametrize("case", range(len(STREAM_CASES)))
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_simplex_stream_shapes_match_oracle(kin, case, prec):
    w = STREAM_CASES[case](prec)
    steps = 3
    with kin.Context.from_workload(w) as ctx:
        ctx.set_state(np.ascontiguousarray(w.W0.reshape(-1)))
        ctx.step(steps)
        W = ctx.get_state()
        f = ctx.get_kinetic()
    P = oracle.Problem(**w.oracle_kwargs())
    fo = oracle.init(P, w.W0)
    oracle.step(P, fo, steps)
    Wo = oracle.moments(P, fo)
    l2, linf = rel_errors(w, W, Wo)
    tol = TOL64 if prec == "f64" else TOL32
    assert l2 < tol and linf < tol, (l2, linf)
    f = f.reshape(w.npop, -1)
    fo = fo.reshape(w.npop, -1)
    fe = max(np.abs(f[k] - fo[k]).max() / np.abs(fo[k]).max() for k in range(w.npop))
    assert fe < (TOL64 if prec == "f64" else 5 * TOL32), fe


def test_simplex_errors(kin):
    w = workloads.densitywave3d(seed=1, n=64, degree=1, tiles=1, velset=1)
    with pytest.raises(kin.KinError) as ei:
        kin.Context.from_workload(w)          # 64 x 64 columns per subdomain: more than 1024 lanes
    assert ei.value.status == kin.KIN_EINVAL
    w = workloads.with_(workloads.densitywave2d(seed=1, n=16, degree=1, tiles=2, velset=1), tiles=(2, 2))
    with kin.Context.from_workload(w) as ctx:
        ctx.set_state(np.ascontiguousarray(w.W0.reshape(-1)))
        with pytest.raises(kin.KinError) as ei:
            kin.kin_batch_create([ctx.ctx])
        assert ei.value.status == kin.KIN_EINVAL


def test_async_host_copies(kin):
    # kin_set_kinetic_async / kin_get_kinetic_async on a d + 1 context give
    # what the synchronous copies give (no interface summaries to defer here)
    import torch
    w = workloads.with_(workloads.densitywave2d(seed=13, n=16, degree=2, tiles=2, dt_mult=20.0, velset=1,
                                                precision="f32"), tiles=(2, 2))
    out = []
    for use_async in (False, True):
        with kin.Context.from_workload(w) as ctx:
            ctx.set_state(np.ascontiguousarray(w.W0.reshape(-1)))
            ctx.step(2)
            h = torch.empty(ctx.info.kinetic_values, dtype=torch.float32, pin_memory=True)
            if use_async:
                kin.kin_get_kinetic_async(ctx.ctx, h)
                torch.cuda.synchronize()
                kin.kin_set_kinetic_async(ctx.ctx, h)
                torch.cuda.synchronize()
            else:
                kin.kin_get_kinetic(ctx.ctx, h.numpy())
                kin.kin_set_kinetic(ctx.ctx, h.numpy())
            ctx.step(2)
            out.append(ctx.get_kinetic())
    assert np.array_equal(out[0], out[1])
