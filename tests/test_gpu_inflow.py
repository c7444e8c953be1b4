"""GPU parity with inflow boundaries (non-periodic axes whose incoming
populations take the Maxwellian of a prescribed face state; the paper
prescribes the solution on the boundary, Sec. 6.2): the CUDA path through
the C ABI against the FP64 oracle on the same seeded inputs, for the generic
and the compile-time-shape kernels, walks that start at the boundary and
walks that start K subdomains upstream, and batches.  Tolerances as in the
periodic parity tests (FP64 1e-12, FP32 1e-5 relative)."""
import numpy as np
import pytest

import workloads
from tests.test_gpu_parity import TOL32, TOL64, gpu_run, kin, oracle_run, rel_errors  # noqa: F401

pytestmark = pytest.mark.gpu


def _euler_free_stream(dim, rho=1.0, u=1.0, p=1.0, gamma=1.4):
    W = [rho] + [rho * u] * dim + [p / (gamma - 1) + 0.5 * rho * dim * u * u]
    return np.array(W)


def _wb(m, faces):
    wb = np.zeros((3, 2, m))
    for (a, side), W in faces.items():
        wb[a, side, :] = W
    return wb


def _cases():
    adv = workloads.advection1d(seed=0, n=48, tiles=4, dt=0.1)
    adv = workloads.with_(adv, inflow=(1,), Wb=_wb(1, {(0, 0): [1.3], (0, 1): [0.7]}))
    ws = _euler_free_stream(2)
    v2 = workloads.vortex2d(seed=1, n=16, degree=2, tiles=2, dt_mult=40.0)
    v2 = workloads.with_(v2, inflow=(1, 0), Wb=_wb(4, {(0, 0): ws, (0, 1): 1.1 * ws}))
    v2b = workloads.with_(workloads.vortex2d(seed=2, n=16, degree=1, tiles=(4, 1), dt_mult=30.0, iters=2),
                          inflow=(1, 1), Wb=_wb(4, {(0, 0): ws, (0, 1): ws, (1, 0): ws, (1, 1): 0.9 * ws}))
    v3 = workloads.with_(workloads.vortex2d(seed=3, n=32, degree=3, tiles=2, dt_mult=30.0),
                         inflow=(0, 1), Wb=_wb(4, {(1, 0): ws, (1, 1): ws}))
    w3 = _euler_free_stream(3)
    d3 = workloads.with_(workloads.densitywave3d(seed=4, n=8, degree=1, tiles=2, dt_mult=30.0),
                         inflow=(1, 1, 1), Wb=_wb(5, {(a, s): w3 for a in range(3) for s in range(2)}))
    mx = workloads.with_(workloads.maxwell3d(seed=5, n=8, degree=1, tiles=2, dt_mult=20.0, sigma=2.0),
                         inflow=(1, 0, 1), Wb=np.zeros((3, 2, 6)))
    return [
        # (workload, block): generic shapes, then compiled fixed shapes (FP32)
        (adv, (4,)), (v2, (4, 8)), (v2b, (4, 4)), (d3, (2, 2, 4)), (mx, (2, 4, 2)),
        (v2, (8, 8)), (v3, (8, 8)), (d3, (4, 4, 4)), (mx, (4, 4, 4)),
    ]


CASES = _cases()


@pytest.mark.parametrize("case", range(len(CASES)))
def test_fp64_matches_oracle(kin, case):
    w, block = CASES[case]
    steps = 4
    W, f, _ = gpu_run(kin, w, steps, precision=kin.KIN_FP64, block=block)
    fo, Wo = oracle_run(w, steps)
    assert np.abs(f - fo).max() / np.abs(fo).max() < TOL64
    l2, linf = rel_errors(w, W, Wo)
    assert linf < TOL64 and l2 < TOL64, (l2, linf)


@pytest.mark.parametrize("case", range(len(CASES)))
def test_fp32_matches_oracle(kin, case):
    w, block = CASES[case]
    steps = 4
    with kin.Context.from_workload(w, precision=kin.KIN_FP32, block=block) as ctx:
        ctx.set_state(np.ascontiguousarray(w.W0.reshape(-1)))
        ctx.step(steps)
        W = ctx.get_state()
        fixed = ctx.info.specialised
    if w.dim >= 2 and block in ((8, 8), (4, 4, 4)):
        assert fixed == 1
    _, Wo = oracle_run(w, steps)
    l2, linf = rel_errors(w, W, Wo)
    assert l2 < TOL32 and linf < TOL32, (l2, linf)


def test_boundary_state_changes_the_result(kin):
    w, block = CASES[1]
    W1, _, _ = gpu_run(kin, w, 3, precision=kin.KIN_FP64, block=block)
    w2 = workloads.with_(w, Wb=1.2 * np.asarray(w.Wb))
    W2, _, _ = gpu_run(kin, w2, 3, precision=kin.KIN_FP64, block=block)
    Wp, _, _ = gpu_run(kin, workloads.with_(w, inflow=(0, 0), Wb=None), 3, precision=kin.KIN_FP64, block=block)
    assert np.abs(W1 - W2).max() > 1e-4 and np.abs(W1 - Wp).max() > 1e-4


def test_missing_boundary_state_and_bad_calls(kin):
    w, block = CASES[1]
    with kin.Context(w.dim, w.n, w.lo, w.hi, w.degree, w.system, w.lam, w.dt, omega=w.omega, gamma=w.gamma,
                     tiles=w.tiles, iters=w.iters, precision=kin.KIN_FP64, inflow=w.inflow) as ctx:
        ctx.set_state(np.ascontiguousarray(w.W0.reshape(-1)))
        ctx.set_boundary(0, 0, w.Wb[0, 0])
        with pytest.raises(kin.KinError) as ei:
            ctx.step(1)                             # the upper x face has no state
        assert ei.value.status == kin.KIN_ESTATE
        for bad in ((1, 0, w.Wb[0, 0]), (0, 2, w.Wb[0, 0]), (0, 1, w.Wb[0, 0][:3]),
                    (0, 1, np.array([0.0, 1.0, 1.0, 3.0]))):
            with pytest.raises(kin.KinError) as ei:
                ctx.set_boundary(*bad)              # periodic axis, bad side, wrong m, rho = 0
            assert ei.value.status == kin.KIN_EINVAL
        ctx.set_boundary(0, 1, w.Wb[0, 1])
        ctx.step(2)
        with pytest.raises(kin.KinError) as ei:
            kin.kin_diag(ctx.ctx, 4)                # the interface defect needs periodic axes
        assert ei.value.status == kin.KIN_EINVAL
        mass, _, _ = kin.kin_diag(ctx.ctx, 4, defect=False)
        assert np.all(np.isfinite(mass))


def test_batch_with_inflow_members_equals_alone(kin):
    picks = [CASES[i] for i in (1, 2, 6, 7, 8)]
    alone, ctxs = [], []
    for w, block in picks:
        with kin.Context.from_workload(w, precision=kin.KIN_FP32, block=block) as c:
            c.set_state(np.ascontiguousarray(w.W0.reshape(-1)))
            c.step(3)
            alone.append(c.get_kinetic())
        c = kin.Context.from_workload(w, precision=kin.KIN_FP32, block=block)
        c.set_state(np.ascontiguousarray(w.W0.reshape(-1)))
        ctxs.append(c)
    try:
        with kin.Batch(ctxs) as batch:
            batch.step(3)
            batch.sync()
        for c, want in zip(ctxs, alone):
            assert np.array_equal(c.get_kinetic(), want)
    finally:
        for c in ctxs:
            c.close()


def _plane_wave(x, t):
    # E_z = cos(2 pi (x - t)), H_y = -E_z: a wave moving along +x (Sec. 6.2 form)
    W = np.zeros((6,) + np.shape(x))
    W[2] = np.cos(2 * np.pi * (x - t))
    W[4] = -W[2]
    return W


@pytest.mark.parametrize("precision,tol", [("f64", TOL64), ("f32", TOL32)])
def test_plane_wave_with_exact_dirichlet_data_matches_oracle(kin, precision, tol):
    # non-periodic x with the exact solution imposed on both x faces at every
    # step's midpoint (boundary states set before each step), periodic y, z
    import oracle
    w = workloads.maxwell3d(seed=6, n=8, degree=2, tiles=2, dt_mult=3.0, precision=precision)
    w = workloads.with_(w, n=(16, 2, 2), tiles=(4, 1, 1), inflow=(1, 0, 0), Wb=np.zeros((3, 2, 6)))
    P = oracle.Problem(**w.oracle_kwargs())
    x = oracle.node_coords(P)[:, 0]
    W0 = _plane_wave(x, 0.0)
    steps = 6
    pr = kin.KIN_FP64 if precision == "f64" else kin.KIN_FP32
    with kin.Context.from_workload(workloads.with_(w, W0=W0), precision=pr) as ctx:
        ctx.set_state(np.ascontiguousarray(W0.reshape(-1)))
        fo = oracle.init(P, W0)
        for s in range(steps):
            tm = (s + 0.5) * w.dt
            wb = np.zeros((3, 2, 6))
            wb[0, 0], wb[0, 1] = _plane_wave(0.0, tm), _plane_wave(1.0, tm)
            ctx.set_boundary(0, 0, wb[0, 0])
            ctx.set_boundary(0, 1, wb[0, 1])
            ctx.step(1)
            P.Wb = wb
            oracle.step(P, fo, 1)
        W = ctx.get_state()
    Wo = oracle.moments(P, fo)
    # E_x, E_y, H_x, H_z stay zero up to round-off, so the error is taken
    # relative to the largest field value rather than per variable
    err = np.abs(W - Wo).max() / np.abs(Wo).max()
    assert err < tol, err
    # and the result is the travelling wave (the scheme's error, not round-off)
    assert np.abs(W.reshape(6, -1) - _plane_wave(x, steps * w.dt)).max() < 0.1
