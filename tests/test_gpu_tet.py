"""GPU parity on tetrahedral meshes (Sec. 3.1 tetrahedral cells, Sec. 3.2
breadth-first downwind levels, Sec. 5.1 subdomains): the CUDA path through
the C ABI (kin_create_tet) against the FP64 oracle on the same seeded inputs,
f element by element at 1e-12 in FP64, W within 1e-5 in FP32."""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-5


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


def oracle_run(w, steps):
    P = oracle.tet_problem(w)
    T = oracle.TetMesh.from_workload(w)
    f = oracle.tet_init(P, T, w.W0)
    oracle.tet_step(P, T, f, steps)
    return f, oracle.tet_moments(P, T, f), oracle.tet_mass(P, T, oracle.tet_moments(P, T, f))


def gpu_run(kin, w, steps, precision):
    with kin.TetContext.from_workload(w, precision=precision) as ctx:
        ctx.set_state(np.ascontiguousarray(w.W0.reshape(-1)))
        ctx.step(steps)
        mass, _, _ = kin.kin_diag(ctx.ctx, w.m, defect=False)
        return ctx.get_state(), ctx.get_kinetic(), mass


CASES = [
    lambda: workloads.tet_advection(seed=0, n=4, tiles=2, velset=1, dt_mult=10.0, iters=3),
    lambda: workloads.tet_advection(seed=1, n=4, tiles=1, velset=0, dt_mult=6.0, iters=2),
    lambda: workloads.tet_densitywave(seed=2, n=4, tiles=2, velset=1, dt_mult=8.0, precision="f64"),
    lambda: workloads.tet_densitywave(seed=3, n=6, tiles=3, velset=0, dt_mult=5.0, iters=1, precision="f64"),
    lambda: workloads.tet_maxwell(seed=4, n=4, tiles=2, velset=0, dt_mult=6.0, sigma=1.5),
    lambda: workloads.tet_maxwell(seed=5, n=4, tiles=2, velset=1, dt_mult=6.0),
    lambda: workloads.with_(workloads.tet_densitywave(seed=6, n=4, tiles=2, velset=1, precision="f64"),
                            omega=1.7),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_fp64_matches_oracle(kin, case):
    w = CASES[case]()
    fo, Wo, mo = oracle_run(w, 4)
    W, f, mass = gpu_run(kin, w, 4, kin.KIN_FP64)
    assert np.abs(f - fo).max() / np.abs(fo).max() < TOL64
    assert np.abs(W - Wo).max() / np.abs(Wo).max() < TOL64
    assert np.abs(mass - mo).max() < 1e-12 * max(1.0, np.abs(mo).max())


@pytest.mark.parametrize("case", range(len(CASES)))
def test_fp32_matches_oracle(kin, case):
    w = CASES[case]()
    _, Wo, _ = oracle_run(w, 4)
    W, _, _ = gpu_run(kin, w, 4, kin.KIN_FP32)
    W, Wo = W.reshape(w.m, -1), Wo.reshape(w.m, -1)
    for v in range(w.m):
        scale = np.abs(Wo[v]).max()
        if scale == 0:
            continue
        assert np.abs(W[v] - Wo[v]).max() / scale < TOL32, v


def test_fp32_density_wave_50_steps(kin):
    # 8^3 cubes (3,072 tetrahedra), 2^3 subdomains, D3Q4, 50 steps
    w = workloads.tet_densitywave(seed=7, n=8, tiles=2, velset=1, dt_mult=5.0)
    fo, Wo, _ = oracle_run(w, 50)
    W, f, _ = gpu_run(kin, w, 50, kin.KIN_FP32)
    W, Wo = W.reshape(w.m, -1), Wo.reshape(w.m, -1)
    err = max(np.abs(W[v] - Wo[v]).max() / np.abs(Wo[v]).max() for v in range(w.m))
    print(f"\n[tet-parity] densitywave 8^3 cubes D3Q4 x 50 FP32: W_linf={err:.3e}")
    assert err < TOL32


def test_constant_state_and_repeatable(kin):
    w = workloads.tet_densitywave(seed=8, n=4, tiles=2, velset=1, dt_mult=10.0)
    W0 = w.W0.copy()
    W0[0] = 1.2
    W0[1:4] = np.array([0.3, -0.1, 0.2])[:, None]
    W0[4] = 2.9
    w = workloads.with_(w, W0=W0)
    for prec in (kin.KIN_FP64, kin.KIN_FP32):
        W, f1, _ = gpu_run(kin, w, 6, prec)
        _, f2, _ = gpu_run(kin, w, 6, prec)
        assert np.array_equal(f1, f2)
        tol = 1e-14 if prec == kin.KIN_FP64 else 1e-6
        assert np.abs(W - W0.reshape(-1)).max() / np.abs(W0).max() < tol


def test_bad_topology_is_rejected(kin):
    w = workloads.tet_advection(seed=0, n=3, tiles=1, velset=1)
    m = w.mesh
    nbr = m.nbr.copy()
    nbr[0, 0] = m.cells + 5
    with pytest.raises(kin.KinError) as ei:
        kin.TetContext(m.xyz, m.vid, nbr, w.subdomains(), m.wrap, w.system, kin.KIN_D3Q4, w.lam, w.dt)
    assert ei.value.status == kin.KIN_EINVAL
    # one subdomain around the periodic box without its wrap faces marked:
    # the oriented graph has cycles
    with pytest.raises(kin.KinError) as ei:
        kin.TetContext(m.xyz, m.vid, m.nbr, w.subdomains(), np.zeros_like(m.wrap), w.system, kin.KIN_D3Q4,
                       w.lam, w.dt)
    assert ei.value.status == kin.KIN_EINVAL and "cycle" in str(ei.value)


def test_async_host_copies(kin):
    # the asynchronous host copies on a tetrahedral context give what the
    # synchronous ones give
    import torch
    w = workloads.tet_densitywave(seed=14, n=4, tiles=2, velset=1, dt_mult=8.0)
    out = []
    for use_async in (False, True):
        with kin.TetContext.from_workload(w) as ctx:
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
