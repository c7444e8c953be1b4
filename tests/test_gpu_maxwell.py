"""GPU parity for Maxwell's equations (Sec. 6.1.1) with a uniform
conductivity (Sec. 6.4): the CUDA path through the C ABI against the FP64
oracle on the same seeded plane waves, plus the closed form of a uniform
field (E multiplied by mu = (1 - sigma dt / 2) / (1 + sigma dt / 2) per
step, H unchanged), which the GPU has to reach without the oracle.

Tolerances as in the Euler parity tests: FP64 1e-12 and FP32 1e-5 relative
(GLL-weighted L2 and max norm per variable, relative to the oracle's norm).
"""
import numpy as np
import pytest

import oracle
import workloads
from tests.test_gpu_parity import TOL32, TOL64, gpu_run, kin, oracle_run, rel_errors  # noqa: F401

pytestmark = pytest.mark.gpu

CASES = [
    # (workload, block)
    (lambda: workloads.maxwell3d(seed=0, n=8, degree=1, tiles=2, dt_mult=30.0), (2, 2, 4)),
    (lambda: workloads.maxwell3d(seed=1, n=8, degree=1, tiles=(2, 1, 2), dt_mult=20.0, sigma=4.0), (4, 4, 2)),
    (lambda: workloads.maxwell3d(seed=2, n=6, degree=2, tiles=(3, 1, 2), dt_mult=20.0, sigma=1.0,
                                 omega=1.7), (1, 3, 3)),
    (lambda: workloads.maxwell3d(seed=3, n=4, degree=3, tiles=(1, 2, 1), dt_mult=15.0, sigma=25.0,
                                 iters=2), (2, 2, 2)),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_fp64_matches_oracle(kin, case):
    make, block = CASES[case]
    w = make()
    steps = 4
    W, f, _ = gpu_run(kin, w, steps, precision=kin.KIN_FP64, block=block)
    fo, Wo = oracle_run(w, steps)
    assert np.abs(f - fo).max() / np.abs(fo).max() < TOL64
    l2, linf = rel_errors(w, W, Wo)
    assert linf < TOL64 and l2 < TOL64, (l2, linf)


@pytest.mark.parametrize("case", range(len(CASES)))
def test_fp32_matches_oracle(kin, case):
    make, block = CASES[case]
    w = make()
    steps = 4
    W, _, _ = gpu_run(kin, w, steps, precision=kin.KIN_FP32, block=block)
    _, Wo = oracle_run(w, steps)
    l2, linf = rel_errors(w, W, Wo)
    assert l2 < TOL32 and linf < TOL32, (l2, linf)


def test_conductivity_changes_the_result(kin):
    # sigma enters the kernel: sigma = 0 and sigma = 4 differ well above round-off
    make, block = CASES[1]
    w = make()
    W1, _, _ = gpu_run(kin, w, 3, precision=kin.KIN_FP64, block=block)
    W0, _, _ = gpu_run(kin, workloads.with_(w, sigma=0.0), 3, precision=kin.KIN_FP64, block=block)
    assert np.abs(W1 - W0).max() > 1e-3


@pytest.mark.parametrize("precision,tol", [("f64", 1e-13), ("f32", 2e-6)])
def test_uniform_field_decays_by_mu_per_step(kin, precision, tol):
    sigma, steps = 6.0, 7
    w = workloads.maxwell3d(seed=4, n=8, degree=2, tiles=2, dt_mult=10.0, sigma=sigma, precision=precision)
    E, H = np.array([0.3, -1.2, 0.7]), np.array([1.1, 0.4, -0.5])
    W0 = np.concatenate([np.repeat(E[:, None], w.W0.shape[1], 1), np.repeat(H[:, None], w.W0.shape[1], 1)])
    w = workloads.with_(w, W0=W0)
    pr = kin.KIN_FP64 if precision == "f64" else kin.KIN_FP32
    W, _, _ = gpu_run(kin, w, steps, precision=pr, block=(2, 2, 2))
    W = W.reshape(6, -1)
    mu = (1 - 0.5 * sigma * w.dt) / (1 + 0.5 * sigma * w.dt)
    assert np.abs(W[:3] - mu ** steps * E[:, None]).max() < tol
    assert np.abs(W[3:] - H[:, None]).max() < tol


def test_plane_waves_converge_to_the_exact_solution(kin):
    # sigma = 0: the GPU result approaches the translated plane waves; the
    # error falls by more than 3x when the mesh is refined at a fixed CFL-like
    # ratio (p = 2)
    errs = []
    for n in (8, 16):
        w = workloads.maxwell3d(seed=5, n=n, degree=2, tiles=2, dt_mult=2.0, precision="f64")
        steps = n // 2
        W, _, _ = gpu_run(kin, w, steps, precision=kin.KIN_FP64)
        ex = w.exact(steps * w.dt)
        errs.append(np.abs(W.reshape(6, -1) - ex).max())
    assert errs[1] < errs[0] / 3, errs
