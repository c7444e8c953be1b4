"""GPU parity on non-cubic meshes: unequal cell counts and box lengths per
axis (so h_a and the per-axis block-inverse coefficients differ), unequal
subdomain counts, for advection, Euler and Maxwell, against the FP64 oracle.
The error is taken relative to the largest value of all variables (some
Maxwell components stay at round-off level)."""
import numpy as np
import pytest

import oracle
from tests.test_gpu_parity import kin  # noqa: F401

pytestmark = pytest.mark.gpu

A, E, MX = oracle.ADVECTION, oracle.EULER, oracle.MAXWELL
CASES = [
    (2, (8, 4), A, 1, (1, 1), (1.0, 1.0)), (2, (4, 8), A, 2, (2, 1), (1.0, 2.0)),
    (2, (16, 4), E, 1, (4, 1), (2.0, 1.0)), (2, (8, 12), E, 2, (2, 3), (1.0, 1.5)),
    (3, (8, 2, 2), A, 1, (2, 1, 1), (1.0, 1.0, 1.0)), (3, (2, 8, 4), A, 2, (1, 2, 2), (1.0, 2.0, 0.5)),
    (3, (8, 4, 2), E, 1, (2, 1, 1), (2.0, 1.0, 1.0)),
    (3, (16, 2, 2), MX, 2, (4, 1, 1), (1.0, 1.0, 1.0)), (3, (4, 4, 8), MX, 1, (1, 2, 2), (1.0, 2.0, 0.5)),
]


def _w0(P, system):
    xyz = oracle.node_coords(P)
    s = np.sin(2 * np.pi * xyz[:, 0] / P.hi[0])
    if P.dim > 1:
        s = s + 0.5 * np.cos(2 * np.pi * xyz[:, 1] / P.hi[1])
    m = P.m
    if system == E:
        W0 = np.zeros((m, P.nodes))
        W0[0] = 1.0 + 0.1 * s
        W0[1] = 0.3 * W0[0]
        W0[-1] = 2.5 + 0.05 * s
        return W0
    return np.stack([s * (1.0 + 0.1 * v) for v in range(m)])


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("precision,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_non_cubic_mesh_matches_oracle(kin, case, precision, tol):
    dim, n, system, degree, tiles, hi = CASES[case]
    lam, dt = (3.3 if system != E else 4.0), 0.02
    P = oracle.Problem(dim=dim, n=n, lo=(0.0,) * dim, hi=hi, degree=degree, system=system, lam=lam, dt=dt,
                       adv=(0.7, -0.4, 0.3), tiles=tiles, iters=3)
    W0 = _w0(P, system)
    pr = kin.KIN_FP64 if precision == "f64" else kin.KIN_FP32
    with kin.Context(dim, n, (0.0,) * dim, hi, degree, system, lam, dt, adv=(0.7, -0.4, 0.3), tiles=tiles,
                     iters=3, precision=pr) as ctx:
        ctx.set_state(np.ascontiguousarray(W0.reshape(-1)))
        ctx.step(3)
        W = ctx.get_state()
    f = oracle.init(P, W0)
    oracle.step(P, f, 3)
    Wo = oracle.moments(P, f)
    err = np.abs(W - Wo).max() / np.abs(Wo).max()
    assert err < tol, err
