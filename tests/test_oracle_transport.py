"""Pins for the oracle's transport (Sec. 3, eq. dg_imp with Crank-Nicolson;
Sec. 5.1, eq. ibvp): dense global solve, dense block-Jacobi iteration,
constant states, and the interface mass defect."""
import numpy as np
import pytest

import oracle
from tests import dense_dg


def _adv_problem(dim, n, p, tiles, iters, lam=1.3, dt=None):
    hi = tuple(1.0 + 0.25 * a for a in range(dim))        # non-square cells
    if dt is None:
        dt = 9.0 * min(hi[a] / n[a] for a in range(dim)) / lam   # lambda dt / h = 9: long reach
    return oracle.Problem(dim=dim, n=n, lo=(0.0,) * dim, hi=hi, degree=p,
                          system=oracle.ADVECTION, lam=lam, dt=dt, tiles=tiles, iters=iters)


def _velocities(P):
    out = []
    for k in range(2 * P.dim):
        V = [0.0] * P.dim
        V[k // 2] = P.lam if k % 2 == 0 else -P.lam
        out.append(V)
    return out


CASES = [
    (1, (8,), 1, (1,)), (1, (8,), 2, (2,)), (1, (8,), 3, (4,)), (1, (6,), 2, (3,)),
    (2, (4, 3), 1, (2, 1)), (2, (4, 4), 2, (2, 2)), (2, (4, 2), 2, (1, 1)),
    (3, (2, 2, 2), 1, (2, 1, 2)),
]


@pytest.mark.parametrize("dim,n,p,tiles", CASES)
@pytest.mark.parametrize("iters", [1, 2, 3])
def test_transport_equals_dense_block_jacobi(dim, n, p, tiles, iters):
    P = _adv_problem(dim, n, p, tiles, iters)
    rng = np.random.default_rng(hash((dim, n, p, tiles, iters)) % 2 ** 32)
    f0 = rng.normal(size=P.npop * P.nodes)
    f = f0.copy()
    oracle.transport(P, f)
    nodes = P.nodes
    for k, V in enumerate(_velocities(P)):
        M, K, Kout = dense_dg.assemble(dim, n, P.lo, P.hi, p, V, tiles)
        want = dense_dg.block_jacobi(M, K, Kout, 0.5 * P.dt, f0[k * nodes:(k + 1) * nodes], iters)
        np.testing.assert_allclose(f[k * nodes:(k + 1) * nodes], want, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("dim,n,p,tiles", CASES)
def test_fixed_point_equals_dense_global_solve(dim, n, p, tiles):
    P = _adv_problem(dim, n, p, tiles, iters=0)
    rng = np.random.default_rng(7)
    f0 = rng.normal(size=P.npop * P.nodes)
    f = f0.copy()
    _, it = oracle.transport(P, f)
    assert it > 3
    nodes = P.nodes
    for k, V in enumerate(_velocities(P)):
        M, K, _ = dense_dg.assemble(dim, n, P.lo, P.hi, p, V, tiles)
        want = dense_dg.global_cn(M, K, 0.5 * P.dt, f0[k * nodes:(k + 1) * nodes])
        np.testing.assert_allclose(f[k * nodes:(k + 1) * nodes], want, rtol=1e-11, atol=1e-11)


@pytest.mark.parametrize("dim,n,p,tiles", CASES)
@pytest.mark.parametrize("iters", [1, 3])
def test_constant_state_is_preserved(dim, n, p, tiles, iters):
    P = _adv_problem(dim, n, p, tiles, iters)
    f = np.repeat(np.arange(1.0, P.npop + 1.0), P.nodes)
    g = f.copy()
    oracle.transport(P, g)
    np.testing.assert_allclose(g, f, rtol=1e-13)


@pytest.mark.parametrize("dim,n,p,tiles", CASES)
@pytest.mark.parametrize("iters", [1, 2, 3])
def test_mass_change_equals_interface_defect(dim, n, p, tiles, iters):
    # Summing eq. dg_imp over all cells and test functions, interior faces
    # cancel; only subdomain-boundary faces, whose inflow uses iterate K-1
    # while the upwind outflow uses iterate K, change the total mass.
    P = _adv_problem(dim, n, p, tiles, iters)
    rng = np.random.default_rng(11)
    f = rng.normal(size=P.npop * P.nodes)
    m0 = oracle.mass(P, oracle.moments(P, f))
    defect, _ = oracle.transport(P, f)
    m1 = oracle.mass(P, oracle.moments(P, f))
    scale = np.sum(np.abs(f)) * np.prod(P.hi) / P.nodes
    assert abs((m1 - m0) - defect)[0] < 1e-13 * max(scale, 1.0)
    if iters < 3 or max(tiles) > 1:
        assert abs(defect[0]) > 1e-9      # the case really exercises the interfaces


def test_single_subdomain_wrap_couples_to_itself():
    # One periodic subdomain: iteration 1 takes the wrap inflow from f^n, so it
    # differs from the global solve; more iterations approach it.
    P1 = _adv_problem(1, (6,), 2, (1,), 1)
    Pinf = _adv_problem(1, (6,), 2, (1,), 0)
    f0 = np.random.default_rng(5).normal(size=P1.npop * P1.nodes)
    a, b = f0.copy(), f0.copy()
    oracle.transport(P1, a)
    oracle.transport(Pinf, b)
    assert np.abs(a - b).max() > 1e-3
    errs = []
    for K in (1, 2, 3, 4):
        c = f0.copy()
        oracle.transport(_adv_problem(1, (6,), 2, (1,), K), c)
        errs.append(np.abs(c - b).max())
    assert all(e2 < e1 for e1, e2 in zip(errs, errs[1:]))
