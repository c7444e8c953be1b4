"""Pins for the oracle with the paper's own d + 1 velocity sets: D2Q3 at 120
degrees (Sec. 2.4) and D3Q4 on the cube diagonals (Sec. 6.1.3), whose
velocities are not aligned with the mesh, so every cell has several inflow
faces and subdomains meet at corners (Sec. 5.1, three-iteration case)."""
import numpy as np
import pytest

import oracle
import workloads
from tests import dense_dg


def _euler(dim, lam=4.0):
    return oracle.Problem(dim=dim, n=(1,) * dim, lo=(0.0,) * dim, hi=(1.0,) * dim, degree=1,
                          system=oracle.EULER, lam=lam, dt=0.1, velset=oracle.SIMPLEX)


def _primitive(rng, dim):
    rho = rng.uniform(0.5, 2.0)
    vel = rng.uniform(-1, 1, size=dim)
    pr = rng.uniform(0.5, 2.0)
    E = pr / 0.4 + 0.5 * rho * vel @ vel
    W = np.concatenate([[rho], rho * vel, [E]])
    Q = [np.concatenate([[rho * vel[a]], rho * vel * vel[a] + pr * (np.arange(dim) == a),
                         [vel[a] * (E + pr)]]) for a in range(dim)]
    return W, Q


def paper_velocities(dim, lam):
    if dim == 2:
        return [lam * np.array([np.cos(2 * np.pi * k / 3), np.sin(2 * np.pi * k / 3)]) for k in range(3)]
    return [lam * np.array(v) for v in ([1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1])]


@pytest.mark.parametrize("dim", [2, 3])
def test_velocities_are_the_papers(dim):
    P = _euler(dim, lam=1.7)
    for k, V in enumerate(paper_velocities(dim, 1.7)):
        np.testing.assert_allclose(oracle.velocity(P, k), V, atol=1e-15)


def test_d3q4_maxwellian_is_the_papers_closed_form(golden):
    rows = {r[0][0]: r[1] for r in golden("d3q4_maxwellian.txt")}
    lam = 2.3
    vels = lam * np.array(rows["velocities"]).reshape(4, 3)
    P = _euler(3, lam)
    rng = np.random.default_rng(0)
    for _ in range(10):
        W, Q = _primitive(rng, 3)
        M = oracle.maxwellian(P, W)
        for k in range(4):
            QV = sum(vels[k][a] * Q[a] for a in range(3))
            want = rows["weight_W"][0] * W + rows["weight_Q_over_lambda2"][0] * QV / lam ** 2
            np.testing.assert_allclose(M[k], want, rtol=1e-13, atol=1e-13)


def test_d2q3_maxwellian_closed_form():
    # sum_k V_k = 0 and sum_k V_k V_k^T = (3 lambda^2 / 2) I for the 120-degree
    # set, so eq. maxwell_def gives M_k = W/3 + 2 Q(W, V_k) / (3 lambda^2)
    lam = 1.9
    P = _euler(2, lam)
    rng = np.random.default_rng(1)
    vels = paper_velocities(2, lam)
    for _ in range(10):
        W, Q = _primitive(rng, 2)
        M = oracle.maxwellian(P, W)
        for k in range(3):
            QV = sum(vels[k][a] * Q[a] for a in range(2))
            np.testing.assert_allclose(M[k], W / 3 + 2 * QV / (3 * lam ** 2), rtol=1e-13, atol=1e-13)


def _adv_simplex(dim, n, p, tiles, iters):
    hi = tuple(1.0 + 0.25 * a for a in range(dim))
    lam = 1.3
    dt = 7.0 * min(hi[a] / n[a] for a in range(dim)) / lam
    return oracle.Problem(dim=dim, n=n, lo=(0.0,) * dim, hi=hi, degree=p, system=oracle.ADVECTION,
                          lam=lam, dt=dt, tiles=tiles, iters=iters, velset=oracle.SIMPLEX)


CASES = [(2, (4, 4), 1, (2, 2)), (2, (4, 2), 2, (2, 1)), (2, (3, 3), 1, (1, 1)),
         (3, (2, 2, 2), 1, (2, 2, 2)), (3, (2, 2, 1), 2, (1, 2, 1))]


@pytest.mark.parametrize("dim,n,p,tiles", CASES)
@pytest.mark.parametrize("iters", [1, 2, 3, 0])
def test_diagonal_transport_equals_dense_assembly(dim, n, p, tiles, iters):
    P = _adv_simplex(dim, n, p, tiles, iters)
    rng = np.random.default_rng(17)
    f0 = rng.normal(size=P.npop * P.nodes)
    f = f0.copy()
    oracle.transport(P, f)
    nodes = P.nodes
    for k, V in enumerate(paper_velocities(dim, P.lam)):
        M, K, Kout = dense_dg.assemble(dim, n, P.lo, P.hi, p, V, tiles)
        if iters == 0:
            want = dense_dg.global_cn(M, K, 0.5 * P.dt, f0[k * nodes:(k + 1) * nodes])
            tol = 1e-11
        else:
            want = dense_dg.block_jacobi(M, K, Kout, 0.5 * P.dt, f0[k * nodes:(k + 1) * nodes], iters)
            tol = 1e-12
        np.testing.assert_allclose(f[k * nodes:(k + 1) * nodes], want, rtol=tol, atol=tol)


@pytest.mark.parametrize("dim,n,p,tiles", CASES)
def test_diagonal_mass_change_equals_interface_defect(dim, n, p, tiles):
    P = _adv_simplex(dim, n, p, tiles, 2)
    f = np.random.default_rng(3).normal(size=P.npop * P.nodes)
    m0 = oracle.mass(P, oracle.moments(P, f))
    defect, _ = oracle.transport(P, f)
    m1 = oracle.mass(P, oracle.moments(P, f))
    assert abs((m1 - m0) - defect)[0] < 1e-12


def test_corner_sharing_subdomains_iteration_converges():
    # 2x2 subdomains meeting at corners, diagonal velocities: the K-th iterate
    # approaches the global solve as K grows (Sec. 5.1)
    base = dict(dim=2, n=(6, 6), p=1, tiles=(2, 2))
    f0 = np.random.default_rng(9).normal(size=_adv_simplex(2, (6, 6), 1, (2, 2), 1).npop * 36 * 4)
    ref = f0.copy()
    oracle.transport(_adv_simplex(2, (6, 6), 1, (2, 2), 0), ref)
    errs = []
    for K in (1, 2, 3, 4, 5):
        g = f0.copy()
        oracle.transport(_adv_simplex(2, (6, 6), 1, (2, 2), K), g)
        errs.append(np.abs(g - ref).max())
    assert all(b < a for a, b in zip(errs, errs[1:])), errs


def test_d2q3_euler_time_order_two():
    base = workloads.densitywave2d(seed=3, n=16, degree=3, tiles=2, velset=1)
    errs = []
    for dt in (0.02, 0.01, 0.005):
        w = workloads.with_(base, dt=dt)
        P = oracle.Problem(**w.oracle_kwargs())
        f = oracle.init(P, w.W0)
        ns = int(round(0.2 / dt))
        oracle.step(P, f, ns)
        W = oracle.moments(P, f).reshape(w.m, -1)
        errs.append(np.abs(W - w.exact(ns * dt)).max())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(orders - 2.0) < 0.15), errs


def test_d3q4_euler_converges():
    errs = []
    for n in (4, 8):
        w = workloads.densitywave3d(seed=2, n=n, degree=1, tiles=2, velset=1)
        P = oracle.Problem(**w.oracle_kwargs())
        f = oracle.init(P, w.W0)
        ns = int(round(0.1 / w.dt))
        oracle.step(P, f, ns)
        W = oracle.moments(P, f).reshape(w.m, -1)
        errs.append(np.abs(W - w.exact(ns * w.dt)).max())
    assert errs[1] < errs[0] / 1.5, errs


def _two_by_two(simplex, iters, cfl=0.5):
    # 24^2 cells, p = 1, 2 x 2 periodic subdomains of 12^2 cells; a small time
    # step (|V| dt = cfl h) so that a subdomain's influence across its
    # neighbour within one step is far below round-off
    lam = 1.3
    kw = dict(velset=oracle.SIMPLEX) if simplex else {}
    return oracle.Problem(dim=2, n=(24, 24), lo=(0.0, 0.0), hi=(1.0, 1.0), degree=1, system=oracle.ADVECTION,
                          lam=lam, dt=cfl / 24 / lam, tiles=(2, 2), iters=iters, adv=(0.7, 0.4, 0.0), **kw)


def test_iterations_to_the_global_solve_aligned_two_corners_three():
    # Sec. 5.1: under dt <= L/|V| the subdomain iteration of eq. ibvp is exact
    # after two iterations when the velocity is aligned with the subdomain
    # faces and after three when subdomains meet at corners.  Discretely:
    # D2Q4 reaches the global solve (iters = 0) at K = 2, the oblique D2Q3
    # only at K = 3, to round-off
    for simplex, exact_at in ((False, 2), (True, 3)):
        P0 = _two_by_two(simplex, 0)
        f0 = np.random.default_rng(1).normal(size=P0.npop * P0.nodes)
        ref = f0.copy()
        oracle.transport(P0, ref)
        errs = {}
        for K in (exact_at - 1, exact_at):
            g = f0.copy()
            oracle.transport(_two_by_two(simplex, K), g)
            errs[K] = np.abs(g - ref).max()
        assert errs[exact_at - 1] > 1e-2, (simplex, errs)
        assert errs[exact_at] < 1e-12, (simplex, errs)
