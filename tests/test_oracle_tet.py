"""Pins for the oracle's tetrahedral-mesh transport (Sec. 3.1 on tetrahedral
cells, Sec. 3.2 downwind order, Sec. 5.1 subdomain iteration).

* the mesh generator: closed, conforming, the cells fill the box;
* the oracle's per-population transport equals an independent dense numpy
  assembly (tests/dense_tet.py: other geometry formulas, quadrature instead
  of closed forms) solved directly (fixed point, iters = 0) and by block
  Jacobi (iters = 1, 2, 3);
* its breadth-first order is topological: every upwind neighbour inside the
  subdomain comes earlier, and levels are one more than the highest upwind
  level (independent V . N from dense_tet);
* constant states stay constant; the mass change of a step is the interface
  defect of the finite iteration;
* convergence to the exact translation of a smooth advected profile and of
  the Euler density wave, at second order in space and time together.
"""
import numpy as np
import pytest

import oracle
import workloads
from tests import dense_tet


def _setup(w):
    return oracle.tet_problem(w), oracle.TetMesh.from_workload(w)


def test_mesh_is_closed_conforming_and_fills_the_box():
    m = workloads.tet_box(3)
    vols = [dense_tet.barycentric(m.xyz[c])[0] for c in range(m.cells)]
    assert np.isclose(sum(vols), 1.0, rtol=1e-13)
    assert np.allclose(vols, vols[0])
    for c in range(m.cells):
        for a in range(4):
            R = m.nbr[c, a]
            assert c in m.nbr[R]                                   # symmetric adjacency
            shared = set(m.vid[c]) - {m.vid[c, a]}
            assert shared <= set(m.vid[R]) and len(shared) == 3    # the face's three vertices


@pytest.mark.parametrize("velset,tiles", [(1, 2), (0, 2), (1, 1)])
def test_transport_equals_dense_assembly(velset, tiles):
    # large dt so that the subdomain coupling matters; 2^3 subdomains, or one
    # subdomain that couples to itself across the periodic boundary
    w = workloads.tet_advection(seed=1, n=4, tiles=tiles, velset=velset, dt_mult=12.0)
    P, T = _setup(w)
    f0 = oracle.tet_init(P, T, w.W0)
    nodes = T.nodes
    sub = w.subdomains()
    for iters in (0, 1, 2, 3):
        P.iters = iters
        f = f0.copy()
        oracle.tet_transport(P, T, f)
        for k in range(P.nvel):
            V = oracle.velocity(P, k)
            A, Mg, Aout = dense_tet.assemble(w.mesh.xyz, w.mesh.vid, w.mesh.nbr, sub, V, 0.5 * w.dt,
                                             w.mesh.wrap)
            fn = f0[k * nodes:(k + 1) * nodes]
            want = dense_tet.global_cn(A, Mg, fn) if iters == 0 else dense_tet.block_jacobi(A, Mg, Aout, fn, iters)
            got = f[k * nodes:(k + 1) * nodes]
            assert np.abs(got - want).max() < 1e-12 * np.abs(want).max(), (velset, iters, k)
    # and the iteration count matters at this dt
    P.iters = 1
    fa = f0.copy()
    oracle.tet_transport(P, T, fa)
    P.iters = 3
    fb = f0.copy()
    oracle.tet_transport(P, T, fb)
    assert np.abs(fa - fb).max() > 1e-6


def test_breadth_first_order_is_topological():
    w = workloads.tet_densitywave(n=4, tiles=2, velset=1, precision="f64")
    P, T = _setup(w)
    sub = w.subdomains()
    for k in range(P.nvel):
        V = oracle.velocity(P, k)
        for s in range(T.nsub):
            order, level = oracle.tet_order(P, T, k, s)
            assert sorted(order) == sorted(np.nonzero(sub == s)[0])
            pos = {int(c): i for i, c in enumerate(order)}
            lev = {int(c): int(l) for c, l in zip(order, level)}
            for c in order:
                _, _, faces = dense_tet.cell_operators(w.mesh.xyz[c], V)
                ups = [int(w.mesh.nbr[c, a]) for a, (vn, _) in enumerate(faces)
                       if vn < 0 and sub[w.mesh.nbr[c, a]] == s and not w.mesh.wrap[c, a]]
                for u in ups:
                    assert pos[u] < pos[int(c)]
                assert lev[int(c)] == (1 + max(lev[u] for u in ups) if ups else 0)


def test_constant_state_is_preserved():
    w = workloads.tet_densitywave(n=4, tiles=2, velset=1, dt_mult=8.0, precision="f64")
    W0 = w.W0.copy()
    W0[0] = 1.3
    W0[1:4] = np.array([0.4, -0.2, 0.3])[:, None]
    W0[4] = 3.1
    P, T = _setup(w)
    f = oracle.tet_init(P, T, W0)
    oracle.tet_step(P, T, f, 3)
    W = oracle.tet_moments(P, T, f).reshape(5, -1)
    assert np.abs(W - W0).max() < 1e-13


@pytest.mark.parametrize("iters", [1, 2])
def test_mass_change_equals_interface_defect(iters):
    # a single Fourier mode sums to zero over the equally spaced subdomain
    # planes, so the density gets a seeded random perturbation
    w = workloads.tet_densitywave(n=4, tiles=2, velset=1, dt_mult=12.0, iters=iters, precision="f64")
    W0 = w.W0.copy()
    W0[0] *= 1.0 + 0.05 * np.random.default_rng(5).standard_normal(W0.shape[1])
    P, T = _setup(w)
    f = oracle.tet_init(P, T, W0)
    m0 = oracle.tet_mass(P, T, oracle.tet_moments(P, T, f))
    defect, _ = oracle.tet_transport(P, T, f)
    oracle.tet_relax(P, T, f)
    m1 = oracle.tet_mass(P, T, oracle.tet_moments(P, T, f))
    assert np.abs(defect).max() > 1e-8                 # the finite iteration leaves a defect here
    assert np.abs((m1 - m0) - defect).max() < 1e-13 * np.abs(m0).max()


def _err(w, steps):
    P, T = _setup(w)
    f = oracle.tet_init(P, T, w.W0)
    oracle.tet_step(P, T, f, steps)
    W = oracle.tet_moments(P, T, f).reshape(w.m, -1)
    return np.abs(W - w.exact(steps * w.dt)).max()


def test_density_wave_converges_at_second_order():
    # mesh and time step refined together (dt = 2 h_min / |V|, 8-cube
    # subdomains, to the same final time): P1 in space and omega = 2 in time
    # are both second order; n = 8 -> 16 is still pre-asymptotic
    errs = [_err(workloads.tet_densitywave(seed=0, n=n, tiles=max(1, n // 8), velset=1, dt_mult=2.0,
                                           precision="f64"), steps=n // 2) for n in (8, 16, 32)]
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert orders[0] > 1.6 and abs(orders[1] - 2.0) < 0.15, (errs, orders)
