"""Pins of the oracle's inflow boundaries: the paper prescribes the solution
on the domain boundary (Sec. 6.2) and takes the upwind value across every
face (eq. dg_imp); on a non-periodic axis the value across a domain-boundary
face is the Maxwellian of the face's boundary state.

* an independent dense assembly with the boundary couplings moved to the
  right-hand side, solved densely (fixed point) and by K block-Jacobi
  iterations (eq. ibvp), equals the oracle's transport;
* a uniform state equal to every boundary state is kept exactly by whole
  steps (Euler in 2D, Maxwell in 3D);
* a smooth bump advected away from both boundaries converges to its exact
  translation at second order, with the inflow state it sits on.
"""
import numpy as np
import pytest

import oracle
from tests import dense_dg


def _adv(dim, n, p, tiles, iters, inflow, Wb, lam=1.3, adv=(0.7, -0.4, 0.3)):
    hi = tuple(1.0 + 0.25 * a for a in range(dim))
    dt = 9.0 * min(hi[a] / n[a] for a in range(dim)) / lam
    return oracle.Problem(dim=dim, n=n, lo=(0.0,) * dim, hi=hi, degree=p, system=oracle.ADVECTION,
                          lam=lam, dt=dt, adv=adv, tiles=tiles, iters=iters, inflow=inflow, Wb=Wb)


def _velocities(P):
    out = []
    for k in range(2 * P.dim):
        V = [0.0] * P.dim
        V[k // 2] = P.lam if k % 2 == 0 else -P.lam
        out.append(V)
    return out


def _boundary_values(P, k):
    """The value across each boundary face for population k of scalar
    advection, from the 2d-velocity Maxwellian u/(2d) +- a_a u/(2 lambda)
    written out here (not the oracle's routine)."""
    a, sgn = k // 2, (1.0 if k % 2 == 0 else -1.0)
    Wb = np.asarray(P.Wb, dtype=float)
    out = {}
    for b in range(P.dim):
        for side, s in ((-1, 0), (1, 1)):
            u = Wb[b, s, 0]
            out[(b, side)] = u / (2 * P.dim) + sgn * P.adv[a] * u / (2 * P.lam)
    return out


CASES = [
    (1, (8,), 1, (1,), (1,)), (1, (8,), 2, (2,), (1,)), (1, (6,), 3, (3,), (1,)),
    (2, (4, 3), 1, (2, 1), (1, 0)), (2, (4, 4), 2, (2, 2), (0, 1)), (2, (4, 2), 2, (1, 2), (1, 1)),
    (3, (2, 2, 2), 1, (2, 1, 2), (1, 0, 1)),
]


def _wb(dim, seed):
    rng = np.random.default_rng(seed)
    wb = np.zeros((3, 2, 1))
    wb[:dim] = rng.uniform(0.5, 2.0, size=(dim, 2, 1))
    return wb


@pytest.mark.parametrize("dim,n,p,tiles,inflow", CASES)
@pytest.mark.parametrize("iters", [1, 2, 3, 0])
def test_transport_equals_dense_assembly_with_boundary_data(dim, n, p, tiles, inflow, iters):
    P = _adv(dim, n, p, tiles, iters, inflow, _wb(dim, dim * 10 + p))
    rng = np.random.default_rng(hash((dim, n, p, tiles, iters)) % 2 ** 32)
    f0 = rng.normal(size=P.npop * P.nodes)
    f = f0.copy()
    oracle.transport(P, f)
    nodes = P.nodes
    for k, V in enumerate(_velocities(P)):
        M, K, Kout, Kb = dense_dg.assemble_bc(dim, n, P.lo, P.hi, p, V, tiles, inflow)
        # one inflow face per open axis along which this velocity moves
        assert len(Kb) == sum(1 for a in range(dim) if inflow[a] and V[a] != 0)
        bv = _boundary_values(P, k)
        fk = f0[k * nodes:(k + 1) * nodes]
        if iters == 0:
            want = dense_dg.global_cn(M, K, 0.5 * P.dt, fk, Kb, bv)
            tol = 1e-11
        else:
            want = dense_dg.block_jacobi(M, K, Kout, 0.5 * P.dt, fk, iters, Kb, bv)
            tol = 1e-12
        np.testing.assert_allclose(f[k * nodes:(k + 1) * nodes], want, rtol=tol, atol=tol)


def test_boundary_data_matter():
    # the same problem with periodic axes, or another boundary state, differs
    P = _adv(1, (8,), 2, (2,), 3, (1,), _wb(1, 3))
    f0 = np.random.default_rng(1).normal(size=P.npop * P.nodes)
    outs = []
    for prob in (P, oracle.Problem(**{**P.__dict__, "inflow": (0,), "_c": None}),
                 oracle.Problem(**{**P.__dict__, "Wb": 2 * np.asarray(P.Wb), "_c": None})):
        f = f0.copy()
        oracle.transport(prob, f)
        outs.append(f)
    assert np.abs(outs[0] - outs[1]).max() > 1e-3
    assert np.abs(outs[0] - outs[2]).max() > 1e-3


def test_uniform_euler_state_equal_to_boundary_state_is_kept():
    gamma = 1.4
    rho, u, v, pr = 1.3, 0.4, -0.2, 0.9
    W = np.array([rho, rho * u, rho * v, pr / (gamma - 1) + 0.5 * rho * (u * u + v * v)])
    wb = np.zeros((3, 2, 4))
    wb[:2] = W
    P = oracle.Problem(dim=2, n=(6, 4), lo=(0, 0), hi=(1, 1), degree=2, system=oracle.EULER, lam=4.0,
                       dt=0.05, tiles=(2, 2), iters=3, inflow=(1, 1), Wb=wb)
    W0 = np.repeat(W[:, None], P.nodes, axis=1)
    f = oracle.init(P, W0)
    oracle.step(P, f, 4)
    Wn = oracle.moments(P, f).reshape(4, -1)
    assert np.abs(Wn - W0).max() < 1e-13


def test_uniform_maxwell_field_equal_to_boundary_state_is_kept():
    E, H = np.array([0.3, -0.5, 0.8]), np.array([0.1, 0.7, -0.2])
    W = np.concatenate([E, H])
    wb = np.zeros((3, 2, 6))
    wb[:] = W
    P = oracle.Problem(dim=3, n=(4, 2, 2), lo=(0, 0, 0), hi=(1, 1, 1), degree=1, system=oracle.MAXWELL,
                       lam=3.3, dt=0.05, tiles=(2, 1, 1), iters=3, inflow=(1, 1, 1), Wb=wb)
    W0 = np.repeat(W[:, None], P.nodes, axis=1)
    f = oracle.init(P, W0)
    oracle.step(P, f, 3)
    Wn = oracle.moments(P, f).reshape(6, -1)
    assert np.abs(Wn - W0).max() < 1e-13


def _bump(x, c=1.0, x0=0.45, width=0.25):
    r = np.clip((x - x0) / width, -1.0, 1.0)
    return c + np.where(np.abs(r) < 1.0, np.cos(0.5 * np.pi * r) ** 6, 0.0)


def test_bump_with_inflow_converges_to_translation_at_second_order():
    # u_t + u_x = 0 on [0, 1], inflow state 1 on both faces, lambda = 1.5.
    # Up to t = 0.1 the bump (support 0.2..0.7 + t) and every kinetic wave it
    # sends (speed lambda) stay inside the domain, so the exact solution is
    # its translation on the constant inflow state
    errs = []
    T = 0.1
    for n in (64, 128, 256):
        steps = n // 8
        P = oracle.Problem(dim=1, n=(n,), lo=(0.0,), hi=(1.0,), degree=2, system=oracle.ADVECTION,
                           lam=1.5, dt=T / steps, adv=(1.0, 0, 0), tiles=(4,), iters=3, inflow=(1,),
                           Wb=np.ones((3, 2, 1)))
        x = oracle.node_coords(P)[:, 0]
        f = oracle.init(P, _bump(x)[None, :])
        oracle.step(P, f, steps)
        u = oracle.moments(P, f).reshape(-1)
        errs.append(np.abs(u - _bump(x - T)).max())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert errs[-1] < 3e-3 and rates.min() > 1.85, (errs, rates)


def _advect_with_boundary_data(n, when, T=0.25):
    # u_t + u_x = 0 on [0, 1], u = sin(2 pi (x - t)) + 2 exactly; the boundary
    # states of both faces are set from the exact solution before every step,
    # at time t^n + when * dt
    steps = n // 4
    dt = T / steps
    P = oracle.Problem(dim=1, n=(n,), lo=(0.0,), hi=(1.0,), degree=2, system=oracle.ADVECTION, lam=1.5,
                       dt=dt, adv=(1.0, 0, 0), tiles=(4,), iters=3, inflow=(1,), Wb=np.zeros((3, 2, 1)))
    x = oracle.node_coords(P)[:, 0]
    exact = lambda x, t: np.sin(2 * np.pi * (x - t)) + 2.0
    f = oracle.init(P, exact(x, 0.0)[None, :])
    for s in range(steps):
        t = (s + when) * dt
        wb = np.zeros((3, 2, 1))
        wb[0, 0, 0], wb[0, 1, 0] = exact(0.0, t), exact(1.0, t)
        P.Wb = wb
        oracle.step(P, f, 1)
    return np.abs(oracle.moments(P, f).reshape(-1) - exact(x, T)).max()


def test_time_dependent_boundary_data_enter_at_the_midpoint():
    # the implicit half step of Crank-Nicolson sits at t^{n+1/2}: boundary
    # data taken there keep second order, data at t^n or t^{n+1} drop to first
    def order(when):
        e = [_advect_with_boundary_data(n, when) for n in (64, 128, 256)]
        return np.log2(e[0] / e[1]), np.log2(e[1] / e[2])
    assert min(order(0.5)) > 1.9
    assert max(order(0.0)) < 1.2 and max(order(1.0)) < 1.2
