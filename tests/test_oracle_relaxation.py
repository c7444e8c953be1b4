"""Pins for the Maxwellians (eq. maxwell_def), the Euler flux and the
over-relaxation (eq. over_relaxation and the Y+ = -Y- identity of Sec. 2.4)."""
import numpy as np
import pytest

import oracle


def _euler(dim, gamma=1.4):
    return oracle.Problem(dim=dim, n=(1,) * dim, lo=(0.0,) * dim, hi=(1.0,) * dim, degree=1,
                          system=oracle.EULER, lam=9.0, dt=0.1, gamma=gamma)


def test_euler_flux_worked_example(golden):
    rows = {r[0][0]: r[1] for r in golden("euler_flux.txt")}
    P = _euler(2, gamma=rows["gamma"][0])
    W = np.array(rows["W"])
    np.testing.assert_allclose(oracle.flux(P, W, 0), rows["Qx"], atol=1e-14)
    np.testing.assert_allclose(oracle.flux(P, W, 1), rows["Qy"], atol=1e-14)


def _primitive_flux(rho, vel, pr, gamma, axis):
    # flux from primitive variables (the physical definition of the Euler
    # fluxes: mass, momentum and energy transported by u_axis, plus pressure)
    kin = 0.5 * rho * sum(u * u for u in vel)
    E = pr / (gamma - 1.0) + kin
    ua = vel[axis]
    mom = [rho * u * ua + (pr if b == axis else 0.0) for b, u in enumerate(vel)]
    return np.array([rho * ua] + mom + [ua * (E + pr)]), np.array([rho] + [rho * u for u in vel] + [E])


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_maxwellian_moments_euler(dim):
    rng = np.random.default_rng(dim)
    P = _euler(dim)
    lam = P.lam
    for _ in range(20):
        rho = rng.uniform(0.5, 2.0)
        vel = list(rng.uniform(-1, 1, size=dim))
        pr = rng.uniform(0.5, 2.0)
        W = _primitive_flux(rho, vel, pr, 1.4, 0)[1]
        M = oracle.maxwellian(P, W)
        np.testing.assert_allclose(M.sum(axis=0), W, rtol=1e-14, atol=1e-14)
        for a in range(dim):
            Qa = _primitive_flux(rho, vel, pr, 1.4, a)[0]
            first = lam * M[2 * a] - lam * M[2 * a + 1]        # sum_k V_k^a M_k
            np.testing.assert_allclose(first, Qa, rtol=1e-13, atol=1e-13)


def test_maxwellian_advection_d1q2():
    P = oracle.Problem(dim=1, n=(1,), lo=(0.0,), hi=(1.0,), degree=1,
                       system=oracle.ADVECTION, lam=2.0, dt=0.1, adv=(0.5, 0, 0))
    M = oracle.maxwellian(P, np.array([3.0]))
    # D1Q2: M_+ + M_- = u, lambda (M_+ - M_-) = a u -> unique (Sec. 2.4, d = 1)
    np.testing.assert_allclose(M[:, 0], [1.5 + 0.375, 1.5 - 0.375], atol=1e-15)


def _random_euler_f(P, rng):
    nodes = P.nodes
    W0 = np.zeros((P.m, nodes))
    W0[0] = rng.uniform(0.8, 1.2, nodes)
    for a in range(P.dim):
        W0[1 + a] = W0[0] * rng.uniform(-0.3, 0.3, nodes)
    W0[-1] = 2.5 + 0.5 * np.sum(W0[1:1 + P.dim] ** 2, axis=0) / W0[0]
    f = oracle.init(P, W0)
    f += rng.normal(0, 0.01, f.size)        # f != M(W): a state after a transport
    return f


def _grid_problem(dim, omega):
    return oracle.Problem(dim=dim, n=(3,) * dim, lo=(0.0,) * dim, hi=(1.0,) * dim, degree=1,
                          system=oracle.EULER, lam=9.0, dt=0.1, omega=omega)


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_relaxation_keeps_W_and_omega2_is_involution(dim):
    rng = np.random.default_rng(10 + dim)
    P = _grid_problem(dim, 2.0)
    f = _random_euler_f(P, rng)
    W = oracle.moments(P, f)
    g = f.copy()
    oracle.relax(P, g)
    np.testing.assert_allclose(oracle.moments(P, g), W, rtol=1e-14, atol=1e-14)
    oracle.relax(P, g)
    np.testing.assert_allclose(g, f, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_flux_error_flips_sign_for_omega2(dim):
    # Y^a = sum_k V_k^a (F_k - M_k(W)) changes sign under the omega = 2 relaxation
    rng = np.random.default_rng(20 + dim)
    P = _grid_problem(dim, 2.0)
    f = _random_euler_f(P, rng)
    nodes = P.nodes
    m = P.m
    W = oracle.moments(P, f).reshape(m, nodes)
    Mx = np.stack([oracle.maxwellian(P, W[:, i]) for i in range(nodes)], axis=-1)  # (nvel, m, nodes)

    def Y(ff):
        F = ff.reshape(2 * dim, m, nodes)
        return [P.lam * ((F[2 * a] - Mx[2 * a]) - (F[2 * a + 1] - Mx[2 * a + 1])) for a in range(dim)]

    before = Y(f)
    g = f.copy()
    oracle.relax(P, g)
    after = Y(g)
    for a in range(dim):
        np.testing.assert_allclose(after[a], -before[a], atol=1e-12)


def test_omega1_projects_on_equilibrium():
    rng = np.random.default_rng(3)
    P = _grid_problem(2, 1.0)
    f = _random_euler_f(P, rng)
    W = oracle.moments(P, f)
    oracle.relax(P, f)
    np.testing.assert_allclose(f, oracle.init(P, W), rtol=1e-14, atol=1e-14)
