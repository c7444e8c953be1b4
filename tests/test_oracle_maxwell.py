"""Pins of the oracle's Maxwell system (Sec. 6.1.1) and conductivity source
(Sec. 2.3, Sec. 6.4): a hand-worked flux, the hyperbolic structure (wave
speeds 0 and +-1), the moment identities of the Maxwellians, the closed form
of a uniform field under the source step, and the exact plane wave with the
scheme's second order in time."""
import numpy as np
import pytest

import oracle

BOX = dict(lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0))


def problem(n=(4, 2, 2), degree=1, dt=0.01, sigma=0.0, lam=3.3, tiles=(1, 1, 1), iters=3, omega=2.0):
    return oracle.Problem(dim=3, n=n, degree=degree, system=oracle.MAXWELL, lam=lam, dt=dt, sigma=sigma,
                          tiles=tiles, iters=iters, omega=omega, **BOX)


def test_flux_hand_worked(golden):
    g = {r[0][0]: r[1] for r in golden("maxwell_flux.txt")}
    P = problem()
    W = np.array(g["W"])
    for a, key in enumerate(("Qx", "Qy", "Qz")):
        assert np.allclose(oracle.flux(P, W, a), g[key], atol=0, rtol=0)


def test_flux_is_linear_with_light_speed_one():
    # Maxwell is linear: Q^a(W) = A_a W; A_a has eigenvalues -1, -1, 0, 0, 1, 1
    P = problem()
    for a in range(3):
        A = np.stack([oracle.flux(P, np.eye(6)[c], a) for c in range(6)], axis=1)
        W = np.random.default_rng(a).normal(size=6)
        assert np.allclose(A @ W, oracle.flux(P, W, a), atol=1e-15)
        ev = np.sort(np.linalg.eigvals(A).real)
        assert np.allclose(ev, [-1, -1, 0, 0, 1, 1], atol=1e-12)


def test_maxwellian_moments():
    P = problem()
    W = np.random.default_rng(7).normal(size=6)
    M = oracle.maxwellian(P, W).reshape(P.nvel, 6)
    assert np.allclose(M.sum(axis=0), W, atol=1e-14)
    for a in range(3):
        VM = sum(oracle.velocity(P, k)[a] * M[k] for k in range(P.nvel))
        assert np.allclose(VM, oracle.flux(P, W, a), atol=1e-14)


def _uniform(P, E, H):
    W0 = np.zeros((6, P.nodes))
    W0[:3] = np.asarray(E)[:, None]
    W0[3:] = np.asarray(H)[:, None]
    return W0


@pytest.mark.parametrize("sigma,dt", [(3.0, 0.05), (40.0, 0.2)])
def test_uniform_field_decays_by_mu_per_step(sigma, dt):
    # a uniform field is transported unchanged; the Crank-Nicolson source step
    # multiplies E by mu = (1 - sigma dt / 2) / (1 + sigma dt / 2) (Sec. 6.4)
    # every step and leaves H alone, for any omega
    for omega in (2.0, 1.5):
        P = problem(dt=dt, sigma=sigma, omega=omega)
        E, H = np.array([0.3, -1.2, 0.7]), np.array([2.0, 0.1, -0.4])
        f = oracle.init(P, _uniform(P, E, H))
        nsteps = 7
        oracle.step(P, f, nsteps)
        W = oracle.moments(P, f).reshape(6, -1)
        mu = (1 - sigma * dt / 2) / (1 + sigma * dt / 2)
        assert np.allclose(W[:3], (mu ** nsteps * E)[:, None], atol=1e-13)
        assert np.allclose(W[3:], H[:, None], atol=1e-13)


def _plane_wave(P, t, phase=0.3):
    # E_y = H_z = cos(2 pi (x - t) + phase): a wave moving along +x with speed 1
    x = oracle.node_coords(P)[:, 0]
    c = np.cos(2 * np.pi * (x - t) + phase)
    W = np.zeros((6, P.nodes))
    W[1] = c
    W[5] = c
    return W


def _wave_error(n, degree, dt, T):
    P = problem(n=(n, 2, 2), degree=degree, dt=dt)
    f = oracle.init(P, _plane_wave(P, 0.0))
    steps = int(round(T / dt))
    oracle.step(P, f, steps)
    W = oracle.moments(P, f).reshape(P.m, -1)
    return np.abs(W - _plane_wave(P, steps * dt)).max()


def test_plane_wave_converges():
    # space and time refined together (dt = h / 2, CFL-less regime for p = 2)
    e = [_wave_error(n, 2, 0.5 / n, 0.5) for n in (8, 16, 32)]
    assert e[0] > e[1] > e[2]
    assert np.log2(e[1] / e[2]) > 1.7


def test_plane_wave_second_order_in_time():
    # fine space (p = 3, 16 cells), large time steps: the time error dominates
    e = [_wave_error(16, 3, dt, 0.8) for dt in (0.05, 0.025, 0.0125)]
    r = [np.log2(e[0] / e[1]), np.log2(e[1] / e[2])]
    assert min(r) > 1.8, (e, r)


def test_zero_conductivity_is_the_plain_relaxation():
    # with sigma = 0 the source step is the identity and the relaxation is
    # omega M(W) + (1 - omega) f (eq. over_relaxation): for omega = 2 an involution
    P = problem(sigma=0.0)
    rng = np.random.default_rng(3)
    f = rng.normal(size=(P.npop, P.nodes))
    g = f.copy()
    oracle.relax(P, g)
    W = oracle.moments(P, f).reshape(P.m, -1)
    M = np.stack([oracle.maxwellian(P, W[:, i]).reshape(-1) for i in range(P.nodes)], axis=1)
    assert np.allclose(g, 2 * M - f, atol=1e-13)
    oracle.relax(P, g)
    assert np.allclose(g, f, atol=1e-13)
