"""The seeded workloads are what they claim to be (host only; no scheme
arithmetic): the Maxwell plane waves solve Maxwell's equations (Sec. 6.1.1)
exactly, checked with centred differences of the recipe's own exact()
against the curl written out here; the recipes are reproducible from their
seed; and the oracle receives every field a recipe sets."""
import numpy as np

import workloads


def test_maxwell_plane_waves_solve_maxwells_equations():
    w = workloads.maxwell3d(seed=3, n=4, degree=2, tiles=1)
    rng = np.random.default_rng(0)
    pts = rng.uniform(0.1, 0.9, size=(20, 3))
    eps = 1e-5

    def field(xyz, t):
        # the documented waves at arbitrary points (they equal the recipe at
        # its nodes: next test)
        return _waves(xyz, t, seed=3)

    for x in pts:
        W_t = (field(x, 0.3 + eps) - field(x, 0.3 - eps)) / (2 * eps)
        grad = np.stack([(field(x + eps * e, 0.3) - field(x - eps * e, 0.3)) / (2 * eps)
                         for e in np.eye(3)])           # grad[a, v] = d W_v / d x_a
        E_x = grad[:, :3]                               # E_x[a, i] = d E_i / d x_a
        H_x = grad[:, 3:]
        curl = lambda D: np.array([D[1, 2] - D[2, 1], D[2, 0] - D[0, 2], D[0, 1] - D[1, 0]])
        assert np.abs(W_t[:3] - curl(H_x)).max() < 1e-6      # E_t = curl H
        assert np.abs(W_t[3:] + curl(E_x)).max() < 1e-6      # H_t = -curl E
    # the recipe's exact() agrees with the initial data at t = 0
    assert np.allclose(w.exact(0.0), w.W0)


def _waves(xyz, t, seed):
    """The documented plane waves: along x (E_y = H_z), y (E_z = H_x), z (E_x = H_y),
    amplitudes ~ U(0.5, 1.5) and phases ~ U(0, 2 pi) from the seed."""
    rng = np.random.default_rng(seed)
    phi = rng.uniform(0.0, 2 * np.pi, size=3)
    amp = rng.uniform(0.5, 1.5, size=3)
    W = np.zeros(6)
    for k, (a, e, h) in enumerate(((0, 1, 2), (1, 2, 0), (2, 0, 1))):
        c = amp[k] * np.cos(2 * np.pi * (xyz[a] - t) + phi[k])
        W[e] += c
        W[3 + h] += c
    return W


def test_documented_waves_match_the_recipe_at_its_nodes():
    w = workloads.maxwell3d(seed=3, n=4, degree=2, tiles=1)
    xyz = workloads.node_coords(3, w.n, w.lo, w.hi, w.degree)
    got = np.stack([_waves(p, 0.25, 3) for p in xyz], axis=1)
    assert np.allclose(got, w.exact(0.25), atol=1e-14)


def test_recipes_are_seeded():
    for make in (lambda s: workloads.vortex2d(seed=s, n=8), lambda s: workloads.densitywave3d(seed=s, n=4),
                 lambda s: workloads.maxwell3d(seed=s, n=4), lambda s: workloads.advection1d(seed=s, n=16)):
        a, b, c = make(1), make(1), make(2)
        assert np.array_equal(a.W0, b.W0) and not np.array_equal(a.W0, c.W0)


def test_oracle_kwargs_carry_every_problem_field():
    wb = np.zeros((3, 2, 6))
    wb[0, 1, 2] = 0.5
    w = workloads.with_(workloads.maxwell3d(seed=0, n=4, sigma=2.5), inflow=(1, 0, 0), Wb=wb)
    kw = w.oracle_kwargs()
    assert kw["sigma"] == 2.5 and kw["inflow"] == (1, 0, 0) and kw["Wb"] is wb
    assert kw["system"] == workloads.MAXWELL and kw["dim"] == 3
