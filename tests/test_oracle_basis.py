"""Pins for the oracle's Gauss-Lobatto rule, differentiation matrix and local
DG cell operator (Sec. 3.1, eq. dg_imp) against closed forms and hand-worked
values."""
import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_gll_matches_closed_forms(golden, p):
    rows = {int(r[0][0]): r for r in golden("gll.txt")}
    nodes = np.array(rows[p][1])
    weights = np.array(rows[p][2])
    xi, w = oracle.gll(p)
    np.testing.assert_allclose(xi, 0.5 * (nodes + 1.0), atol=1e-15)
    np.testing.assert_allclose(w, 0.5 * weights, atol=1e-15)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_gll_quadrature_exact_to_degree_2p_minus_1(p):
    xi, w = oracle.gll(p)
    for k in range(2 * p):
        assert abs(np.sum(w * xi ** k) - 1.0 / (k + 1)) < 1e-14


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_diff_matrix_differentiates_polynomials_exactly(p):
    xi, _ = oracle.gll(p)
    D = oracle.diff_matrix(p)
    for k in range(p + 1):
        want = k * xi ** (k - 1) if k else np.zeros_like(xi)
        np.testing.assert_allclose(D @ xi ** k, want, atol=1e-12)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_summation_by_parts(p):
    # Q = W D satisfies Q + Q^T = diag(-1, 0, ..., 0, 1) (discrete integration
    # by parts, exact because the GLL rule integrates l_i l_j' exactly).
    xi, w = oracle.gll(p)
    Q = np.diag(w) @ oracle.diff_matrix(p)
    B = np.zeros((p + 1, p + 1))
    B[0, 0], B[p, p] = -1.0, 1.0
    np.testing.assert_allclose(Q + Q.T, B, atol=1e-13)


def test_cell_matrix_worked_example(golden):
    rows = {r[0][0]: r[1] for r in golden("cell_p1.txt")}
    P = oracle.Problem(dim=1, n=(1,), lo=(0.0,), hi=(1.0,), degree=1,
                       system=oracle.ADVECTION, lam=2.0, dt=2.0)
    A = oracle.cell_matrix(P, 0)              # V = +2
    np.testing.assert_allclose(A.reshape(-1), rows["A"], atol=1e-15)
    g = np.linalg.solve(A, np.array([2.0, 0.0]))
    np.testing.assert_allclose(g, rows["g"], atol=1e-15)
    # the opposite velocity is the mirror image of the same block
    Am = oracle.cell_matrix(P, 1)
    np.testing.assert_allclose(Am, A[::-1, ::-1], atol=1e-15)


@pytest.mark.parametrize("dim,p", [(2, 1), (2, 2), (3, 1)])
def test_axis_velocity_block_is_kronecker(dim, p):
    # V = lambda e_x: faces normal to the other axes carry no flux (V.N = 0),
    # so the cell block is (1D block along x) (x) (transverse mass).
    n = (1,) * dim
    P = oracle.Problem(dim=dim, n=n, lo=(0.0,) * dim, hi=(1.0,) * dim, degree=p,
                       system=oracle.ADVECTION, lam=1.7, dt=0.9)
    P1 = oracle.Problem(dim=1, n=(1,), lo=(0.0,), hi=(1.0,), degree=p,
                        system=oracle.ADVECTION, lam=1.7, dt=0.9)
    _, w = oracle.gll(p)
    A1 = oracle.cell_matrix(P1, 0)
    T = np.diag(w)
    want = A1
    for _ in range(dim - 1):
        want = np.kron(T, want)
    np.testing.assert_allclose(oracle.cell_matrix(P, 0), want, atol=1e-14)
