"""Independent dense restatement of the implicit upwind DG transport on
tetrahedral meshes (test helper; shares nothing with the oracle or the CUDA
library).

eq. dg_imp (Sec. 3.1) with the P1 Lagrange basis of each cell's vertices, for
one population with constant velocity V, assembled over every (cell, node)
unknown.  The route differs from the oracle's on purpose:

* barycentric coordinates from the inverse of the 4 x 4 matrix
  [[1, 1, 1, 1], [x_0, x_1, x_2, x_3]] (the oracle uses cross products);
* the outward normal of face a is -grad(lambda_a) / |grad(lambda_a)| and its
  area 3 |L| |grad(lambda_a)| (the oracle crosses two edges);
* every integral by quadrature -- the 4-point degree-2 rule on the
  tetrahedron and the 3-point edge-midpoint rule on each face -- instead of
  the closed forms.

``global_cn`` solves (M + tau K) f* = M f^n densely (the sweep's fixed
point) and returns f^{n+1} = 2 f* - f^n; ``block_jacobi`` runs the subdomain
iteration of eq. ibvp in matrix form, K iterations from x^0 = f^n with the
couplings across subdomain boundaries on the previous iterate.
"""
import numpy as np

_A4 = 0.5854101966249685
_B4 = 0.1381966011250105
_TET_RULE = [np.array(p) for p in ((_A4, _B4, _B4, _B4), (_B4, _A4, _B4, _B4), (_B4, _B4, _A4, _B4),
                                  (_B4, _B4, _B4, _A4))]          # barycentric points, weight 1/4 each
PARALLEL_TOL = 1e-12


def barycentric(x):
    """(volume, G) with G[a] = grad lambda_a for the vertices x (4, 3)."""
    B = np.vstack([np.ones(4), x.T])                 # B @ lambda = (1, X)
    Binv = np.linalg.inv(B)                          # lambda = Binv @ (1, X)
    return abs(np.linalg.det(B)) / 6.0, Binv[:, 1:]


def cell_operators(x, V):
    """(M, Kv, faces): the mass matrix, the volume term
    Kv[i, j] = -int psi_j V . grad psi_i, and per face a (vn, F) with
    vn = V . N_a and F[i, j] = int_{face a} psi_i psi_j."""
    vol, G = barycentric(x)
    M = np.zeros((4, 4))
    for lam in _TET_RULE:
        M += vol / 4.0 * np.outer(lam, lam)
    Kv = np.zeros((4, 4))
    for i in range(4):
        for j in range(4):
            Kv[i, j] = -(V @ G[i]) * sum(vol / 4.0 * lam[j] for lam in _TET_RULE)
    faces = []
    vmag = np.linalg.norm(V)
    for a in range(4):
        g = G[a]
        normal = -g / np.linalg.norm(g)
        area = 3.0 * vol * np.linalg.norm(g)
        vn = V @ normal
        if abs(vn) <= PARALLEL_TOL * vmag:
            vn = 0.0
        others = [b for b in range(4) if b != a]
        F = np.zeros((4, 4))
        for p, q in ((0, 1), (1, 2), (0, 2)):        # edge midpoints of the face
            lam = np.zeros(4)
            lam[others[p]] = 0.5
            lam[others[q]] = 0.5
            F += area / 3.0 * np.outer(lam, lam)
        faces.append((vn, F))
    return M, Kv, faces


def assemble(mesh_xyz, vid, nbr, sub, V, tau, wrap=None):
    """(A, Mg, Aout): A = M + tau K over all unknowns, Mg the global mass,
    Aout the part of A that couples across subdomain interfaces: faces
    between different subdomains, and faces that cross the periodic
    boundary (wrap[c, a] = 1), where a subdomain couples to itself."""
    n = vid.shape[0]
    N = 4 * n
    A = np.zeros((N, N))
    Mg = np.zeros((N, N))
    Aout = np.zeros((N, N))
    for c in range(n):
        M, Kv, faces = cell_operators(mesh_xyz[c], V)
        sl = slice(4 * c, 4 * c + 4)
        Mg[sl, sl] += M
        A[sl, sl] += M + tau * Kv
        for a, (vn, F) in enumerate(faces):
            if vn > 0:
                A[sl, sl] += tau * vn * F
            elif vn < 0:
                R = nbr[c, a]
                for i in range(4):
                    for j in range(4):
                        if F[i, j] == 0.0:
                            continue
                        jr = int(np.nonzero(vid[R] == vid[c, j])[0][0])
                        val = tau * vn * F[i, j]
                        A[4 * c + i, 4 * R + jr] += val
                        if sub[R] != sub[c] or (wrap is not None and wrap[c, a]):
                            Aout[4 * c + i, 4 * R + jr] += val
    return A, Mg, Aout


def global_cn(A, Mg, fn):
    fstar = np.linalg.solve(A, Mg @ fn)
    return 2.0 * fstar - fn


def block_jacobi(A, Mg, Aout, fn, iters):
    D = A - Aout
    b = Mg @ fn
    x = fn.copy()
    for _ in range(iters):
        x = np.linalg.solve(D, b - Aout @ x)
    return 2.0 * x - fn
