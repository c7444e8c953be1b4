"""Independent dense restatement of the implicit upwind DG transport for tiny
meshes (test helper; shares nothing with the oracle or the CUDA library).

The global matrix of eq. dg_imp (Sec. 3.1) for one population with constant
velocity V is assembled from the weak form over every (cell, node) degree of
freedom, with Gauss-Lobatto collocation on tensor Cartesian cells.  Here the
GLL rule comes from numpy's Legendre roots plus a moment-matching weight
solve, and the Lagrange derivatives from an inverse Vandermonde matrix - a
different route from the oracle's Newton iteration and product formula.

* ``global_cn``     Crank-Nicolson as (M + tau K) f* = M f^n, f^{n+1} = 2f* - f^n,
                    solved densely: the downwind sweep's fixed point.
* ``block_jacobi``  the subdomain iteration of eq. ibvp in matrix form: the
                    couplings across subdomain-boundary faces (K_out) use the
                    previous iterate, x^0 = f^n, K iterations.

With ``inflow[a] = 1`` axis a is not periodic: a face on the domain boundary
couples to a prescribed boundary value instead of the cell across the wrap.
``assemble_bc`` returns those couplings per face, and the solves take the
boundary values as a known right-hand side.
"""
import numpy as np


def gll_numpy(p):
    c = np.zeros(p + 1)
    c[p] = 1.0
    inner = np.polynomial.legendre.legroots(np.polynomial.legendre.legder(c))
    x = np.concatenate([[-1.0], np.sort(np.real(inner)), [1.0]])
    V = np.vander(x, p + 1, increasing=True).T          # V[k, j] = x_j^k
    rhs = np.array([(1.0 - (-1.0) ** (k + 1)) / (k + 1) for k in range(p + 1)])
    w = np.linalg.solve(V, rhs)
    return 0.5 * (x + 1.0), 0.5 * w


def lagrange_derivative(xi):
    """Dl[i, j] = l_j'(xi_i) from the inverse Vandermonde coefficients."""
    n = len(xi)
    V = np.vander(xi, n, increasing=True)                # V[i, k] = xi_i^k
    C = np.linalg.inv(V)                                 # l_j = sum_k C[k, j] x^k
    Dl = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            Dl[i, j] = sum(k * C[k, j] * xi[i] ** (k - 1) for k in range(1, n))
    return Dl


def assemble(dim, n, lo, hi, p, V, tiles):
    """Return (M, K, Kout): mass (diagonal), full transport operator and the
    part of K that couples across subdomain-boundary faces."""
    M, K, Kout, _ = assemble_bc(dim, n, lo, hi, p, V, tiles, (0, 0, 0))
    return M, K, Kout


def assemble_bc(dim, n, lo, hi, p, V, tiles, inflow):
    """(M, K, Kout, Kb): as ``assemble``, plus Kb[(a, side)], the coupling of
    every node to the boundary value of face (axis a, side -1 lower / +1
    upper) of the axes with inflow[a] = 1, where K has no coupling."""
    xi, w = gll_numpy(p)
    Dl = lagrange_derivative(xi)
    npn = p + 1
    n = tuple(n) + (1,) * (3 - dim)
    tiles = tuple(tiles) + (1,) * (3 - dim)
    h = [(hi[a] - lo[a]) / n[a] for a in range(dim)]
    L = [n[a] // tiles[a] for a in range(3)]
    nn = npn ** dim
    ncell = n[0] * n[1] * n[2]
    N = ncell * nn
    M = np.zeros(N)
    K = np.zeros((N, N))
    Kout = np.zeros((N, N))
    Kb = {}
    inflow = tuple(inflow) + (0,) * (3 - len(inflow))
    vol = np.prod(h)

    def nidx(ix):
        r = 0
        for a in reversed(range(dim)):
            r = r * npn + ix[a]
        return r

    def cidx(c):
        return (c[2] * n[1] + c[1]) * n[0] + c[0]

    nodes = [tuple(int(v) for v in ix) for ix in np.ndindex(*(npn,) * dim)]
    for cz in range(n[2]):
        for cy in range(n[1]):
            for cx in range(n[0]):
                c = (cx, cy, cz)
                base = cidx(c) * nn
                sub = tuple(c[a] // L[a] for a in range(3))
                for ii in nodes:
                    gi = base + nidx(ii)
                    wi = vol * np.prod([w[ii[a]] for a in range(dim)])
                    M[gi] = wi
                    for iq in nodes:
                        gq = base + nidx(iq)
                        wq = vol * np.prod([w[iq[a]] for a in range(dim)])
                        vg = 0.0
                        for a in range(dim):
                            if all(ii[b] == iq[b] for b in range(dim) if b != a):
                                vg += V[a] * Dl[iq[a], ii[a]] / h[a]
                        K[gi, gq] -= wq * vg
                    for a in range(dim):
                        for side in (-1, 1):
                            if ii[a] != (0 if side < 0 else p):
                                continue
                            vn = side * V[a]
                            fw = vol / h[a] * np.prod([w[ii[b]] for b in range(dim) if b != a])
                            if vn > 0:
                                K[gi, gi] += vn * fw
                            elif vn < 0:
                                nb = list(c)
                                raw = c[a] + side
                                if inflow[a] and (raw < 0 or raw >= n[a]):
                                    Kb.setdefault((a, side), np.zeros(N))[gi] += vn * fw
                                    continue
                                nb[a] = raw % n[a]
                                jj = list(ii)
                                jj[a] = p if side < 0 else 0
                                gj = cidx(nb) * nn + nidx(jj)
                                nsub = tuple(nb[b] // L[b] for b in range(3))
                                crosses = (nsub != sub) or raw < 0 or raw >= n[a]
                                K[gi, gj] += vn * fw
                                if crosses:
                                    Kout[gi, gj] += vn * fw
    return M, K, Kout, Kb


def _boundary_rhs(Kb, bvals, N):
    r = np.zeros(N)
    for face, col in (Kb or {}).items():
        r += col * bvals[face]
    return r


def global_cn(M, K, tau, fn, Kb=None, bvals=None):
    A = np.diag(M) + tau * K
    fstar = np.linalg.solve(A, M * fn - tau * _boundary_rhs(Kb, bvals, len(fn)))
    return 2.0 * fstar - fn


def block_jacobi(M, K, Kout, tau, fn, iters, Kb=None, bvals=None):
    Ain = np.diag(M) + tau * (K - Kout)
    rb = tau * _boundary_rhs(Kb, bvals, len(fn))
    x = fn.copy()
    for _ in range(iters):
        x = np.linalg.solve(Ain, M * fn - tau * (Kout @ x) - rb)
    return 2.0 * x - fn
