/*
 * kin_oracle.c -- plain FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).
 *
 * What it computes, in the paper's order (arXiv:2212.11010):
 *   Sec. 2.2   kinetic algorithm: F_k = M_k(W0) initially; per step a free
 *              transport of every population over dt, then W = sum_k F_k and
 *              the over-relaxation F_k <- omega M_k(W) + (1 - omega) F_k
 *              (eq. over_relaxation).
 *   Sec. 3.1   the transport of one population is the implicit upwind DG
 *              scheme of eq. dg_imp; the paper uses Crank-Nicolson in time,
 *              written here as the implicit half step f* over tau = dt/2
 *              followed by f^{n+1} = 2 f* - f^n (algebraically the CN step).
 *   Sec. 3.2   the implicit system is solved cell by cell in downwind
 *              (topological) order, every local system being a small dense
 *              solve whose inflow data are already known.
 *   Sec. 5.1   with subdomains, eq. ibvp: iteration p sweeps every subdomain
 *              with the inflow on its upwind boundary taken from the
 *              neighbour's iterate p-1; iterate 0 is the data at t^n.
 *
 * Nothing here is blocked, fused or reordered beyond that description: every
 * cell assembles its weak-form right-hand side and solves its local system
 * with an LU factorisation (the local matrix is the same for every cell of a
 * uniform Cartesian mesh, so it is factorised once per population).
 *
 * Readings where the paper is silent (also listed in the design notes):
 *   - Cartesian cells with tensor-product Gauss-Lobatto nodes and collocated
 *     quadrature (lumped mass) replace the paper's tetrahedra.
 *   - 2d velocities +-lambda e_a with M_{a,+-} = W/(2d) +- Q^a(W)/(2 lambda),
 *     which satisfies both moment conditions of eq. maxwell_def.
 *   - On a periodic domain a subdomain's face at its own box boundary is an
 *     interface face even when the neighbour across it is itself (one
 *     subdomain couples to itself through the periodic wrap).
 *   - Inflow boundaries (axes with inflow[a] = 1): the paper prescribes the
 *     solution on the domain boundary (Sec. 6.2) and upwinds with the cell
 *     across each face (eq. dg_imp); at a domain boundary the value across
 *     the face is the Maxwellian M_k(Wb) of the face's boundary state.  It is
 *     data, the same in every subdomain iteration, and such faces are not
 *     interfaces (no mass defect).
 *
 * Threads (OpenMP, when the library is built with it): within one
 * subdomain iteration the subdomains are independent (every inflow across a
 * subdomain boundary comes from the previous iterate), so the loop over
 * subdomains runs in parallel -- the paper's own subdomain parallelism of
 * Sec. 5.1 -- and the pointwise loops (initialisation, moments, relaxation)
 * run in parallel over nodes.  Each cell's arithmetic is the same whatever
 * the thread count, so results are bitwise independent of it.
 *
 * parity pinned: see tests/test_oracle_*.py (closed forms, dense global
 * assembly, dense block-Jacobi assembly, conservation, exact solutions).
 */
#include "kin_oracle.h"

#define _USE_MATH_DEFINES
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define KO_MAXP 4
#define KO_MAXNP (KO_MAXP + 1)
#define KO_MAXNN (KO_MAXNP * KO_MAXNP * KO_MAXNP)

/* ------------------------------------------------------------------ */
/* problem bookkeeping                                                */
/* ------------------------------------------------------------------ */

static int check_problem(const ko_problem* P)
{
    if (!P) return -1;
    if (P->dim < 1 || P->dim > 3) return -2;
    if (P->degree < 1 || P->degree > KO_MAXP) return -3;
    if (P->system != KO_ADVECTION && P->system != KO_EULER && P->system != KO_MAXWELL) return -4;
    if (P->system == KO_MAXWELL && (P->dim != 3 || !(P->sigma >= 0.0))) return -4;
    for (int a = 0; a < 3; ++a) {
        if (a < P->dim) {
            if (P->n[a] < 1 || P->tiles[a] < 1 || P->n[a] % P->tiles[a]) return -5;
            if (!(P->hi[a] > P->lo[a])) return -6;
        } else if (P->n[a] != 1 || P->tiles[a] != 1) {
            return -7;
        }
    }
    if (!(P->lambda > 0) || !(P->dt > 0)) return -8;
    if (P->iters < 0) return -9;
    if (P->velset != KO_AXIS && P->velset != KO_SIMPLEX) return -10;
    for (int a = 0; a < 3; ++a) {
        if (P->inflow[a] != 0 && P->inflow[a] != 1) return -11;
        if (P->inflow[a] && (a >= P->dim || P->velset != KO_AXIS)) return -11;
    }
    return 0;
}

int ko_num_vars(const ko_problem* P)
{
    if (P->system == KO_MAXWELL) return 6;
    return P->system == KO_EULER ? P->dim + 2 : 1;
}
int ko_num_vel(const ko_problem* P)
{
    return (P->velset == KO_SIMPLEX && P->dim > 1) ? P->dim + 1 : 2 * P->dim;
}

static int nodes_per_axis(const ko_problem* P, int a) { return a < P->dim ? P->degree + 1 : 1; }

static int nodes_per_cell(const ko_problem* P)
{
    int nn = 1;
    for (int a = 0; a < P->dim; ++a) nn *= P->degree + 1;
    return nn;
}

static size_t num_cells(const ko_problem* P) { return (size_t)P->n[0] * P->n[1] * P->n[2]; }

size_t ko_num_nodes(const ko_problem* P) { return num_cells(P) * (size_t)nodes_per_cell(P); }

static double cell_size(const ko_problem* P, int a)
{
    return a < P->dim ? (P->hi[a] - P->lo[a]) / P->n[a] : 1.0;
}

/* ------------------------------------------------------------------ */
/* Gauss-Lobatto nodes and the Lagrange differentiation matrix         */
/* ------------------------------------------------------------------ */

/* Legendre polynomial P_n(x) by the three-term recurrence. */
static double legendre(int n, double x, double* pm1)
{
    double p0 = 1.0, p1 = x;
    if (n == 0) { if (pm1) *pm1 = 0.0; return 1.0; }
    for (int k = 1; k < n; ++k) {
        double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
    }
    if (pm1) *pm1 = p0;
    return p1;
}

/* GLL nodes: x = +-1 and the roots of P_p'(x), found by Newton iteration on
 * (1 - x^2) P_p'(x) = p (P_{p-1} - x P_p), whose derivative is -p(p+1) P_p
 * (Legendre equation).  Weights 2 / (p (p+1) P_p(x_j)^2).  Mapped to [0,1]. */
int ko_gll(int p, double* xi, double* w)
{
    if (p < 1 || p > KO_MAXP || !xi || !w) return -1;
    double x[KO_MAXNP];
    for (int j = 0; j <= p; ++j) {
        double t = -cos(M_PI * j / p);
        if (j > 0 && j < p) {
            for (int it = 0; it < 100; ++it) {
                double pm1;
                double pp = legendre(p, t, &pm1);
                double dt = (pm1 - t * pp) / ((p + 1.0) * pp);
                t += dt;
                if (fabs(dt) < 1e-16) break;
            }
        }
        x[j] = t;
    }
    for (int j = 0; j <= p; ++j) {
        double pp = legendre(p, x[j], NULL);
        xi[j] = 0.5 * (x[j] + 1.0);
        w[j] = 0.5 * 2.0 / (p * (p + 1.0) * pp * pp);
    }
    xi[0] = 0.0;
    xi[p] = 1.0;
    return 0;
}

/* l_j'(x) = sum_{m != j} 1/(xi_j - xi_m) prod_{k != j, m} (x - xi_k)/(xi_j - xi_k) */
int ko_diff_matrix(int p, double* D)
{
    double xi[KO_MAXNP], w[KO_MAXNP];
    if (ko_gll(p, xi, w)) return -1;
    int np = p + 1;
    for (int i = 0; i < np; ++i) {
        for (int j = 0; j < np; ++j) {
            double s = 0.0;
            for (int m = 0; m < np; ++m) {
                if (m == j) continue;
                double prod = 1.0 / (xi[j] - xi[m]);
                for (int k = 0; k < np; ++k) {
                    if (k == j || k == m) continue;
                    prod *= (xi[i] - xi[k]) / (xi[j] - xi[k]);
                }
                s += prod;
            }
            D[i * np + j] = s;
        }
    }
    return 0;
}

/* node multi-index of local node id (x fastest) */
static void node_index(const ko_problem* P, int id, int ix[3])
{
    for (int a = 0; a < 3; ++a) {
        int na = nodes_per_axis(P, a);
        ix[a] = id % na;
        id /= na;
    }
}

int ko_node_coords(const ko_problem* P, double* xyz)
{
    if (check_problem(P) || !xyz) return -1;
    double xi[KO_MAXNP], w[KO_MAXNP];
    ko_gll(P->degree, xi, w);
    int nn = nodes_per_cell(P);
    size_t node = 0;
    for (int cz = 0; cz < P->n[2]; ++cz)
        for (int cy = 0; cy < P->n[1]; ++cy)
            for (int cx = 0; cx < P->n[0]; ++cx) {
                int c[3] = {cx, cy, cz};
                for (int id = 0; id < nn; ++id) {
                    int ix[3];
                    node_index(P, id, ix);
                    for (int a = 0; a < 3; ++a)
                        xyz[3 * node + a] = a < P->dim
                            ? P->lo[a] + (c[a] + xi[ix[a]]) * cell_size(P, a) : 0.0;
                    ++node;
                }
            }
    return 0;
}

/* ------------------------------------------------------------------ */
/* physical flux and Maxwellians                                       */
/* ------------------------------------------------------------------ */

/* Q^a(W).  Scalar advection: a_a u.  Euler (gamma law):
 * W = (rho, rho u_1..rho u_d, E), p = (gamma-1)(E - |rho u|^2 / (2 rho)),
 * Q^a = (rho u_a, rho u_a u_b + p delta_ab, (E + p) u_a). */
int ko_flux(const ko_problem* P, const double* W, int axis, double* Q)
{
    if (axis < 0 || axis >= P->dim) return -1;
    if (P->system == KO_ADVECTION) {
        Q[0] = P->adv[axis] * W[0];
        return 0;
    }
    if (P->system == KO_MAXWELL) {
        /* Sec. 6.1.1: Q(W, N) = (-N x H, N x E) with N = e_axis; the cross
         * product N x v written component by component */
        const double* E = W;
        const double* H = W + 3;
        double NxE[3] = {0, 0, 0}, NxH[3] = {0, 0, 0};
        const int i = axis, j = (axis + 1) % 3, k = (axis + 2) % 3;
        /* e_i x v = e_i x (v_j e_j + v_k e_k) = v_j e_k - v_k e_j */
        NxE[k] = E[j];
        NxE[j] = -E[k];
        NxH[k] = H[j];
        NxH[j] = -H[k];
        (void)i;
        for (int c = 0; c < 3; ++c) {
            Q[c] = -NxH[c];
            Q[3 + c] = NxE[c];
        }
        return 0;
    }
    int d = P->dim;
    double rho = W[0];
    double ke = 0.0;
    for (int b = 0; b < d; ++b) ke += W[1 + b] * W[1 + b];
    ke *= 0.5 / rho;
    double E = W[1 + d];
    double pr = (P->gamma - 1.0) * (E - ke);
    double ua = W[1 + axis] / rho;
    Q[0] = W[1 + axis];
    for (int b = 0; b < d; ++b) Q[1 + b] = W[1 + b] * ua + (b == axis ? pr : 0.0);
    Q[1 + d] = (E + pr) * ua;
    return 0;
}

static void velocity(const ko_problem* P, int k, double V[3])
{
    V[0] = V[1] = V[2] = 0.0;
    if (P->velset == KO_SIMPLEX && P->dim == 2) {
        /* D2Q3, Sec. 2.4: V_k = lambda (cos(2 k pi / 3), sin(2 k pi / 3)) */
        V[0] = P->lambda * cos(2.0 * M_PI * k / 3.0);
        V[1] = P->lambda * sin(2.0 * M_PI * k / 3.0);
        return;
    }
    if (P->velset == KO_SIMPLEX && P->dim == 3) {
        /* D3Q4, Sec. 6.1.3: (l,l,l), (l,-l,-l), (-l,l,-l), (-l,-l,l) */
        static const double s[4][3] = {{1, 1, 1}, {1, -1, -1}, {-1, 1, -1}, {-1, -1, 1}};
        for (int a = 0; a < 3; ++a) V[a] = P->lambda * s[k][a];
        return;
    }
    V[k / 2] = (k % 2 == 0) ? P->lambda : -P->lambda;
}

int ko_velocity(const ko_problem* P, int k, double* V)
{
    if (check_problem(P) || k < 0 || k >= ko_num_vel(P) || !V) return -1;
    velocity(P, k, V);
    return 0;
}

static int lu_factor(int n, double* A, int* piv);
static void lu_solve(int n, const double* LU, const int* piv, double* b);

/* Axis sets: M_{k=2a+s}(W) = W/(2d) + (s ? -1 : +1) Q^a(W)/(2 lambda), so that
 * sum_k M_k = W and sum_k V_k^a M_k = lambda (M_{2a} - M_{2a+1}) = Q^a.
 * Simplex sets: eq. maxwell_def is a square system for the d + 1 unknowns of
 * every variable, rows (sum_k M_k, sum_k V_k^1 M_k, ..., sum_k V_k^d M_k)
 * = (W, Q^1, ..., Q^d); it is solved here by LU. */
int ko_maxwellian(const ko_problem* P, const double* W, double* M)
{
    int m = ko_num_vars(P), d = P->dim, nv = ko_num_vel(P);
    double Q[3][8];
    for (int a = 0; a < d; ++a) ko_flux(P, W, a, Q[a]);
    if (nv == 2 * d) {
        for (int a = 0; a < d; ++a)
            for (int v = 0; v < m; ++v) {
                M[(2 * a) * m + v] = W[v] / (2.0 * d) + Q[a][v] / (2.0 * P->lambda);
                M[(2 * a + 1) * m + v] = W[v] / (2.0 * d) - Q[a][v] / (2.0 * P->lambda);
            }
        return 0;
    }
    double A[16], V[3];
    int piv[4];
    for (int k = 0; k < nv; ++k) {
        velocity(P, k, V);
        A[0 * nv + k] = 1.0;
        for (int a = 0; a < d; ++a) A[(1 + a) * nv + k] = V[a];
    }
    if (lu_factor(nv, A, piv)) return -2;
    for (int v = 0; v < m; ++v) {
        double b[4];
        b[0] = W[v];
        for (int a = 0; a < d; ++a) b[1 + a] = Q[a][v];
        lu_solve(nv, A, piv, b);
        for (int k = 0; k < nv; ++k) M[k * m + v] = b[k];
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* local DG operator of eq. dg_imp on one Cartesian cell               */
/* ------------------------------------------------------------------ */

/* Quadrature weight of a volume node: |L| prod_a w_{i_a}. */
static double vol_weight(const ko_problem* P, const double* w, int id)
{
    int ix[3];
    node_index(P, id, ix);
    double q = 1.0;
    for (int a = 0; a < P->dim; ++a) q *= cell_size(P, a) * w[ix[a]];
    return q;
}

/* Quadrature weight of a node lying on a face normal to axis a:
 * |face| prod_{b != a} w_{i_b}. */
static double face_weight(const ko_problem* P, const double* w, int id, int a)
{
    int ix[3];
    node_index(P, id, ix);
    double q = 1.0;
    for (int b = 0; b < P->dim; ++b)
        if (b != a) q *= cell_size(P, b) * w[ix[b]];
    return q;
}

/* Implicit cell matrix for velocity k over tau = dt/2, from eq. dg_imp with
 * the test function psi_i:
 *   A f  =  M f  -  tau * int f V.grad(psi_i)  +  tau * sum_{outflow faces}
 *           int f_L (V.N)_+ psi_i
 * with every integral taken by the collocated GLL quadrature. */
int ko_cell_matrix(const ko_problem* P, int k, double* A)
{
    if (check_problem(P) || k < 0 || k >= ko_num_vel(P)) return -1;
    int p = P->degree, np = p + 1, nn = nodes_per_cell(P), d = P->dim;
    double xi[KO_MAXNP], w[KO_MAXNP], D[KO_MAXNP * KO_MAXNP], V[3];
    ko_gll(p, xi, w);
    ko_diff_matrix(p, D);
    velocity(P, k, V);
    double tau = 0.5 * P->dt;
    memset(A, 0, sizeof(double) * nn * nn);
    for (int i = 0; i < nn; ++i) {
        int ii[3];
        node_index(P, i, ii);
        A[i * nn + i] += vol_weight(P, w, i);
        /* volume term: - tau * sum_q W_q f_q (V . grad psi_i)(x_q) */
        for (int q = 0; q < nn; ++q) {
            int iq[3];
            node_index(P, q, iq);
            double vg = 0.0;
            for (int a = 0; a < d; ++a) {
                int same = 1;
                for (int b = 0; b < d; ++b)
                    if (b != a && ii[b] != iq[b]) same = 0;
                if (!same) continue;
                /* d psi_i/dx_a at x_q = l'_{i_a}(xi_{q_a}) / h_a */
                vg += V[a] * D[iq[a] * np + ii[a]] / cell_size(P, a);
            }
            A[i * nn + q] -= tau * vol_weight(P, w, q) * vg;
        }
        /* outflow faces: (V.N)_+ > 0 */
        for (int a = 0; a < d; ++a) {
            for (int side = -1; side <= 1; side += 2) {
                double vn = side * V[a];
                int on_face = (side < 0) ? (ii[a] == 0) : (ii[a] == p);
                if (vn > 0 && on_face) A[i * nn + i] += tau * vn * face_weight(P, w, i, a);
            }
        }
    }
    return 0;
}

/* Dense LU with partial pivoting (a plain library-style primitive). */
static int lu_factor(int n, double* A, int* piv)
{
    for (int c = 0; c < n; ++c) {
        int r = c;
        for (int i = c + 1; i < n; ++i)
            if (fabs(A[i * n + c]) > fabs(A[r * n + c])) r = i;
        if (A[r * n + c] == 0.0) return -1;
        piv[c] = r;
        if (r != c)
            for (int j = 0; j < n; ++j) {
                double t = A[c * n + j];
                A[c * n + j] = A[r * n + j];
                A[r * n + j] = t;
            }
        for (int i = c + 1; i < n; ++i) {
            double l = A[i * n + c] / A[c * n + c];
            A[i * n + c] = l;
            for (int j = c + 1; j < n; ++j) A[i * n + j] -= l * A[c * n + j];
        }
    }
    return 0;
}

static void lu_solve(int n, const double* LU, const int* piv, double* b)
{
    for (int c = 0; c < n; ++c) {
        double t = b[c];
        b[c] = b[piv[c]];
        b[piv[c]] = t;
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < i; ++j) b[i] -= LU[i * n + j] * b[j];
    for (int i = n - 1; i >= 0; --i) {
        for (int j = i + 1; j < n; ++j) b[i] -= LU[i * n + j] * b[j];
        b[i] /= LU[i * n + i];
    }
}

/* ------------------------------------------------------------------ */
/* transport of one population: downwind sweeps + subdomain iteration  */
/* ------------------------------------------------------------------ */

static size_t cell_id(const ko_problem* P, const int c[3])
{
    return ((size_t)c[2] * P->n[1] + c[1]) * P->n[0] + c[0];
}

/* neighbour node across the face normal to axis a: the node index along a
 * flips between 0 and p, the others stay. */
static int across(const ko_problem* P, int id, int a)
{
    int ix[3];
    node_index(P, id, ix);
    ix[a] = (ix[a] == 0) ? P->degree : 0;
    int np = P->degree + 1, r = 0;
    for (int b = P->dim - 1; b >= 0; --b) r = r * np + ix[b];
    return r;
}

typedef struct {
    const ko_problem* P;
    int k;
    double V[3];
    double w[KO_MAXNP];
    double LU[KO_MAXNN * KO_MAXNN];
    int piv[KO_MAXNN];
    int nn;
    int L[3];                     /* subdomain extent in cells              */
    double volw[KO_MAXNN];        /* volume quadrature weight of each node  */
    double facew[3][KO_MAXNN];    /* face quadrature weight, face normal a  */
    int face_lo[3][KO_MAXNN];     /* node lies on the face at x_a = lower   */
    int face_hi[3][KO_MAXNN];     /* node lies on the face at x_a = upper   */
    int acr[3][KO_MAXNN];         /* matching node of the neighbour cell    */
    double bval[3][2];            /* inflow value M_k(Wb)[v] of face (axis, lower/upper) */
} pop_ctx;

static void fill_node_tables(pop_ctx* C)
{
    const ko_problem* P = C->P;
    for (int i = 0; i < C->nn; ++i) {
        int ix[3];
        node_index(P, i, ix);
        C->volw[i] = vol_weight(P, C->w, i);
        for (int a = 0; a < 3; ++a) {
            C->facew[a][i] = a < P->dim ? face_weight(P, C->w, i, a) : 0.0;
            C->face_lo[a][i] = a < P->dim && ix[a] == 0;
            C->face_hi[a][i] = a < P->dim && ix[a] == P->degree;
            C->acr[a][i] = a < P->dim ? across(P, i, a) : i;
        }
    }
}

/* Solve one cell: rhs = M f^n + tau sum_{inflow faces} |V.N| int f_up psi_i,
 * with f_up from the current iterate inside the subdomain and from the
 * previous iterate across the subdomain boundary (eq. ibvp3). */
static void solve_cell(const pop_ctx* C, const int c[3], const double* fn,
                       const double* prev, double* cur)
{
    const ko_problem* P = C->P;
    int nn = C->nn, d = P->dim;
    double tau = 0.5 * P->dt;
    size_t base = cell_id(P, c) * nn;
    double b[KO_MAXNN];
    for (int i = 0; i < nn; ++i) b[i] = C->volw[i] * fn[base + i];
    for (int a = 0; a < d; ++a) {
        for (int side = -1; side <= 1; side += 2) {
            double vn = side * C->V[a];
            if (!(vn < 0)) continue;              /* inflow faces only */
            int nb[3] = {c[0], c[1], c[2]};
            nb[a] = (c[a] + side + P->n[a]) % P->n[a];
            const int* on_face = (side < 0) ? C->face_lo[a] : C->face_hi[a];
            if (P->inflow[a] && c[a] + side != nb[a]) {
                /* domain boundary: the prescribed Maxwellian */
                const double fb = C->bval[a][side < 0 ? 0 : 1];
                for (int i = 0; i < nn; ++i)
                    if (on_face[i]) b[i] += tau * (-vn) * C->facew[a][i] * fb;
                continue;
            }
            int boundary = (side < 0) ? (c[a] % C->L[a] == 0)
                                      : (c[a] % C->L[a] == C->L[a] - 1);
            const double* src = boundary ? prev : cur;
            size_t nbase = cell_id(P, nb) * nn;
            for (int i = 0; i < nn; ++i) {
                if (!on_face[i]) continue;
                b[i] += tau * (-vn) * C->facew[a][i] * src[nbase + C->acr[a][i]];
            }
        }
    }
    lu_solve(nn, C->LU, C->piv, b);
    for (int i = 0; i < nn; ++i) cur[base + i] = b[i];
}

/* Visit the cells of subdomain s in downwind order: every axis is traversed
 * in the direction of V_a (ascending when V_a = 0), which is a topological
 * order of the oriented cell graph (Sec. 3.2). */
static void sweep_subdomain(const pop_ctx* C, const int s[3], const double* fn,
                            const double* prev, double* cur)
{
    int lo[3], step[3], cnt[3];
    for (int a = 0; a < 3; ++a) {
        cnt[a] = C->L[a];
        if (C->V[a] < 0) {
            lo[a] = s[a] * C->L[a] + C->L[a] - 1;
            step[a] = -1;
        } else {
            lo[a] = s[a] * C->L[a];
            step[a] = 1;
        }
    }
    for (int kz = 0; kz < cnt[2]; ++kz)
        for (int ky = 0; ky < cnt[1]; ++ky)
            for (int kx = 0; kx < cnt[0]; ++kx) {
                int c[3] = {lo[0] + step[0] * kx, lo[1] + step[1] * ky, lo[2] + step[2] * kz};
                solve_cell(C, c, fn, prev, cur);
            }
}

/* Mass defect of the final iterate: sum over the inflow faces that lie on a
 * subdomain boundary of dt |V.N| int (f_up^{K-1} - f_up^{K}). */
static double interface_defect(const pop_ctx* C, const double* prev, const double* cur)
{
    const ko_problem* P = C->P;
    double acc = 0.0;
    int nn = C->nn, d = P->dim;
    for (int cz = 0; cz < P->n[2]; ++cz)
        for (int cy = 0; cy < P->n[1]; ++cy)
            for (int cx = 0; cx < P->n[0]; ++cx) {
                int c[3] = {cx, cy, cz};
                for (int a = 0; a < d; ++a)
                    for (int side = -1; side <= 1; side += 2) {
                        double vn = side * C->V[a];
                        if (!(vn < 0)) continue;
                        int boundary = (side < 0) ? (c[a] % C->L[a] == 0)
                                                  : (c[a] % C->L[a] == C->L[a] - 1);
                        if (!boundary) continue;
                        int nb[3] = {c[0], c[1], c[2]};
                        nb[a] = (c[a] + side + P->n[a]) % P->n[a];
                        if (P->inflow[a] && c[a] + side != nb[a]) continue;   /* domain boundary */
                        size_t nbase = cell_id(P, nb) * nn;
                        const int* on_face = (side < 0) ? C->face_lo[a] : C->face_hi[a];
                        for (int i = 0; i < nn; ++i) {
                            if (!on_face[i]) continue;
                            int j = C->acr[a][i];
                            acc += P->dt * (-vn) * C->facew[a][i] * (prev[nbase + j] - cur[nbase + j]);
                        }
                    }
            }
    return acc;
}

static int transport_population(const ko_problem* P, int k, int v, double* f, double* defect,
                                int* iters_done)
{
    pop_ctx C;
    double xi[KO_MAXNP];
    C.P = P;
    C.k = k;
    for (int a = 0; a < 3; ++a)
        for (int sd = 0; sd < 2; ++sd) {
            C.bval[a][sd] = 0.0;
            if (a < P->dim && P->inflow[a]) {
                double M[4 * KO_MAXM * 2];
                int rc = ko_maxwellian(P, P->Wb[a][sd], M);
                if (rc) return rc;
                C.bval[a][sd] = M[k * ko_num_vars(P) + v];
            }
        }
    C.nn = nodes_per_cell(P);
    velocity(P, k, C.V);
    ko_gll(P->degree, xi, C.w);
    for (int a = 0; a < 3; ++a) C.L[a] = P->n[a] / P->tiles[a];
    fill_node_tables(&C);
    ko_cell_matrix(P, k, C.LU);
    if (lu_factor(C.nn, C.LU, C.piv)) return -10;

    size_t nodes = ko_num_nodes(P);
    double* prev = (double*)malloc(sizeof(double) * nodes);
    double* cur = (double*)malloc(sizeof(double) * nodes);
    if (!prev || !cur) { free(prev); free(cur); return -11; }
    /* iterate 0: f_i^0(X, t) = f^0(X), i.e. the data at t^n (eq. ibvp2) */
    memcpy(prev, f, sizeof(double) * nodes);
    memcpy(cur, f, sizeof(double) * nodes);

    int maxit = P->iters > 0 ? P->iters : 100000;
    int it;
    const int nsub = P->tiles[0] * P->tiles[1] * P->tiles[2];
    for (it = 1; it <= maxit; ++it) {
        /* the subdomains of one iteration are independent (eq. ibvp) */
#pragma omp parallel for schedule(dynamic, 1)
        for (int si = 0; si < nsub; ++si) {
            int s[3] = {si % P->tiles[0], (si / P->tiles[0]) % P->tiles[1], si / (P->tiles[0] * P->tiles[1])};
            sweep_subdomain(&C, s, f, prev, cur);
        }
        if (P->iters == 0) {
            double dmax = 0.0, fmax = 0.0;
            for (size_t i = 0; i < nodes; ++i) {
                double e = fabs(cur[i] - prev[i]);
                if (e > dmax) dmax = e;
                if (fabs(cur[i]) > fmax) fmax = fabs(cur[i]);
            }
            if (dmax <= 1e-15 * (fmax > 0 ? fmax : 1.0)) break;
        }
        if (it < maxit) memcpy(prev, cur, sizeof(double) * nodes);
    }
    if (it > maxit) it = maxit;
    if (iters_done) *iters_done = it;
    if (defect) *defect = interface_defect(&C, prev, cur);
    /* Crank-Nicolson: f^{n+1} = 2 f* - f^n */
    for (size_t i = 0; i < nodes; ++i) f[i] = 2.0 * cur[i] - f[i];
    free(prev);
    free(cur);
    return 0;
}

int ko_transport(const ko_problem* P, double* f, double* defect, int* iters_done)
{
    int rc = check_problem(P);
    if (rc) return rc;
    if (!f) return -1;
    int m = ko_num_vars(P), nv = ko_num_vel(P);
    size_t nodes = ko_num_nodes(P);
    if (defect)
        for (int v = 0; v < m; ++v) defect[v] = 0.0;
    int maxdone = 0;
    for (int k = 0; k < nv; ++k)
        for (int v = 0; v < m; ++v) {
            double dfc = 0.0;
            int done = 0;
            rc = transport_population(P, k, v, f + (size_t)(k * m + v) * nodes, &dfc, &done);
            if (rc) return rc;
            if (defect) defect[v] += dfc;
            if (done > maxdone) maxdone = done;
        }
    if (iters_done) *iters_done = maxdone;
    return 0;
}

/* ------------------------------------------------------------------ */
/* moments, relaxation, initialisation, mass                           */
/* ------------------------------------------------------------------ */

int ko_moments(const ko_problem* P, const double* f, double* W)
{
    if (check_problem(P) || !f || !W) return -1;
    return ko_moments_n(P, f, W, ko_num_nodes(P));
}

int ko_moments_n(const ko_problem* P, const double* f, double* W, size_t nodes)
{
    if (check_problem(P) || !f || !W) return -1;
    int m = ko_num_vars(P), nv = ko_num_vel(P);
    for (int v = 0; v < m; ++v) {
#pragma omp parallel for schedule(static)
        for (size_t i = 0; i < nodes; ++i) {
            double s = 0.0;
            for (int k = 0; k < nv; ++k) s += f[(size_t)(k * m + v) * nodes + i];
            W[(size_t)v * nodes + i] = s;
        }
    }
    return 0;
}

int ko_relax(const ko_problem* P, double* f)
{
    if (check_problem(P) || !f) return -1;
    return ko_relax_n(P, f, ko_num_nodes(P));
}

int ko_relax_n(const ko_problem* P, double* f, size_t nodes)
{
    if (check_problem(P) || !f) return -1;
    int m = ko_num_vars(P), nv = ko_num_vel(P);
#pragma omp parallel for schedule(static)
    for (size_t i = 0; i < nodes; ++i) {
        double W[8], M[64];
        for (int v = 0; v < m; ++v) {
            double s = 0.0;
            for (int k = 0; k < nv; ++k) s += f[(size_t)(k * m + v) * nodes + i];
            W[v] = s;
        }
        ko_maxwellian(P, W, M);
        if (P->system == KO_MAXWELL) {
            /* source step on W (Crank-Nicolson in time), then relaxation of
             * the non-equilibrium part about the equilibrium of the new W */
            const double mu = (1.0 - 0.5 * P->sigma * P->dt) / (1.0 + 0.5 * P->sigma * P->dt);
            double Wp[8], Mp[64];
            for (int v = 0; v < m; ++v) Wp[v] = v < 3 ? mu * W[v] : W[v];
            ko_maxwellian(P, Wp, Mp);
            for (int pop = 0; pop < nv * m; ++pop) {
                double* fp = f + (size_t)pop * nodes + i;
                *fp = Mp[pop] + (1.0 - P->omega) * (*fp - M[pop]);
            }
            continue;
        }
        for (int pop = 0; pop < nv * m; ++pop) {
            double* fp = f + (size_t)pop * nodes + i;
            *fp = P->omega * M[pop] + (1.0 - P->omega) * (*fp);
        }
    }
    return 0;
}

int ko_init(const ko_problem* P, const double* W0, double* f)
{
    if (check_problem(P) || !W0 || !f) return -1;
    return ko_init_n(P, W0, f, ko_num_nodes(P));
}

int ko_init_n(const ko_problem* P, const double* W0, double* f, size_t nodes)
{
    if (check_problem(P) || !W0 || !f) return -1;
    int m = ko_num_vars(P), nv = ko_num_vel(P);
#pragma omp parallel for schedule(static)
    for (size_t i = 0; i < nodes; ++i) {
        double W[8], M[64];
        for (int v = 0; v < m; ++v) W[v] = W0[(size_t)v * nodes + i];
        ko_maxwellian(P, W, M);
        for (int pop = 0; pop < nv * m; ++pop) f[(size_t)pop * nodes + i] = M[pop];
    }
    return 0;
}

int ko_step(const ko_problem* P, double* f, int nsteps)
{
    int rc = check_problem(P);
    if (rc) return rc;
    if (nsteps < 0) return -1;
    for (int s = 0; s < nsteps; ++s) {
        rc = ko_transport(P, f, NULL, NULL);
        if (rc) return rc;
        rc = ko_relax(P, f);
        if (rc) return rc;
    }
    return 0;
}

int ko_mass(const ko_problem* P, const double* W, double* mass)
{
    if (check_problem(P) || !W || !mass) return -1;
    double xi[KO_MAXNP], w[KO_MAXNP];
    ko_gll(P->degree, xi, w);
    int m = ko_num_vars(P), nn = nodes_per_cell(P);
    size_t cells = num_cells(P), nodes = ko_num_nodes(P);
    for (int v = 0; v < m; ++v) {
        double s = 0.0;
        for (size_t c = 0; c < cells; ++c)
            for (int i = 0; i < nn; ++i) s += vol_weight(P, w, i) * W[(size_t)v * nodes + c * nn + i];
        mass[v] = s;
    }
    return 0;
}

int ko_set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
    return omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}
