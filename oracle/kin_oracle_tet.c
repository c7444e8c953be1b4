/*
 * kin_oracle_tet.c -- plain FP64 CPU oracle of the kinetic DG transport on
 * tetrahedral meshes (TEST INFRASTRUCTURE ONLY; see kin_oracle.h).
 *
 * What it computes, in the paper's order (arXiv:2212.11010):
 *   Sec. 3.1   eq. dg_imp on tetrahedral cells (n_f = 4 faces) with a nodal
 *              basis: here the P1 Lagrange functions of the four vertices,
 *              every integral exact (mass |L|/20 (1 + delta_ij), volume term
 *              (V . grad psi_i) |L|/4 for every j, face mass
 *              |F|/12 (1 + delta_ij) for the face's three vertices).  The
 *              upwind flux takes the cell's own trace on outflow faces
 *              (V.N > 0) and the neighbour's trace on inflow faces
 *              (V.N < 0); a face with V.N = 0 carries no flux.  Time:
 *              Crank-Nicolson as an implicit half step f* over tau = dt/2
 *              followed by f^{n+1} = 2 f* - f^n.
 *   Sec. 3.2   the cells of each subdomain are visited in a topological
 *              order of the graph whose edges are the faces oriented by V
 *              (an edge from R to L when V enters L across their face),
 *              found by breadth-first search from the cells without an
 *              upwind neighbour in the subdomain (Kahn's algorithm); every
 *              local system is then a dense 4 x 4 solve with known data.
 *   Sec. 5.1   eq. ibvp: iteration p sweeps every subdomain with the inflow
 *              across its boundary taken from the neighbour's iterate p-1;
 *              iterate 0 is the data at t^n.
 *
 * Readings (listed in the design notes): P1 nodal basis at the vertices
 * (the paper does not name its nodal basis); faces with |V.N| <= 1e-12 |V|
 * count as parallel to V (no flux, no graph edge), since a face parallel to
 * V computes to a tiny non-zero V.N in floating point.
 *
 * parity pinned: tests/test_oracle_tet.py (an independent dense global
 * assembly in numpy solved directly and by block Jacobi, constants kept,
 * mass change = interface defect, convergence to the exact translation).
 */
#include "kin_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define KT_PARALLEL_TOL 1e-12

typedef struct {
    double vol;            /* |L|                                        */
    double grad[4][3];     /* grad psi_a                                 */
    double area[4];        /* |F_a|, face a opposite vertex a            */
    double normal[4][3];   /* outward unit normal of face a              */
} tet_geom;

static void sub3(const double* a, const double* b, double* r)
{
    for (int i = 0; i < 3; ++i) r[i] = a[i] - b[i];
}

static void cross3(const double* a, const double* b, double* r)
{
    r[0] = a[1] * b[2] - a[2] * b[1];
    r[1] = a[2] * b[0] - a[0] * b[2];
    r[2] = a[0] * b[1] - a[1] * b[0];
}

static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* Volume, basis gradients, face areas and outward normals of one cell. */
static int cell_geometry(const ko_tetmesh* T, int c, tet_geom* g)
{
    const double* x = T->xyz + (size_t)c * 12;
    double e[3][3];
    for (int b = 0; b < 3; ++b) sub3(x + 3 * (b + 1), x, e[b]);
    /* J has columns e[0], e[1], e[2]; barycentric coordinates lambda_{b+1}
     * are the rows of J^{-1} applied to (X - x_0) */
    double c01[3], c12[3], c20[3];
    cross3(e[1], e[2], c12);
    cross3(e[2], e[0], c20);
    cross3(e[0], e[1], c01);
    const double det = dot3(e[0], c12);
    if (!(fabs(det) > 0)) return -1;
    g->vol = fabs(det) / 6.0;
    for (int i = 0; i < 3; ++i) {
        g->grad[1][i] = c12[i] / det;    /* rows of J^{-1}: (e1 x e2, e2 x e0, e0 x e1) / det */
        g->grad[2][i] = c20[i] / det;
        g->grad[3][i] = c01[i] / det;
        g->grad[0][i] = -(g->grad[1][i] + g->grad[2][i] + g->grad[3][i]);
    }
    for (int a = 0; a < 4; ++a) {
        int v[3], k = 0;
        for (int b = 0; b < 4; ++b)
            if (b != a) v[k++] = b;
        double u[3], w[3], n[3], to_a[3];
        sub3(x + 3 * v[1], x + 3 * v[0], u);
        sub3(x + 3 * v[2], x + 3 * v[0], w);
        cross3(u, w, n);
        const double len = sqrt(dot3(n, n));
        g->area[a] = 0.5 * len;
        sub3(x + 3 * a, x + 3 * v[0], to_a);
        const double s = dot3(n, to_a) > 0 ? -1.0 : 1.0;   /* away from vertex a */
        for (int i = 0; i < 3; ++i) g->normal[a][i] = s * n[i] / len;
    }
    return 0;
}

/* V.N_a with faces (nearly) parallel to V set to exactly zero. */
static double face_flux(const double* V, const tet_geom* g, int a)
{
    const double vn = dot3(V, g->normal[a]);
    const double vmag = sqrt(dot3(V, V));
    return fabs(vn) <= KT_PARALLEL_TOL * vmag ? 0.0 : vn;
}

int ko_tet_cell_matrix(const ko_problem* P, const ko_tetmesh* T, int c, int k, double* A, double* M,
                       double* vn_area)
{
    if (!P || !T || c < 0 || c >= T->ncells || P->dim != 3 || k < 0 || k >= ko_num_vel(P)) return -1;
    tet_geom g;
    if (cell_geometry(T, c, &g)) return -2;
    double V[3];
    ko_velocity(P, k, V);
    const double tau = 0.5 * P->dt;
    for (int i = 0; i < 4; ++i) {
        const double vg = dot3(V, g.grad[i]);
        for (int j = 0; j < 4; ++j) {
            const double mij = g.vol / 20.0 * (i == j ? 2.0 : 1.0);
            if (M) M[i * 4 + j] = mij;
            /* mass, minus the volume term int f V . grad psi_i */
            A[i * 4 + j] = mij - tau * vg * g.vol / 4.0;
        }
    }
    for (int a = 0; a < 4; ++a) {
        const double vn = face_flux(V, &g, a);
        if (vn_area) vn_area[a] = vn * g.area[a];
        if (!(vn > 0)) continue;                       /* outflow faces only: the cell's own trace */
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j)
                if (i != a && j != a) A[i * 4 + j] += tau * vn * g.area[a] / 12.0 * (i == j ? 2.0 : 1.0);
    }
    return 0;
}

/* Dense Gaussian elimination with partial pivoting on a 4 x 4 system. */
static int solve4(const double* A0, double* b)
{
    double A[16];
    memcpy(A, A0, sizeof A);
    for (int c = 0; c < 4; ++c) {
        int p = c;
        for (int r = c + 1; r < 4; ++r)
            if (fabs(A[r * 4 + c]) > fabs(A[p * 4 + c])) p = r;
        if (!(fabs(A[p * 4 + c]) > 0)) return -1;
        if (p != c) {
            for (int j = 0; j < 4; ++j) {
                double t = A[c * 4 + j];
                A[c * 4 + j] = A[p * 4 + j];
                A[p * 4 + j] = t;
            }
            double t = b[c];
            b[c] = b[p];
            b[p] = t;
        }
        for (int r = c + 1; r < 4; ++r) {
            const double l = A[r * 4 + c] / A[c * 4 + c];
            for (int j = c; j < 4; ++j) A[r * 4 + j] -= l * A[c * 4 + j];
            b[r] -= l * b[c];
        }
    }
    for (int i = 3; i >= 0; --i) {
        for (int j = i + 1; j < 4; ++j) b[i] -= A[i * 4 + j] * b[j];
        b[i] /= A[i * 4 + i];
    }
    return 0;
}

/* Face a of cell c is a subdomain interface: another subdomain across it, or
 * the periodic boundary of the box. */
static int is_interface(const ko_tetmesh* T, int c, int a)
{
    const long long R = T->nbr[(size_t)c * 4 + a];
    return T->sub[R] != T->sub[c] || T->wrap[(size_t)c * 4 + a];
}

/* Local index in cell R of the vertex with global id gid. */
static int local_vertex(const ko_tetmesh* T, long long R, long long gid)
{
    for (int j = 0; j < 4; ++j)
        if (T->vid[R * 4 + j] == gid) return j;
    return -1;
}

int ko_tet_order(const ko_problem* P, const ko_tetmesh* T, int k, int s, int* order, int* level)
{
    if (!P || !T || !order || k < 0 || k >= ko_num_vel(P)) return -1;
    double V[3];
    ko_velocity(P, k, V);
    const int n = T->ncells;
    int* indeg = (int*)calloc((size_t)n, sizeof(int));
    int* lev = (int*)calloc((size_t)n, sizeof(int));
    if (!indeg || !lev) {
        free(indeg);
        free(lev);
        return -2;
    }
    int total = 0;
    /* edges of the subdomain's graph: R -> L when V enters L across face a */
    for (int c = 0; c < n; ++c) {
        if (T->sub[c] != s) continue;
        ++total;
        tet_geom g;
        cell_geometry(T, c, &g);
        for (int a = 0; a < 4; ++a)
            if (face_flux(V, &g, a) < 0 && !is_interface(T, c, a)) indeg[c]++;
    }
    /* breadth-first: start from the cells with no upwind neighbour inside */
    int head = 0, tail = 0;
    for (int c = 0; c < n; ++c)
        if (T->sub[c] == s && indeg[c] == 0) order[tail++] = c;
    while (head < tail) {
        const int c = order[head++];
        tet_geom g;
        cell_geometry(T, c, &g);
        for (int a = 0; a < 4; ++a) {
            const long long R = T->nbr[(size_t)c * 4 + a];
            if (!(face_flux(V, &g, a) > 0) || is_interface(T, c, a)) continue;   /* outflow to R */
            if (lev[R] < lev[c] + 1) lev[R] = lev[c] + 1;
            if (--indeg[R] == 0) order[tail++] = (int)R;
        }
    }
    if (level)
        for (int i = 0; i < tail; ++i) level[i] = lev[order[i]];
    free(indeg);
    free(lev);
    return tail == total ? tail : -3;      /* -3: the graph has a cycle */
}

/* Per velocity: every cell's A, M and V.N |F| per face (ko_tet_cell_matrix),
 * and for every face the neighbour's local index of each of the cell's
 * vertices (-1 for the vertex opposite the face). */
typedef struct {
    double* A;     /* [cell][16] */
    double* M;     /* [cell][16] */
    double* vna;   /* [cell][4]  */
    int* match;    /* [cell][4 faces][4 vertices] */
} tet_cache;

/* One population over all subdomains: K Jacobi iterations of eq. ibvp. */
static int tet_transport_pop(const ko_problem* P, const ko_tetmesh* T, const tet_cache* C, double* f,
                             const int* orders, const int* ostart, double* defect, int* iters_done)
{
    const int n = T->ncells;
    const size_t nodes = (size_t)n * 4;
    const double tau = 0.5 * P->dt;
    double* prev = (double*)malloc(sizeof(double) * nodes);
    double* cur = (double*)malloc(sizeof(double) * nodes);
    if (!prev || !cur) {
        free(prev);
        free(cur);
        return -11;
    }
    memcpy(prev, f, sizeof(double) * nodes);   /* iterate 0: the data at t^n */
    memcpy(cur, f, sizeof(double) * nodes);
    const int maxit = P->iters > 0 ? P->iters : 100000;
    int it, singular = 0;
    for (it = 1; it <= maxit; ++it) {
#pragma omp parallel for schedule(dynamic, 1)
        for (int s = 0; s < T->nsub; ++s) {
            for (int q = ostart[s]; q < ostart[s + 1]; ++q) {
                const int c = orders[q];
                const double* A = C->A + (size_t)c * 16;
                const double* M = C->M + (size_t)c * 16;
                const double* vna = C->vna + (size_t)c * 4;
                double b[4];
                for (int i = 0; i < 4; ++i) {
                    b[i] = 0.0;
                    for (int j = 0; j < 4; ++j) b[i] += M[i * 4 + j] * f[(size_t)c * 4 + j];
                }
                for (int a = 0; a < 4; ++a) {
                    if (!(vna[a] < 0)) continue;                    /* inflow faces */
                    const long long R = T->nbr[(size_t)c * 4 + a];
                    const double* src = is_interface(T, c, a) ? prev : cur;  /* eq. ibvp3 */
                    double fr[4] = {0, 0, 0, 0};
                    for (int j = 0; j < 4; ++j)
                        if (j != a) fr[j] = src[(size_t)R * 4 + C->match[((size_t)c * 4 + a) * 4 + j]];
                    for (int i = 0; i < 4; ++i) {
                        if (i == a) continue;
                        for (int j = 0; j < 4; ++j)
                            if (j != a) b[i] += tau * (-vna[a]) / 12.0 * (i == j ? 2.0 : 1.0) * fr[j];
                    }
                }
                if (solve4(A, b)) {
                    singular = 1;
                    continue;
                }
                for (int i = 0; i < 4; ++i) cur[(size_t)c * 4 + i] = b[i];
            }
        }
        if (singular) break;
        if (P->iters == 0) {
            double dmax = 0.0, fmax = 0.0;
            for (size_t i = 0; i < nodes; ++i) {
                const double e = fabs(cur[i] - prev[i]);
                if (e > dmax) dmax = e;
                if (fabs(cur[i]) > fmax) fmax = fabs(cur[i]);
            }
            if (dmax <= 1e-15 * (fmax > 0 ? fmax : 1.0)) break;
        }
        if (it < maxit) memcpy(prev, cur, sizeof(double) * nodes);
    }
    if (singular) {
        free(prev);
        free(cur);
        return -12;
    }
    if (it > maxit) it = maxit;
    if (iters_done) *iters_done = it;
    if (defect) {
        /* dt |V.N| int_F (f_R^{K-1} - f_R^{K}) over the inflow faces on a
         * subdomain boundary; int_F of a P1 trace = |F|/3 (sum of its three
         * vertex values) */
        double acc = 0.0;
        for (int c = 0; c < n; ++c) {
            const double* vna = C->vna + (size_t)c * 4;
            for (int a = 0; a < 4; ++a) {
                const long long R = T->nbr[(size_t)c * 4 + a];
                if (!(vna[a] < 0) || !is_interface(T, c, a)) continue;
                double sum = 0.0;
                for (int j = 0; j < 4; ++j) {
                    if (j == a) continue;
                    const size_t r = (size_t)R * 4 + C->match[((size_t)c * 4 + a) * 4 + j];
                    sum += prev[r] - cur[r];
                }
                acc += P->dt * (-vna[a]) / 3.0 * sum;
            }
        }
        *defect = acc;
    }
    /* Crank-Nicolson: f^{n+1} = 2 f* - f^n */
    for (size_t i = 0; i < nodes; ++i) f[i] = 2.0 * cur[i] - f[i];
    free(prev);
    free(cur);
    return 0;
}

int ko_tet_transport(const ko_problem* P, const ko_tetmesh* T, double* f, double* defect, int* iters_done)
{
    if (!P || !T || !f || P->dim != 3 || T->nsub < 1) return -1;
    const int m = ko_num_vars(P), nv = ko_num_vel(P);
    const int n = T->ncells;
    const size_t nodes = (size_t)n * 4;
    int* orders = (int*)malloc(sizeof(int) * (size_t)n);
    int* ostart = (int*)malloc(sizeof(int) * (size_t)(T->nsub + 1));
    tet_cache C;
    C.A = (double*)malloc(sizeof(double) * 16 * (size_t)n);
    C.M = (double*)malloc(sizeof(double) * 16 * (size_t)n);
    C.vna = (double*)malloc(sizeof(double) * 4 * (size_t)n);
    C.match = (int*)malloc(sizeof(int) * 16 * (size_t)n);
    if (!orders || !ostart || !C.A || !C.M || !C.vna || !C.match) {
        free(orders);
        free(ostart);
        free(C.A);
        free(C.M);
        free(C.vna);
        free(C.match);
        return -11;
    }
    for (int c = 0; c < n; ++c)
        for (int a = 0; a < 4; ++a)
            for (int j = 0; j < 4; ++j)
                C.match[((size_t)c * 4 + a) * 4 + j] =
                    j == a ? -1 : local_vertex(T, T->nbr[(size_t)c * 4 + a], T->vid[(size_t)c * 4 + j]);
    if (defect)
        for (int v = 0; v < m; ++v) defect[v] = 0.0;
    int maxdone = 0, rc = 0;
    for (int k = 0; k < nv && !rc; ++k) {
        for (int c = 0; c < n && !rc; ++c)
            rc = ko_tet_cell_matrix(P, T, c, k, C.A + (size_t)c * 16, C.M + (size_t)c * 16, C.vna + (size_t)c * 4);
        /* the topological order of every subdomain for this velocity */
        ostart[0] = 0;
        for (int s = 0; s < T->nsub && !rc; ++s) {
            const int cnt = ko_tet_order(P, T, k, s, orders + ostart[s], NULL);
            if (cnt < 0) rc = cnt;
            ostart[s + 1] = ostart[s] + (cnt < 0 ? 0 : cnt);
        }
        for (int v = 0; v < m && !rc; ++v) {
            double dfc = 0.0;
            int done = 0;
            rc = tet_transport_pop(P, T, &C, f + (size_t)(k * m + v) * nodes, orders, ostart,
                                   defect ? &dfc : NULL, &done);
            if (defect) defect[v] += dfc;
            if (done > maxdone) maxdone = done;
        }
    }
    if (iters_done) *iters_done = maxdone;
    free(orders);
    free(ostart);
    free(C.A);
    free(C.M);
    free(C.vna);
    free(C.match);
    return rc;
}

int ko_tet_step(const ko_problem* P, const ko_tetmesh* T, double* f, int nsteps)
{
    if (!P || !T || !f || nsteps < 0) return -1;
    for (int s = 0; s < nsteps; ++s) {
        int rc = ko_tet_transport(P, T, f, NULL, NULL);
        if (rc) return rc;
        rc = ko_relax_n(P, f, (size_t)T->ncells * 4);
        if (rc) return rc;
    }
    return 0;
}

int ko_tet_mass(const ko_problem* P, const ko_tetmesh* T, const double* W, double* mass)
{
    if (!P || !T || !W || !mass) return -1;
    const int m = ko_num_vars(P);
    const size_t nodes = (size_t)T->ncells * 4;
    for (int v = 0; v < m; ++v) {
        double s = 0.0;
        for (int c = 0; c < T->ncells; ++c) {
            tet_geom g;
            if (cell_geometry(T, c, &g)) return -2;
            double sum = 0.0;
            for (int a = 0; a < 4; ++a) sum += W[(size_t)v * nodes + (size_t)c * 4 + a];
            s += g.vol / 4.0 * sum;
        }
        mass[v] = s;
    }
    return 0;
}
