/*
 * kin_oracle.h -- plain FP64 CPU oracle for the CFL-less kinetic DG step
 * (Gerhard, Helluy, Michel-Dansac, Weber, "Parallel kinetic schemes for
 * conservation laws, with large time steps", arXiv:2212.11010).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the independent reference that
 * the CUDA path is checked against.  Only the test-suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it.  It shares no code,
 * header, table or helper with the GPU library.
 *
 * Conventions (identical on both sides, but written separately):
 *   d        space dimension (1..3), m conserved variables.  Systems:
 *            scalar advection (m = 1), Euler (m = d + 2) and, in 3D,
 *            Maxwell's equations (Sec. 6.1.1; m = 6, W = (E, H)).
 *   k        kinetic velocity index.  Axis sets (velset KO_AXIS; D1Q2, D2Q4,
 *            D3Q6): k = 2*a + s, V_k = +lambda e_a (s = 0) or -lambda e_a
 *            (s = 1).  Simplex sets (velset KO_SIMPLEX; d + 1 velocities,
 *            Sec. 2.1): D1Q2 as above, D2Q3 V_k = lambda (cos 2k pi/3,
 *            sin 2k pi/3) (Sec. 2.4), D3Q4 the cube diagonals with components
 *            +-lambda (Sec. 6.1.3).
 *   pop      population index pop = k*m + v  (velocity-major).
 *   Storage  W[v][cz][cy][cx][nz][ny][nx] and f[pop][cz][cy][cx][nz][ny][nx]:
 *            cells row-major with x fastest, then the (p+1)^d tensor GLL
 *            nodes of the cell with the x node index fastest.
 *
 * All functions return 0 on success and a negative value on bad arguments.
 */
#ifndef KIN_ORACLE_H
#define KIN_ORACLE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { KO_ADVECTION = 0, KO_EULER = 1, KO_MAXWELL = 2 };
#define KO_MAXM 6       /* most conserved variables of a system (Maxwell)       */
enum { KO_AXIS = 0, KO_SIMPLEX = 1 };

typedef struct {
    int dim;            /* d, 1..3                                            */
    int n[3];           /* cells per axis (axes >= d must be 1)               */
    double lo[3];       /* domain lower corner                                */
    double hi[3];       /* domain upper corner (periodic in every axis)       */
    int degree;         /* DG degree p (p+1 GLL nodes per axis), 1..4         */
    int system;         /* KO_ADVECTION (m = 1) or KO_EULER (m = d + 2)       */
    double lambda;      /* kinetic speed |V_k|                                */
    double gamma;       /* ratio of specific heats (Euler)                    */
    double adv[3];      /* advection velocity a (scalar advection)            */
    double omega;       /* over-relaxation parameter, in [1, 2]               */
    double dt;          /* time step                                          */
    int tiles[3];       /* subdomains per axis; must divide n[a]              */
    int iters;          /* subdomain iterations K (>= 1); 0 = to fixed point  */
    int velset;         /* KO_AXIS (2d velocities) or KO_SIMPLEX (d + 1)      */
    double sigma;       /* conductivity (Maxwell only; uniform), >= 0         */
    int inflow[3];      /* 0: axis a periodic; 1: both faces of axis a are
                           domain boundaries where the incoming populations
                           take the Maxwellian of the face state Wb (axis
                           velocity sets only)                                */
    double Wb[3][2][KO_MAXM];  /* boundary state of face (axis, 0 = lower,
                                  1 = upper), constant in time              */
} ko_problem;

int    ko_num_vars(const ko_problem* P);          /* m                      */
int    ko_num_vel(const ko_problem* P);           /* 2d or d + 1            */
/* V_k (3 components, unused ones 0). */
int    ko_velocity(const ko_problem* P, int k, double* V);
size_t ko_num_nodes(const ko_problem* P);         /* cells * (p+1)^d        */

/* GLL nodes on [0,1] and weights summing to 1 (Sec. 3.1 basis; Gauss-Lobatto
 * collocation is the reading for Cartesian cells). */
int ko_gll(int p, double* xi, double* w);
/* D[i*(p+1)+j] = l_j'(xi_i) for the Lagrange basis on the GLL nodes. */
int ko_diff_matrix(int p, double* D);
/* Node coordinates xyz[3*node] in storage order. */
int ko_node_coords(const ko_problem* P, double* xyz);

/* Physical flux Q^a(W) (eq. conslaw) and the Maxwellians M_k(W) of all
 * velocities at one point: eq. maxwell_def solved as a linear system for the
 * d + 1 simplex velocities, and the 2d-velocity reading for axis sets. */
int ko_flux(const ko_problem* P, const double* W, int axis, double* Q);
int ko_maxwellian(const ko_problem* P, const double* W, double* M);

/* The local implicit cell matrix of velocity k (weak form eq. dg_imp with the
 * Crank-Nicolson half step tau = dt/2); A is (p+1)^d x (p+1)^d row-major. */
int ko_cell_matrix(const ko_problem* P, int k, double* A);

/* f = M(W0) at every node (Sec. 2.2, initialisation). */
int ko_init(const ko_problem* P, const double* W0, double* f);
/* W = sum_k f_k (Sec. 2.2, step 3). */
int ko_moments(const ko_problem* P, const double* f, double* W);
/* The same three pointwise steps on 'nodes' nodes of any mesh (the
 * tetrahedral meshes below): storage W[v][node], f[pop][node]. */
int ko_init_n(const ko_problem* P, const double* W0, double* f, size_t nodes);
int ko_moments_n(const ko_problem* P, const double* f, double* W, size_t nodes);
int ko_relax_n(const ko_problem* P, double* f, size_t nodes);
/* Crank-Nicolson DG transport of every population over dt, solved by the
 * downwind sweep inside each subdomain with the lagged subdomain coupling of
 * eq. ibvp.  If defect != NULL it receives, per variable, the mass change
 * that the finite iteration count leaves at subdomain interfaces.
 * If iters_done != NULL it receives the number of iterations used. */
int ko_transport(const ko_problem* P, double* f, double* defect, int* iters_done);
/* Over-relaxation f <- omega M(W) + (1 - omega) f (eq. over_relaxation).
 * Maxwell with conductivity sigma: first the Crank-Nicolson source step of
 * Sec. 2.3 on W = sum f (E <- mu E, H unchanged, mu = (1 - sigma dt/2) /
 * (1 + sigma dt/2), Sec. 6.4), then the non-equilibrium part relaxed about
 * the new equilibrium: f <- M(W+) + (1 - omega)(f - M(W-)). */
int ko_relax(const ko_problem* P, double* f);
/* nsteps applications of S(dt) = relaxation o transport. */
int ko_step(const ko_problem* P, double* f, int nsteps);
/* Quadrature mass per variable: sum over nodes of cell volume x weights x W. */
int ko_mass(const ko_problem* P, const double* W, double* mass);
/* Threads of the parallel loops (subdomains of one iteration, nodes of the
 * pointwise steps) when built with OpenMP; nthreads <= 0 leaves the count
 * unchanged.  Returns the count now in use (1 without OpenMP).  Results do
 * not depend on it. */
int ko_set_threads(int nthreads);

/* ---- tetrahedral meshes (Sec. 3.1: tetrahedral cells, n_f = 4 faces) ----
 * P1 nodal basis: the four vertices of each cell (Lagrange functions,
 * exact integration of the mass, stiffness and face matrices).  Storage:
 * f[pop][cell][a] with a the cell's local vertex.  Face a of a cell is the
 * face opposite its vertex a.  Only the kinetic model (system, velset,
 * lambda, gamma, adv, sigma, omega), dt and iters of the ko_problem are
 * used, with dim = 3; the mesh and its subdomains come from ko_tetmesh.
 * Periodic meshes only (every face has a neighbour).  A face is a subdomain
 * interface (eq. ibvp: inflow from the previous iterate) when the cell across
 * it lies in another subdomain or when it crosses the periodic boundary (a
 * subdomain that wraps around the box couples to itself there, as on the
 * Cartesian meshes; the oriented graph inside a subdomain is then acyclic). */
typedef struct {
    int ncells;
    const double* xyz;  /* [cell][4][3] vertex coordinates (one geometric tetrahedron per cell) */
    const long long* vid;  /* [cell][4] global vertex ids (matching nodes across faces)   */
    const long long* nbr;  /* [cell][4] the cell across face a                            */
    const int* sub;     /* [cell] subdomain id, 0..nsub-1 (Sec. 5.1)                       */
    int nsub;
    const int* wrap;    /* [cell][4] 1: face a crosses the periodic boundary of the box    */
} ko_tetmesh;

/* Local matrices of cell c and velocity k for the implicit half step
 * tau = dt/2 of eq. dg_imp: A = M + tau (-K + sum_{outflow faces}
 * (V.N) F_face) (4 x 4, row-major), the mass matrix M (4 x 4), and per face
 * a the flux V.N_a |F_a| (so the caller sees the orientation). */
int ko_tet_cell_matrix(const ko_problem* P, const ko_tetmesh* T, int c, int k, double* A, double* M,
                       double* vn_area);
/* Crank-Nicolson transport of every population, cells visited in the
 * topological order of the oriented cell graph of each subdomain (Sec. 3.2,
 * breadth-first), subdomains coupled by eq. ibvp with P->iters iterations
 * (0: to the fixed point).  defect (m doubles or NULL): the interface mass
 * defect of the finite iteration. */
int ko_tet_transport(const ko_problem* P, const ko_tetmesh* T, double* f, double* defect, int* iters_done);
/* nsteps applications of relaxation o transport. */
int ko_tet_step(const ko_problem* P, const ko_tetmesh* T, double* f, int nsteps);
/* Mass per variable: sum over cells of |L|/4 times the sum of W over the
 * cell's nodes (the exact integral of the P1 function). */
int ko_tet_mass(const ko_problem* P, const ko_tetmesh* T, const double* W, double* mass);
/* Breadth-first topological order of the cells of subdomain s for velocity
 * k (Sec. 3.2): order receives the cell ids, level their BFS level (the
 * wavefront: cells of one level are independent).  Returns the count. */
int ko_tet_order(const ko_problem* P, const ko_tetmesh* T, int k, int s, int* order, int* level);

#ifdef __cplusplus
}
#endif
#endif
