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

#ifdef __cplusplus
}
#endif
#endif
