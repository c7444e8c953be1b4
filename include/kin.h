/*
 * kin.h -- C ABI of the GB300 (sm_103a) kinetic DG library.
 *
 * The library advances the kinetic representation of a hyperbolic system of
 * conservation laws (Gerhard, Helluy, Michel-Dansac, Weber, "Parallel kinetic
 * schemes for conservation laws, with large time steps", arXiv:2212.11010):
 *
 *   one step S(dt) = R_omega o T_CN(dt)
 *     T_CN  Crank-Nicolson implicit upwind DG transport of every population
 *           f_k at its constant velocity V_k (Sec. 3.1, eq. dg_imp; "which we
 *           use in practice", Sec. 3.1), solved cell by cell in downwind order
 *           (Sec. 3.2) inside each subdomain, the subdomains coupled by the
 *           lagged iteration of Sec. 5.1 (eq. ibvp) with K iterations;
 *     R     W = sum_k f_k, f_k <- omega M_k(W) + (1 - omega) f_k
 *           (Sec. 2.2, eq. over_relaxation).
 *
 * Meshes are periodic Cartesian boxes with tensor Gauss-Lobatto nodes
 * (degree p, (p+1)^d nodes per cell).  Velocity sets: 2d velocities
 * +-lambda e_a (D1Q2, D2Q4, D3Q6) with M_{a,+-} = W/(2d) +- Q^a(W)/(2 lambda),
 * which satisfies the moment conditions of eq. maxwell_def.
 *
 * Storage order (host and device, every call):
 *   W  (macroscopic)  double  [v][cz][cy][cx][nz][ny][nx]
 *   f  (kinetic)      ctx precision (float or double)
 *                     [pop][cz][cy][cx][nz][ny][nx],  pop = k*m + v,
 *                     k = 2a + s: V_k = +lambda e_a (s = 0) or -lambda e_a (s = 1)
 *   Cells are row-major with x fastest; inside a cell the x node is fastest.
 *   m = 1 (scalar advection) or d + 2 (Euler: rho, rho u_1..rho u_d, E).
 *
 * Errors: every call returns a kin_status.  No exception crosses the ABI.
 * After the first failure of a call that touched the device the context is
 * poisoned: later calls return KIN_ESTATE until kin_destroy.  A message for
 * the last error is available from kin_last_error().
 *
 * Threads: a context may be used by one host thread at a time.  Work is
 * stream-ordered on the context's stream (kin_opts.stream).
 */
#ifndef KIN_H
#define KIN_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct kin_ctx kin_ctx;               /* opaque, owned by the library */

typedef enum {
    KIN_OK = 0,
    KIN_EINVAL = 1,     /* bad argument: nothing was done                     */
    KIN_ENOMEM = 2,     /* device allocation failed                           */
    KIN_EBUDGET = 3,    /* request exceeds kin_opts.mem_budget                */
    KIN_ECUDA = 4,      /* a CUDA call failed (context is poisoned)           */
    KIN_ETIMEOUT = 5,   /* a bounded device wait gave up (context poisoned)   */
    KIN_ESTATE = 6      /* context poisoned by an earlier error, or no state  */
} kin_status;

/* kin_model.system: scalar advection (m = 1), Euler (m = d + 2), or
 * Maxwell's equations in 3D (Sec. 6.1.1; m = 6, W = (E, H), axis velocity
 * set D3Q6 only) with a uniform conductivity kin_model.sigma. */
enum { KIN_ADVECTION = 0, KIN_EULER = 1, KIN_MAXWELL = 2 };
/* kin_model.velset: 2d axis velocities +-lambda e_a (D1Q2, D2Q4, D3Q6; the
 * value is the dimension), or the paper's d + 1 sets: D2Q3 with
 * V_k = lambda (cos 2k pi/3, sin 2k pi/3) (Sec. 2.4) and D3Q4 with the cube
 * diagonals (+-lambda, +-lambda, +-lambda) (Sec. 6.1.3), whose Maxwellians
 * solve eq. maxwell_def exactly.  The d + 1 sets are transported by K
 * literal subdomain iterations with wavefront sweeps whose lanes are the
 * subdomain's columns along its sweep axis: a subdomain may have at most 1024
 * columns (2D: max(L0, L1); 3D: L0 L1), else kin_create returns KIN_EINVAL;
 * degree <= 3 in 2D, <= 2 in 3D; periodic axes only.  kin_diag's
 * next_defect is not available for them. */
enum { KIN_D1Q2 = 1, KIN_D2Q4 = 2, KIN_D3Q6 = 3, KIN_D2Q3 = 4, KIN_D3Q4 = 5 };
enum { KIN_FP64 = 0, KIN_FP32 = 1 };                /* kin_opts.precision */

/* Cartesian box [lo, hi] with n[a] cells along axis a (axes >= dim must have
 * n = 1).  inflow[a] = 0: axis a is periodic; inflow[a] = 1: both faces of
 * axis a are domain boundaries where the populations entering the box take
 * the Maxwellian of the face's boundary state (kin_set_boundary); axis
 * velocity sets only.  The paper prescribes the solution on the boundary
 * (Sec. 6.2) and upwinds with the value across every face (eq. dg_imp). */
typedef struct {
    int dim;
    int n[3];
    double lo[3];
    double hi[3];
    int inflow[3];
} kin_mesh;

/* Kinetic model.  lambda: kinetic speed |V_k| (must satisfy the
 * sub-characteristic condition of Sec. 2.1 for the data; the library does not
 * check it).  omega in [1, 2] (eq. over_relaxation).  gamma: Euler gas
 * constant.  adv: advection velocity of the scalar law.  sigma: Maxwell
 * conductivity (>= 0, uniform; ignored by the other systems): each step
 * applies the Crank-Nicolson source step of Sec. 2.3 to W = sum f,
 * E <- mu E with mu = (1 - sigma dt/2) / (1 + sigma dt/2) (Sec. 6.4), and
 * relaxes the non-equilibrium part about the new equilibrium,
 * f <- M(W+) + (1 - omega)(f - M(W-)) (for sigma = 0 this is
 * eq. over_relaxation). */
typedef struct {
    int system;
    int velset;
    double lambda;
    double gamma;
    double adv[3];
    double omega;
    double sigma;
} kin_model;

/* Device allocator hook: called with the context's stream.  Both NULL means
 * cudaMalloc / cudaFree. */
typedef void* (*kin_alloc_fn)(size_t bytes, void* stream, void* user);
typedef void (*kin_free_fn)(void* ptr, size_t bytes, void* stream, void* user);

/* Options.  tiles[a]: number of subdomains along axis a (must divide n[a];
 * Sec. 5.1).  iters: subdomain iterations K per step (>= 1; the paper uses 3,
 * Sec. 5.2).  block[a]: cells per thread block along a (must divide the
 * subdomain extent n[a]/tiles[a]; 0 = chosen by the library).  The block
 * size changes only the schedule, never the result beyond round-off.
 * mem_budget: upper bound in bytes on device memory the context may hold
 * (0 = unbounded).  stream: cudaStream_t (NULL = the legacy default stream). */
typedef struct {
    int tiles[3];
    int iters;
    int precision;
    int block[3];
    size_t mem_budget;
    void* stream;
    kin_alloc_fn alloc;
    kin_free_fn free;
    void* alloc_user;
    double wait_timeout_s;  /* bound on every device-side wait (0 = 1 s)        */
    int debug_flags;        /* KIN_DEBUG_* test hooks; 0 in production          */
    int threads;            /* threads per thread block, 32..256 (0 = auto)     */
    int stages;             /* shared-memory tile buffers, 1 or 2 (0 = auto)    */
} kin_opts;

/* Test hook: the bulk-load barrier of every thread block expects 16 bytes
 * that never arrive, so its bounded wait runs out; the step reports
 * KIN_ETIMEOUT at the next synchronising call and the CUDA context stays
 * usable. */
enum { KIN_DEBUG_STALL_LOAD = 1 };

/* Sizes of a context. */
typedef struct {
    int dim, degree, m, nvel, npop, nodes_per_cell;
    size_t cells, nodes;            /* nodes = cells * nodes_per_cell          */
    size_t kinetic_values;          /* npop * nodes (elements of f)            */
    size_t state_values;            /* m * nodes (elements of W)               */
    size_t device_bytes;            /* device memory held by the context       */
    int precision;
    int block[3];                   /* thread-block cell extents in use        */
    int smem_bytes;                 /* dynamic shared memory per thread block  */
    int grid;                       /* thread blocks per step launch           */
    int threads;                    /* threads per thread block                */
    int stages;                     /* shared-memory tile buffers              */
    long long steps_done;
    int specialised;                /* 1: compile-time block-shape kernel      */
} kin_info;

/* Create a context: validates arguments, computes on the GPU in FP64 the
 * Gauss-Lobatto rule and, per velocity, the inverse of the local implicit
 * block of eq. dg_imp (Crank-Nicolson half step tau = dt/2; Sec. 3.2 notes
 * this preprocessing happens once), and allocates f, the interface-trace
 * buffers of eq. ibvp and the FP64 staging buffers.  Returns KIN_EINVAL
 * (bad mesh/model/opts, tiles not dividing n, degree outside 1..3),
 * KIN_EBUDGET, KIN_ENOMEM or KIN_ECUDA; *out is NULL on failure. */
kin_status kin_create(const kin_mesh* mesh, const kin_model* model, int degree, double dt,
                      const kin_opts* opts, kin_ctx** out);

/* Tetrahedral meshes -- the paper's own setting (Sec. 3.1: unstructured
 * tetrahedral cells with n_f = 4 faces; Sec. 3.2: the cell graph oriented by
 * V, a DAG swept in breadth-first topological order; Sec. 5.1: subdomains
 * coupled by eq. ibvp).  Basis: P1 nodal, the four vertices of each cell,
 * with exact integrals.  Face a of a cell is the face opposite its local
 * vertex a; a face with |V.N| <= 1e-12 |V| is parallel to V (no flux).
 * Meshes are periodic: every face has a neighbour.  A face is a subdomain
 * interface -- its inflow comes from the previous iterate -- when the cell
 * across it lies in another subdomain or when wrap marks it (a face across
 * the periodic boundary, so that a subdomain wrapping around the box is
 * acyclic).  All arrays are host memory, read during kin_create_tet only. */
typedef struct {
    int ncells;
    const double* xyz;       /* [cell][4][3] vertex coordinates (one geometric tetrahedron per cell) */
    const long long* vid;    /* [cell][4] global vertex ids: nodes that meet across a face share an id */
    const long long* nbr;    /* [cell][4] the cell across face a                                      */
    const int* sub;          /* [cell] subdomain id, 0..nsub-1                                        */
    const int* wrap;         /* [cell][4] 1: face a crosses the periodic boundary (may be NULL: none) */
} kin_tetmesh;

/* Create a context on a tetrahedral mesh.  model: system (advection, Euler
 * with m = 5, Maxwell with m = 6), velset KIN_D3Q6 or KIN_D3Q4 (the cube
 * diagonals of Sec. 6.1.3), lambda, gamma, adv, omega, sigma as for
 * kin_create.  opts: iters, precision, stream, the allocator hooks and
 * mem_budget are used; tiles, block, threads and stages are not (the
 * subdomains come from mesh->sub).  The FP64 set-up inverts the local
 * implicit block of every (cell, velocity) on the GPU; the host orients the
 * faces and sorts every subdomain breadth-first into levels.  Storage of W
 * and f: [v][cell][a] and [pop][cell][a] (a the local vertex, pop = k m + v;
 * D3Q6 k = 2 axis + sign, D3Q4 k in the order (+,+,+), (+,-,-), (-,+,-),
 * (-,-,+)).  The context then takes kin_set_state, kin_set_kinetic,
 * kin_step, kin_get_state, kin_get_kinetic, kin_diag (mass only),
 * kin_query, kin_sync and kin_destroy; kin_set_boundary and batches return
 * KIN_EINVAL.  Each step is K sweep launches (one thread block per
 * (subdomain, velocity) walking the levels) and one launch for the
 * Crank-Nicolson extrapolation and the relaxation.  Errors: KIN_EINVAL (bad
 * arguments or topology: a neighbour out of range, a face whose vertices are
 * not in the neighbour, a degenerate cell, a cycle in a subdomain's oriented
 * graph), KIN_EBUDGET, KIN_ENOMEM, KIN_ECUDA. */
kin_status kin_create_tet(const kin_tetmesh* mesh, const kin_model* model, double dt, const kin_opts* opts,
                          kin_ctx** out);

/* Set f = M(W) at every node (Sec. 2.2: the natural initial choice
 * F_k = M_k(W(., 0))).  W: m * nodes doubles in the storage order above, on
 * the host (on_device = 0, pageable or pinned; copied before return) or on
 * the device (on_device = 1, read in stream order).  n_values must equal
 * m * nodes (else KIN_EINVAL).  Resets the step counter. */
kin_status kin_set_state(kin_ctx* ctx, const double* W, size_t n_values, int on_device);

/* Boundary state of face (axis, side) of an inflow axis (side 0: x_a = lo,
 * side 1: x_a = hi): W holds m doubles (host memory, read before return).
 * The populations entering the box through that face take M_k(W) there in
 * every step and every subdomain iteration (the value is data) until the
 * next call.  Time-dependent boundary data: set the state at the step's
 * midpoint t^n + dt/2 before each kin_step(ctx, 1) (the implicit half step of
 * Crank-Nicolson sits there; data at t^n or t^{n+1} lose an order).  Every
 * face of an inflow axis needs a state before the first step (else kin_step
 * returns KIN_ESTATE).  KIN_EINVAL: axis not an inflow axis,
 * side not 0 or 1, m wrong, or an Euler state with rho <= 0. */
kin_status kin_set_boundary(kin_ctx* ctx, int axis, int side, const double* W, size_t m);

/* Set the kinetic state f directly (checkpoint resume: after the first step
 * f != M(W), Sec. 2.2 remark, so W alone cannot restart a run).  f holds
 * npop * nodes values of the context precision. */
kin_status kin_set_kinetic(kin_ctx* ctx, const void* f, size_t n_values, int on_device);

/* Enqueue nsteps applications of S(dt) on the context stream and return
 * (asynchronous).  nsteps < 0: KIN_EINVAL; no state set, or an inflow face
 * without a boundary state: KIN_ESTATE. */
kin_status kin_step(kin_ctx* ctx, int nsteps);

/* W = sum_k f_k (Sec. 2.2, step 3) into W (m * nodes doubles).  Host
 * destination: synchronises the stream before return.  Device destination:
 * stream-ordered. */
kin_status kin_get_state(kin_ctx* ctx, double* W, size_t n_values, int on_device);

/* Copy out the kinetic state f (npop * nodes values of the context precision). */
kin_status kin_get_kinetic(kin_ctx* ctx, void* f, size_t n_values, int on_device);

/* Host copies for pipelines.  As kin_set_kinetic and kin_get_kinetic with a
 * host buffer, but enqueued on `stream` (a cudaStream_t; NULL = the context's
 * stream) and not waited for.  After kin_set_kinetic_async the interface
 * summaries of the new f (axis velocity sets) are computed by the next
 * kin_step, kin_batch_step or defect diagnostic: a batch does it for all its
 * members in one pass per kernel type.
 * Ownership: f stays the caller's.  It must be page-locked host memory and
 * must not be modified (set) or read (get) until the copy has completed; the
 * caller orders that with an event or a stream synchronisation.
 * Ordering: the caller orders these copies against kin_step or
 * kin_batch_step on other streams with events (cudaStreamWaitEvent).  A copy
 * and a step of the same context must not overlap in time.
 * Errors: KIN_EINVAL (NULL f, wrong n_values) and KIN_ESTATE (get before any
 * state) at the call.  A failure of the enqueued work shows at the next
 * synchronising call (kin_sync, kin_get_state, kin_diag). */
kin_status kin_set_kinetic_async(kin_ctx* ctx, const void* f, size_t n_values, void* stream);
kin_status kin_get_kinetic_async(kin_ctx* ctx, void* f, size_t n_values, void* stream);

/* FP64 diagnostics, synchronous.  mass_per_var (m doubles, may be NULL): the
 * quadrature integral of every conserved variable over the box.
 * next_defect (m doubles, may be NULL): the mass change that the next step's
 * finite subdomain iteration will leave at subdomain interfaces, dt |V.N|
 * times the face integral of (trace^{K-1} - trace^{K}) summed over every
 * upwind subdomain boundary (zero up to round-off when the iteration has
 * converged).  iter_residual (may be NULL): max over those faces of
 * |trace^{K} - trace^{K-1}|.  With inflow axes only mass_per_var is
 * available (next_defect or iter_residual: KIN_EINVAL). */
kin_status kin_diag(kin_ctx* ctx, double* mass_per_var, double* next_defect, double* iter_residual);

/* kin_step_noalloc -- nsteps steps of S(dt) without any device allocation.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot let a library allocate device memory -- host applications whose own
 * memory pool reserves the device memory up front, and code that runs on a
 * fixed memory plan where an allocation failure at run time is not
 * acceptable.
 *
 * mesh, model, degree, dt: as kin_create (periodic axes only: a mesh with an
 * inflow axis is KIN_EINVAL).  opts: tiles, iters, precision, block,
 * threads, stages, wait_timeout_s and stream are used as in kin_create;
 * mem_budget, debug_flags and the allocator hooks are ignored.
 * f: device pointer to the caller's kinetic state, npop * nodes values of
 * opts->precision in the storage order above; read as f^n and overwritten
 * in place with f^{n + nsteps} (the caller owns it).  errbuf/errlen: optional
 * buffer that receives a message on failure.
 *
 * Everything else the step needs (block-inverse coefficients, the
 * Gauss-Lobatto rule, the block summaries) lives in one static device array
 * of 16 MiB that every GPU loading this library holds until process exit.
 * Problems whose scratch would exceed it are rejected with KIN_EINVAL and a
 * message naming the limit; nothing is launched then.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture.
 * Every call re-initialises the parts of the array it reads, so the previous
 * call's leftovers never matter -- but all calls on a device share the one
 * array, so calls whose work overlaps on the GPU (different streams, or
 * different host threads) race and corrupt each other: serialise them.
 * Work runs on opts->stream; the call returns once that stream has drained
 * (KIN_ECUDA on a CUDA error, KIN_ETIMEOUT if a bounded device wait ran out). */
kin_status kin_step_noalloc(const kin_mesh* mesh, const kin_model* model, int degree, double dt,
                            const kin_opts* opts, void* f, int nsteps, char* errbuf, size_t errlen);

/* Batched stepping of several independent problems (the paper's method
 * applied to each; Sec. 2.2, 3, 5.1).  A batch groups existing contexts with
 * a state; kin_batch_step advances every member by nsteps steps, replayed
 * from a captured CUDA graph.  Per step, the members run in one persistent
 * launch per kernel type covering the tiles of all members of that type
 * (problems of different mesh size share a launch; a member without a
 * fixed-shape kernel gets its own launch).  With KIN_BATCH_MIXED the 2D
 * Euler FP32 members of degrees 1..3 whose cell blocks match one of the
 * library's compiled mixed-degree kernels (the default cell blocks of
 * kin_create, 0 in kin_opts.block, match the first) share ONE persistent
 * launch over a work list of all their tiles, the most expensive first.
 * Results equal stepping each member alone (bitwise: the same kernel
 * arithmetic per tile).  kin_set_state and kin_set_kinetic on a member keep
 * the batch valid (they rebuild the member's summaries in place).
 *
 * members: count distinct contexts of one device, each with a state; they
 * stay owned by the caller and must outlive the batch.  stream: cudaStream_t
 * of the batch (NULL = a stream the batch creates and owns; the legacy
 * default stream cannot hold the captured graphs); work already queued on a
 * member's stream runs before the batch step, and later work on it after.
 * That second order is lazy: a batch step records an event per member, and
 * the member's next call of this library (on its own stream, or on the
 * stream an asynchronous copy names) waits for that event, so a stream that
 * several contexts share is held up only by their own steps.  A new batch of
 * members still in flight in another batch waits for them the same way; a
 * member's own stream, used directly (not through this library), is not
 * ordered after the step until kin_sync or another call on the member.
 * Stepping a member alone while it is in a batch invalidates the batch
 * (KIN_ESTATE on the next kin_batch_step).  A member's kin_set_boundary
 * applies from the next batch step on.  Errors: KIN_EINVAL (bad
 * arguments), KIN_ESTATE (member without state or without a boundary state
 * on an inflow face / poisoned / stepped alone),
 * KIN_ECUDA, KIN_ENOMEM; messages from kin_batch_last_error. */
typedef struct kin_batch kin_batch;
kin_status kin_batch_create(kin_ctx* const* members, int count, void* stream, kin_batch** out);
/* As kin_batch_create, with flags: KIN_BATCH_DIRECT enqueues each step's
 * launches directly instead of capturing and replaying CUDA graphs (cheaper
 * to create: for batches whose membership changes often, as in a serving
 * loop); KIN_BATCH_MIXED puts the eligible 2D members into one mixed-degree
 * launch (see above).  Results are the same.  Unknown flags: KIN_EINVAL. */
enum { KIN_BATCH_DIRECT = 1, KIN_BATCH_MIXED = 2 };
kin_status kin_batch_create_ex(kin_ctx* const* members, int count, void* stream, int flags, kin_batch** out);
/* Launches of this library per batch step, and how many members share the
 * mixed-degree launch (either pointer may be NULL). */
kin_status kin_batch_info(const kin_batch* batch, int* launches_per_step, int* mixed_members);
/* Enqueue nsteps steps of every member on the batch's stream (asynchronous).
 * KIN_ESTATE if a member is poisoned, was stepped outside the batch or lacks
 * a boundary state on an inflow face; KIN_ECUDA on a launch error. */
kin_status kin_batch_step(kin_batch* batch, int nsteps);
/* Wait for the batch's stream, then read every member's device error word
 * (on the batch's stream): KIN_ETIMEOUT names the first member whose bounded
 * device wait ran out. */
kin_status kin_batch_sync(kin_batch* batch);
/* Wait for the batch's stream and free the batch; the members stay. */
kin_status kin_batch_destroy(kin_batch* batch);
/* Message of the last error of this batch (or of the last failed
 * kin_batch_create on this thread when batch is NULL); never NULL. */
const char* kin_batch_last_error(const kin_batch* batch);

/* Block the host until the context's queued work is done. */
kin_status kin_sync(kin_ctx* ctx);

kin_status kin_query(const kin_ctx* ctx, kin_info* info);

/* Release every resource of the context (after synchronising its stream).
 * NULL is accepted. */
kin_status kin_destroy(kin_ctx* ctx);

/* Message of the last error of this context (or of the last failed
 * kin_create on this thread when ctx is NULL); never NULL. */
const char* kin_last_error(const kin_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif
