// kin_aux.h -- internal launch interface between the C ABI layer and the
// kernels (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>

namespace kin {

constexpr int kMaxNP = 4;          // degree <= 3
constexpr int kMaxVars = 6;        // conserved variables (Maxwell: E, H)
constexpr int kDiagBlocks = 304;   // 2 x 152 SMs

struct Inst;

struct SetupArgs {
    int dim, degree;
    double lambda, dt;
    double h[3];
    int B[3];
    double* c64;    // [2*dim][kCoefStride] FP64 coefficients
    float* c32;     // same, rounded to FP32 (NULL for an FP64 context)
    double* gll;    // xi[kMaxNP], w[kMaxNP]
};

struct PointArgs {
    int dim, degree, m, system, nvel;
    long long nodes;
    double lambda, gamma;
    double adv[3];
    double h[3];
};

struct DefectArgs {
    int dim, degree, m, iters;
    long long total;         // sum of per_pop
    long long per_pop[48];   // NS[a] * glines[a] for the population's axis
    long long glines[3];
    long long sig_stride;
    long long raw_stride;
    int nb[3], NS[3];
    double dt, lambda;
    double h[3];
};

typedef void (*StepKernel)(Inst);

// ---- d + 1 velocity sets (kin_simplex.cu) ----
constexpr int kSxMaxNN = 27;      // (p+1)^d <= 27 (3D p <= 2, 2D p <= 3)

struct SxSetupArgs {
    int dim, degree;
    double lambda, dt;
    double h[3];
    int stride;          // elements per velocity record
    double* c64;         // [d+1][stride] FP64 records
    double* minv;        // [(d+1)^2] inverse moment matrix
    double* work;        // [(d+1)][2 kSxMaxNN^2] scratch
};

struct SxArgs {
    void* f;
    const void* tr_in[3];         // per axis: [pop][NS_a][glines_a]
    void* tr_out[3];
    long long nodes;
    long long glines[3];
    long long trace_total;        // entries written by the trace pass
    int n[3], L[3], NS[3];
    int vsgn[4][3];               // sign of V_k along each axis (+1, -1, 0)
    int dim, degree, nn, m, nvel, npop, system;
    int from_f;                   // iterate 1: interface inflow is f^n of the upwind cell
    int final_iter;
    double omega, gamma;
    double adv[3];
    double minv[16];
};

cudaError_t sx_launch_setup(const SxSetupArgs& a, cudaStream_t st);
cudaError_t sx_launch_trace0(const SxArgs& a, int prec, cudaStream_t st);
// Launch plan of a sweep: threads per block (the subdomain's columns rounded
// to warps), dynamic shared memory, blocks per velocity, one launch per
// velocity (split) or one for all.
struct SxPlan {
    int threads, bpv, split, occupancy;
    size_t smem;
};
int sx_sweep_shape(const SxArgs& a, int prec, SxPlan* plan);   // host only: 0 if no shape fits
cudaError_t sx_sweep_plan(const SxArgs& a, int prec, SxPlan* plan);
cudaError_t sx_launch_sweep(const SxArgs& a, int prec, const double* hrec, int rstride, const SxPlan& plan,
                            cudaStream_t st);
cudaError_t sx_launch_relax(const SxArgs& a, int prec, cudaStream_t st);
cudaError_t sx_launch_init(const SxArgs& a, const double* W, int prec, cudaStream_t st);

// ---- tetrahedral meshes (kin_tet.cu) ----
constexpr int kTetRec = 21;       // coefficient slots per (velocity, cell): A^{-1}, |L|/20, four face factors
constexpr int kTetSweepThreads = 640;

struct TetSetupArgs {
    int ncells, nvel;
    const double* xyz;            // [cell][4][3] vertex coordinates
    double vel[6][3];             // V_k
    double dt;
    const unsigned char* ftype;   // [velocity][cell]: 2 bits per face a: 1 inflow, 2 outflow, 0 parallel
    const int* rank;              // [velocity][cell]: the cell's position in the velocity's level order
    double* c64;                  // [velocity][position][kTetRec] FP64 records, in level order
    float* c32;                   // FP32 copy (NULL for FP64)
};

struct TetArgs {
    int ncells, nvel, m, npop, nsub, system, velset;
    long long nodes;              // 4 ncells
    const void* coef;             // T records [velocity][position in order][kTetRec]
    const int* order;             // [velocity][ncells]: cells by subdomain, then breadth-first
    const int* lstart;            // [velocity][nsub + 1]: first level index of each subdomain in bounds
    const int* bounds;            // level l of the order holds positions [bounds[l], bounds[l + 1])
    const int* fref;              // [velocity][position][face a]: neighbour cell << 7 | its local index of
                                  // the face's vertices (bits 5, 3, 1) | 1 at an interface; -1 if not inflow
    void* f;                      // T [pop][cell][4]
    double lambda, gamma, omega, mu;
    double adv[3];
    int sgn[4][3];                // D3Q4 velocity signs
};

cudaError_t tet_launch_setup(const TetSetupArgs& a, cudaStream_t st);
cudaError_t tet_launch_sweep(const TetArgs& a, const void* prev, void* cur, int prec, cudaStream_t st);
cudaError_t tet_launch_relax(const TetArgs& a, const void* star, int prec, cudaStream_t st);
cudaError_t tet_launch_init(const TetArgs& a, const double* W, int prec, cudaStream_t st);

cudaError_t launch_setup(const SetupArgs& a, cudaStream_t st);
cudaError_t launch_init(const PointArgs& a, const double* W, void* f, int prec, cudaStream_t st);
// host: the 2d-velocity Maxwellians M[(2a + s) m + v] of one state (FP64)
void axis_maxwellian(const PointArgs& a, const double* W, double* M);
cudaError_t launch_moments(const PointArgs& a, const void* f, double* W, int prec, cudaStream_t st);
cudaError_t launch_mass(const PointArgs& a, const void* f, const double* gll, double* partial,
                        double* out, int prec, cudaStream_t st);
cudaError_t launch_defect(const DefectArgs& a, const void* sig, const void* raw, const double* c64,
                          const double* gll, double* partial, double* out, int prec,
                          cudaStream_t st);

// A compiled fixed-shape step kernel (see kin_fixed.cuh).
struct FixedKernel {
    StepKernel fn;           // single problem: fn(Inst)
    const void* batch_fn;    // several problems: batch_fn(const Inst*, const int2*, int)
    int threads;
    size_t smem;
};

// A compiled one-launch kernel for batches of 2D Euler FP32 problems of
// degrees 1..3 (step_kernel_mixed2d): fn(const Inst*, const int2*, int).
// block[p - 1] is the cell block a member of degree p must use to join it.
struct MixedKernel {
    const void* fn;
    int threads;
    int min_blocks;          // resident blocks per SM the kernel is built for
    size_t smem;
    int block[3][2];
};
// The compiled mixed kernels (at most max of them); returns their count.
int mixed_kernels_2d(MixedKernel* out, int max);

// Fixed-shape kernel for (degree, system, precision, block) with one or two
// shared-memory tile buffers, or fn == nullptr.
FixedKernel fixed_kernel_d2(int degree, int system, int prec, const int B[3], int stages);
FixedKernel fixed_kernel_d3(int degree, int system, int prec, const int B[3], int stages);
// Tile buffers the fixed-shape kernel of a shape uses unless asked otherwise.
int fixed_default_stages(int dim, int degree, int system, int prec, const int B[3]);
// Preferred fixed block shapes for a (dim, degree, system, precision), best first;
// returns the count written (at most 4).
int fixed_shapes(int dim, int degree, int system, int prec, int out[4][3]);

// Step kernels, one translation unit per space dimension.
StepKernel step_kernel_d1(int degree, int system, int prec);
StepKernel step_kernel_d2(int degree, int system, int prec);
StepKernel step_kernel_d3(int degree, int system, int prec);

}  // namespace kin
