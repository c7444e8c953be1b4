// kin_aux.cu -- FP64 preprocessing and the non-hot-path kernels: local block
// inverses (once per context), f = M(W), W = sum_k f_k and the FP64
// conservation diagnostics.
#include "kin_aux.h"
#include "kin_device.cuh"

#include <math.h>

namespace kin {

// ---------------------------------------------------------------------------
// Preprocessing (Sec. 3.2: done once, before the time loop), all in FP64 on
// the device, one thread per (axis, sign).
// ---------------------------------------------------------------------------

// Legendre P_p and its derivative at x (|x| < 1) by the three-term recurrence.
__device__ static void legendre_pd(int p, double x, double* P, double* dP)
{
    double a = 1.0, b = x;
    for (int k = 1; k < p; ++k) {
        double c = ((2 * k + 1) * x * b - k * a) / (k + 1);
        a = b;
        b = c;
    }
    *P = b;
    *dP = p * (a - x * b) / (1.0 - x * x);
}

// Gauss-Lobatto nodes on [0,1] and weights (sum 1): interior nodes are the
// zeros of P_p', refined by Newton with P_p'' from Legendre's equation
// (1 - x^2) P'' = 2x P' - p(p+1) P.
__device__ static void gll01(int p, double* xi, double* w)
{
    for (int j = 0; j <= p; ++j) {
        double x = -cos(M_PI * j / p);
        if (j > 0 && j < p) {
            for (int it = 0; it < 60; ++it) {
                double P, dP;
                legendre_pd(p, x, &P, &dP);
                double d2P = (2.0 * x * dP - p * (p + 1.0) * P) / (1.0 - x * x);
                double step = dP / d2P;
                x -= step;
                if (fabs(step) < 1e-17) break;
            }
        }
        double Pend;
        if (j == 0) Pend = (p % 2) ? -1.0 : 1.0;
        else if (j == p) Pend = 1.0;
        else {
            double dP;
            legendre_pd(p, x, &Pend, &dP);
        }
        xi[j] = (j == 0) ? 0.0 : (j == p ? 1.0 : 0.5 * (x + 1.0));
        w[j] = 1.0 / (p * (p + 1.0) * Pend * Pend);
    }
}

__global__ void setup_kernel(SetupArgs A)
{
    const int dir = threadIdx.x;
    const int p = A.degree, np = p + 1;
    double xi[kMaxNP], w[kMaxNP];
    gll01(p, xi, w);
    if (dir == 0)
        for (int j = 0; j < np; ++j) {
            A.gll[j] = xi[j];
            A.gll[kMaxNP + j] = w[j];
        }
    if (dir >= 2 * A.dim) return;
    const int a = dir / 2, sgn = dir % 2;

    // differentiation matrix from barycentric weights: D_ij = (b_j / b_i) /
    // (xi_i - xi_j) for i != j, rows summing to zero.
    double bw[kMaxNP], Dm[kMaxNP][kMaxNP];
    for (int i = 0; i < np; ++i) {
        double prod = 1.0;
        for (int k = 0; k < np; ++k)
            if (k != i) prod *= xi[i] - xi[k];
        bw[i] = 1.0 / prod;
    }
    for (int i = 0; i < np; ++i) {
        double diag = 0.0;
        for (int j = 0; j < np; ++j) {
            if (j == i) continue;
            Dm[i][j] = (bw[j] / bw[i]) / (xi[i] - xi[j]);
            diag -= Dm[i][j];
        }
        Dm[i][i] = diag;
    }

    // local block of one line (eq. dg_imp on a cell of unit size, divided by
    // h; transverse quadrature weights cancel for an axis-aligned velocity):
    //   V > 0:  A = W + nu (Q + e_0 e_0^T),   inflow at node 0, outflow at p
    //   V < 0:  A = W + nu (-Q + e_p e_p^T),  inflow at node p, outflow at 0
    // with W = diag(w), Q = W D, nu = lambda (dt/2) / h_a.
    const double nu = A.lambda * 0.5 * A.dt / A.h[a];
    const int in = sgn == 0 ? 0 : p;
    const int out = sgn == 0 ? p : 0;
    double M[kMaxNP][2 * kMaxNP];
    for (int i = 0; i < np; ++i)
        for (int j = 0; j < np; ++j) {
            double q = w[i] * Dm[i][j];
            double v = (i == j ? w[i] : 0.0) + nu * (sgn == 0 ? q : -q);
            if (i == in && j == in) v += nu;
            M[i][j] = v;
            M[i][np + j] = (i == j) ? 1.0 : 0.0;
        }
    // Gauss-Jordan inverse with partial pivoting
    for (int c = 0; c < np; ++c) {
        int piv = c;
        for (int r = c + 1; r < np; ++r)
            if (fabs(M[r][c]) > fabs(M[piv][c])) piv = r;
        if (piv != c)
            for (int j = 0; j < 2 * np; ++j) {
                double t = M[c][j];
                M[c][j] = M[piv][j];
                M[piv][j] = t;
            }
        double d = 1.0 / M[c][c];
        for (int j = 0; j < 2 * np; ++j) M[c][j] *= d;
        for (int r = 0; r < np; ++r) {
            if (r == c) continue;
            double l = M[r][c];
            if (l != 0.0)
                for (int j = 0; j < 2 * np; ++j) M[r][j] -= l * M[c][j];
        }
    }
    double* rec = A.c64 + dir * kCoefStride;
    for (int k = 0; k < kCoefStride; ++k) rec[k] = 0.0;
    for (int i = 0; i < np; ++i) {
        for (int j = 0; j < np; ++j) {
            double P = M[i][np + j] * w[j];     // (A^{-1} W)_{ij}
            rec[i * np + j] = P - (i == j ? 1.0 : 0.0);
            if (i == out) rec[kOffProw + j] = P;
        }
        rec[kOffG + i] = nu * M[i][np + in];
    }
    const double rho = rec[kOffG + out];
    rec[kOffRho] = rho;
    double rb = 1.0;
    for (int k = 0; k < A.B[a]; ++k) rb *= rho;
    rec[kOffRhoB] = rb;
    if (A.c32)
        for (int k = 0; k < kCoefStride; ++k) A.c32[dir * kCoefStride + k] = (float)rec[k];
}

// ---------------------------------------------------------------------------
// point-wise kernels (grid-stride over nodes)
// ---------------------------------------------------------------------------

// Flux in FP64 (eq. conslaw): scalar advection, Euler, or Maxwell in 3D
// (Sec. 6.1.1: Q(W, e_a) = (-e_a x H, e_a x E), W = (E, H)).
__host__ __device__ static void flux64(const PointArgs& A, const double* W, int a, double* Q)
{
    if (A.system == kAdvection) {
        Q[0] = A.adv[a] * W[0];
        return;
    }
    if (A.system == kMaxwell) {
        const int j = (a + 1) % 3, k = (a + 2) % 3;     // e_a x v = v_j e_k - v_k e_j
        Q[a] = 0.0;
        Q[k] = -W[3 + j];
        Q[j] = W[3 + k];
        Q[3 + a] = 0.0;
        Q[3 + k] = W[j];
        Q[3 + j] = -W[k];
        return;
    }
    const int d = A.dim;
    double ke = 0.0;
    for (int b = 0; b < d; ++b) ke += W[1 + b] * W[1 + b];
    const double rho = W[0], E = W[1 + d];
    const double pr = (A.gamma - 1.0) * (E - 0.5 * ke / rho);
    const double ua = W[1 + a] / rho;
    Q[0] = W[1 + a];
    for (int b = 0; b < d; ++b) Q[1 + b] = W[1 + b] * ua + (b == a ? pr : 0.0);
    Q[1 + d] = (E + pr) * ua;
}

// The 2d-velocity Maxwellians of one state on the host, in FP64, with the
// formulas of init_kernel: M[(2a + s) m + v] = W_v/(2d) +- Q^a(W)_v/(2 lambda).
void axis_maxwellian(const PointArgs& A, const double* W, double* M)
{
    double Q[kMaxVars];
    for (int a = 0; a < A.dim; ++a) {
        flux64(A, W, a, Q);
        for (int v = 0; v < A.m; ++v) {
            const double base = W[v] / (2.0 * A.dim), half = Q[v] / (2.0 * A.lambda);
            M[(2 * a) * A.m + v] = base + half;
            M[(2 * a + 1) * A.m + v] = base - half;
        }
    }
}

// f = M(W) (Sec. 2.2 initialisation), W in FP64, f stored in T.
template <typename T>
__global__ void init_kernel(PointArgs A, const double* __restrict__ W, T* __restrict__ f)
{
    const long long nodes = A.nodes;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nodes;
         i += (long long)gridDim.x * blockDim.x) {
        double w[kMaxVars], Q[kMaxVars];
        for (int v = 0; v < A.m; ++v) w[v] = W[v * nodes + i];
        for (int a = 0; a < A.dim; ++a) {
            flux64(A, w, a, Q);
            for (int v = 0; v < A.m; ++v) {
                const double base = w[v] / (2.0 * A.dim), half = Q[v] / (2.0 * A.lambda);
                f[((2 * a) * A.m + v) * nodes + i] = (T)(base + half);
                f[((2 * a + 1) * A.m + v) * nodes + i] = (T)(base - half);
            }
        }
    }
}

// W = sum_k f_k in FP64 (k ascending).
template <typename T>
__global__ void moments_kernel(PointArgs A, const T* __restrict__ f, double* __restrict__ W)
{
    const long long nodes = A.nodes;
    const int nv = A.nvel;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nodes;
         i += (long long)gridDim.x * blockDim.x) {
        for (int v = 0; v < A.m; ++v) {
            double s = 0.0;
            for (int k = 0; k < nv; ++k) s += (double)f[(k * A.m + v) * nodes + i];
            W[v * nodes + i] = s;
        }
    }
}

// Deterministic FP64 reductions: every block writes one partial per output
// slot, a single block then adds the partials in block order.
template <int NOUT>
__device__ static void block_reduce_store(double (&val)[NOUT], double* partial, bool is_max)
{
    __shared__ double red[kThreads / 32][NOUT];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int o = 0; o < NOUT; ++o) {
        double x = val[o];
        for (int off = 16; off; off >>= 1) {
            double y = __shfl_down_sync(0xffffffffu, x, off);
            x = is_max ? fmax(x, y) : x + y;
        }
        if (lane == 0) red[wid][o] = x;
    }
    __syncthreads();
    if (threadIdx.x < NOUT) {
        double x = is_max ? 0.0 : 0.0;
        for (int wv = 0; wv < (int)(blockDim.x / 32); ++wv)
            x = is_max ? fmax(x, red[wv][threadIdx.x]) : x + red[wv][threadIdx.x];
        partial[blockIdx.x * NOUT + threadIdx.x] = x;
    }
}

// Quadrature mass per variable of W = sum_k f_k: sum_nodes |cell| prod w * W.
template <typename T>
__global__ void mass_kernel(PointArgs A, const T* __restrict__ f, const double* __restrict__ gll,
                            double* __restrict__ partial)
{
    const long long nodes = A.nodes;
    const int np = A.degree + 1, nv = A.nvel;
    int nn = 1;
    for (int a = 0; a < A.dim; ++a) nn *= np;
    double vol = 1.0;
    for (int a = 0; a < A.dim; ++a) vol *= A.h[a];
    double acc[kMaxVars] = {0, 0, 0, 0, 0, 0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nodes;
         i += (long long)gridDim.x * blockDim.x) {
        int id = (int)(i % nn);
        double wq = vol;
        for (int a = 0; a < A.dim; ++a) {
            wq *= gll[kMaxNP + id % np];
            id /= np;
        }
        for (int v = 0; v < A.m; ++v) {
            double s = 0.0;
            for (int k = 0; k < nv; ++k) s += (double)f[(k * A.m + v) * nodes + i];
            acc[v] += wq * s;
        }
    }
    block_reduce_store<kMaxVars>(acc, partial, false);
}

// Next-step interface defect and iteration residual from the block
// summaries: for every population, line and subdomain S the trace that the
// final iterate takes as inflow (K-1 subdomain maps applied to raw(S-K)) and
// the upwind subdomain's own final outflow (K maps applied to raw(S-K-1)).
template <typename T>
__global__ void defect_kernel(DefectArgs A, const T* __restrict__ sig, const T* __restrict__ raw,
                              const double* __restrict__ c64, const double* __restrict__ gll,
                              double* __restrict__ partial, double* __restrict__ partial_max)
{
    double acc[kMaxVars] = {0, 0, 0, 0, 0, 0};
    double mx[1] = {0.0};
    const int np = A.degree + 1;
    int tn = 1;
    for (int b = 1; b < A.dim; ++b) tn *= np;
    for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < A.total;
         it += (long long)gridDim.x * blockDim.x) {
        // decompose: pop-major, then subdomain, then line
        long long rest = it;
        int pop = 0;
        while (rest >= A.per_pop[pop]) { rest -= A.per_pop[pop]; ++pop; }
        const int k = pop / A.m, v = pop % A.m, a = k / 2;
        const long long glines = A.glines[a];
        const int S = (int)(rest / glines);
        const long long gl = rest % glines;
        const int nb = A.nb[a], NS = A.NS[a], K = A.iters;
        const double RB = c64[k * kCoefStride + kOffRhoB];
        const T* sigp = sig + (long long)pop * A.sig_stride;
        const T* rawp = raw + (long long)pop * A.raw_stride;
        // inflow of subdomain S after 'maps' whole upwind subdomains, starting
        // from the raw outflow value of subdomain S - maps - 1
        auto chain = [&](int maps) {
            int s0 = (S - maps - 1) % NS;
            if (s0 < 0) s0 += NS;
            double t = (double)rawp[(long long)s0 * glines + gl];
            for (int j = 0; j < maps; ++j) {
                int sj = (S - maps + j) % NS;
                if (sj < 0) sj += NS;
                for (int rr = 0; rr < nb; ++rr)
                    t = RB * t + (double)sigp[(long long)(sj * nb + rr) * glines + gl];
            }
            return t;
        };
        const double used = chain(K - 1), actual = chain(K);
        // face quadrature weight of the line: prod over transverse axes of h_b w_{j_b}
        int tnode = (int)(gl % tn);
        double fw = 1.0;
        for (int b = 0; b < A.dim; ++b) {
            if (b == a) continue;
            fw *= A.h[b] * gll[kMaxNP + tnode % np];
            tnode /= np;
        }
        acc[v] += A.dt * A.lambda * fw * (used - actual);
        mx[0] = fmax(mx[0], fabs(used - actual));
    }
    block_reduce_store<kMaxVars>(acc, partial, false);
    __syncthreads();
    block_reduce_store<1>(mx, partial_max, true);
}

__global__ void finish_kernel(const double* partial, int nblocks, int nout, int is_max, double* out)
{
    const int o = threadIdx.x;
    if (o >= nout) return;
    double x = 0.0;
    for (int b = 0; b < nblocks; ++b) {
        double y = partial[b * nout + o];
        x = is_max ? fmax(x, y) : x + y;
    }
    out[o] = x;
}

// ---------------------------------------------------------------------------
// host-side launchers
// ---------------------------------------------------------------------------

cudaError_t launch_setup(const SetupArgs& a, cudaStream_t st)
{
    setup_kernel<<<1, 32, 0, st>>>(a);
    return cudaGetLastError();
}

static int grid_for(long long n)
{
    long long g = (n + kThreads - 1) / kThreads;
    if (g > 152 * 16) g = 152 * 16;
    return (int)(g < 1 ? 1 : g);
}

cudaError_t launch_init(const PointArgs& a, const double* W, void* f, int prec, cudaStream_t st)
{
    int g = grid_for(a.nodes);
    if (prec == 1) init_kernel<float><<<g, kThreads, 0, st>>>(a, W, (float*)f);
    else init_kernel<double><<<g, kThreads, 0, st>>>(a, W, (double*)f);
    return cudaGetLastError();
}

cudaError_t launch_moments(const PointArgs& a, const void* f, double* W, int prec, cudaStream_t st)
{
    int g = grid_for(a.nodes);
    if (prec == 1) moments_kernel<float><<<g, kThreads, 0, st>>>(a, (const float*)f, W);
    else moments_kernel<double><<<g, kThreads, 0, st>>>(a, (const double*)f, W);
    return cudaGetLastError();
}

cudaError_t launch_mass(const PointArgs& a, const void* f, const double* gll, double* partial,
                        double* out, int prec, cudaStream_t st)
{
    const int g = kDiagBlocks;
    if (prec == 1) mass_kernel<float><<<g, kThreads, 0, st>>>(a, (const float*)f, gll, partial);
    else mass_kernel<double><<<g, kThreads, 0, st>>>(a, (const double*)f, gll, partial);
    finish_kernel<<<1, 32, 0, st>>>(partial, g, kMaxVars, 0, out);
    return cudaGetLastError();
}

cudaError_t launch_defect(const DefectArgs& a, const void* sig, const void* raw, const double* c64,
                          const double* gll, double* partial, double* out, int prec,
                          cudaStream_t st)
{
    const int g = kDiagBlocks;
    double* pmax = partial + g * kMaxVars;
    if (prec == 1)
        defect_kernel<float><<<g, kThreads, 0, st>>>(a, (const float*)sig, (const float*)raw, c64,
                                                     gll, partial, pmax);
    else
        defect_kernel<double><<<g, kThreads, 0, st>>>(a, (const double*)sig, (const double*)raw,
                                                      c64, gll, partial, pmax);
    finish_kernel<<<1, 32, 0, st>>>(partial, g, kMaxVars, 0, out);
    finish_kernel<<<1, 32, 0, st>>>(pmax, g, 1, 1, out + kMaxVars);
    return cudaGetLastError();
}

}  // namespace kin
