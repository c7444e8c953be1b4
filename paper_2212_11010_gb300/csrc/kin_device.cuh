// kin_device.cuh -- device-side pieces of the kinetic DG step (internal).
//
// One thread block owns a box of B[0] x B[1] x B[2] cells ("cell block") and
// every population on it.  A step launch does, per cell block:
//   1. load f^n of all populations of the block into shared memory;
//   2. transport (Sec. 3.2 downwind algorithm, Sec. 5.1 subdomain iteration):
//      for an axis-aligned velocity every (cell row, transverse node) line of
//      the block is an independent 1D recurrence.  Its inflow trace is
//      obtained from the block summaries written by the previous launch (see
//      below); the line is then swept in downwind order, each cell applying
//      the precomputed local block inverse to its mass term plus the upwind
//      trace (eq. dg_imp, Crank-Nicolson half step), and f^{n+1} = 2f* - f^n
//      replaces f^n in place (Sec. 3.2: the solution replaces the data);
//   3. relaxation at every node (eq. over_relaxation), fused;
//   4. block summaries of the relaxed state for the next step: per line, the
//      outflow trace that the block would produce from a zero inflow
//      ("sigma") and the raw outflow-node value of the relaxed f ("raw");
//   5. store f^{n+1}.
//
// Why summaries reproduce the K-iteration of eq. ibvp exactly: the outflow
// trace of a cell is affine in its inflow trace, t_out = prow . u + rho t_in,
// so the outflow of a whole block is sigma_b + rho^{B} t_in.  Iterate p of a
// subdomain S takes its inflow from iterate p-1 of the upwind subdomain S-1,
// and iterate 0 is the data at t^n.  Unrolling, the inflow of subdomain S at
// the final iterate K is
//     A_{S-1} o A_{S-2} o ... o A_{S-K+1} ( raw(S-K) ),
// where A_j is the affine map of subdomain j (the composition of its blocks'
// maps) and raw(S-K) the t^n outflow-node value of subdomain S-K (periodic
// indices).  Inside S, a block's inflow is the composition of the preceding
// blocks of S applied to that.  This is the same linear algebra as K Jacobi
// sweeps, so f moves through HBM once per step (read + write) instead of K
// times.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace kin {

constexpr int kAdvection = 0;
constexpr int kEuler = 1;
constexpr int kCoefStride = 32;    // coefficient slots per (axis, sign)
constexpr int kThreads = 256;

// coefficient slot layout inside one (axis, sign) record
//   [0, NP*NP)            Pm = A^{-1} W - I  (row-major)
//   [16, 16 + NP)         g  = nu A^{-1} e_in
//   [20, 20 + NP)         prow = row 'out' of A^{-1} W
//   24                    rho = g[out]   (one-cell trace gain)
//   25                    rho^{B_a}      (one-block trace gain)
constexpr int kOffG = 16;
constexpr int kOffProw = 20;
constexpr int kOffRho = 24;
constexpr int kOffRhoB = 25;

struct Inst {
    void* f;                 // T*: [pop][cells][nodes], updated in place
    const void* sig_in;      // T*: block summaries of the current state
    const void* raw_in;
    void* sig_out;           // T*: summaries of the state this launch writes
    void* raw_out;
    const void* coef;        // T*: 2*dim records of kCoefStride
    long long nodes;         // cells * nodes per cell
    long long sig_stride;    // elements per population in sig/raw
    int n[3];                // cells per axis
    int B[3];                // cell-block extents
    int nblk[3];             // blocks per axis
    int nb[3];               // blocks per subdomain along each axis
    int NS[3];               // subdomains along each axis
    int iters;               // K
    int mode;                // 0: full step, 1: summaries only (no transport, no store)
    double lambda, gamma, omega;
    double adv[3];
};

__host__ __device__ constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }

template <typename T>
__device__ __forceinline__ T ldc(const T* p) { return __ldg(p); }

// Compensated (Kahan) accumulation, used for W = sum_k f_k in FP32.
template <typename T>
struct Acc {
    T s, c;
    __device__ __forceinline__ Acc() : s(0), c(0) {}
    __device__ __forceinline__ void add(T x)
    {
        T y = x - c;
        T t = s + y;
        c = (t - s) - y;
        s = t;
    }
};
template <>
struct Acc<double> {
    double s;
    __device__ __forceinline__ Acc() : s(0) {}
    __device__ __forceinline__ void add(double x) { s += x; }
};

// Flux Q^a(W) of the conservation law (eq. conslaw): advection a_a u, or the
// Euler flux of a gamma-law gas.
template <int D, int SYS, typename T>
__device__ __forceinline__ void flux(const Inst& I, const T* W, int a, T* Q)
{
    if (SYS == kAdvection) {
        Q[0] = T(I.adv[a]) * W[0];
    } else {
        const T rho = W[0];
        const T inv = T(1) / rho;
        T ke = 0;
#pragma unroll
        for (int b = 0; b < D; ++b) ke += W[1 + b] * W[1 + b];
        const T E = W[1 + D];
        const T pr = T(I.gamma - 1.0) * (E - T(0.5) * ke * inv);
        const T ua = W[1 + a] * inv;
        Q[0] = W[1 + a];
#pragma unroll
        for (int b = 0; b < D; ++b) Q[1 + b] = W[1 + b] * ua + (b == a ? pr : T(0));
        Q[1 + D] = (E + pr) * ua;
    }
}

// Geometry of the lines of one axis inside a cell block.
template <int D, int NP>
struct LineGeom {
    int cs;        // shared-memory stride between consecutive cells along a
    int ns;        // stride between consecutive nodes along a
    int base;      // shared-memory offset of the line's first element (pop 0)
    long long gline;   // global line id within the population's summary slab
    long long glines;  // lines per summary row for this axis
};

// Decompose (axis a, local line id) into shared-memory addressing and the
// global line id.  Local line id = tnode + NP^{D-1} * tcell with tnode the
// transverse node index and tcell the transverse cell index in the block.
template <int D, int NP>
__device__ __forceinline__ LineGeom<D, NP> line_geom(const Inst& I, int a, int line,
                                                     int bx, int by, int bz)
{
    constexpr int NN = ipow(NP, D);
    constexpr int TN = ipow(NP, D - 1);
    const int B0 = I.B[0], B1 = D > 1 ? I.B[1] : 1;
    LineGeom<D, NP> G;
    const int tnode = line % TN;
    const int tcell = line / TN;
    const int jt1 = tnode % NP, jt2 = tnode / NP;
    int c[3] = {0, 0, 0};   // local cell coordinates (axis a entry = 0)
    int j[3] = {0, 0, 0};   // node coordinates (axis a entry = 0)
    int t1 = -1, t2 = -1;   // transverse axes
    for (int b = 0; b < D; ++b) {
        if (b == a) continue;
        if (t1 < 0) t1 = b; else t2 = b;
    }
    if (t1 >= 0) {
        const int e1 = I.B[t1];
        c[t1] = tcell % e1;
        if (t2 >= 0) c[t2] = tcell / e1;
        j[t1] = jt1;
        if (t2 >= 0) j[t2] = jt2;
    }
    const int cstr[3] = {1, B0, B0 * B1};
    const int nstr[3] = {1, NP, NP * NP};
    G.cs = cstr[a] * NN;
    G.ns = nstr[a];
    G.base = (c[0] * cstr[0] + c[1] * cstr[1] + c[2] * cstr[2]) * NN + j[0] + j[1] * NP + j[2] * NP * NP;
    // global transverse cell index: row-major over the transverse axes
    const int org[3] = {bx * I.B[0], by * (D > 1 ? I.B[1] : 1), bz * (D > 2 ? I.B[2] : 1)};
    long long gt = 0;
    if (t2 >= 0) gt = (long long)(org[t2] + c[t2]) * I.n[t1] + (org[t1] + c[t1]);
    else if (t1 >= 0) gt = org[t1] + c[t1];
    G.gline = gt * TN + tnode;
    long long trans_cells = 1;
    for (int b = 0; b < D; ++b)
        if (b != a) trans_cells *= I.n[b];
    G.glines = trans_cells * TN;
    return G;
}

template <int D>
__device__ __forceinline__ int items_per_axis(const Inst& I, int a, int NP, int m)
{
    int bc = 1;
    for (int b = 0; b < D; ++b) bc *= I.B[b];
    int tn = 1;
    for (int b = 1; b < D; ++b) tn *= NP;
    return 2 * m * (bc / I.B[a]) * tn;
}

// The fused step on one cell block.  s: dynamic shared memory holding
// NPOP * cells * NN values of T.
template <int D, int P, int SYS, typename T>
__device__ void step_block(const Inst& I, int bx, int by, int bz, T* s)
{
    constexpr int NP = P + 1;
    constexpr int NN = ipow(NP, D);
    constexpr int M = SYS == kAdvection ? 1 : D + 2;
    constexpr int NV = 2 * D;
    constexpr int NPOP = NV * M;
    constexpr int TN = ipow(NP, D - 1);

    const int B0 = I.B[0];
    const int B1 = D > 1 ? I.B[1] : 1;
    const int B2 = D > 2 ? I.B[2] : 1;
    const int bcells = B0 * B1 * B2;
    const int x0 = bx * B0, y0 = by * B1, z0 = bz * B2;
    T* __restrict__ f = static_cast<T*>(I.f);
    const int tid = threadIdx.x;
    const int nth = blockDim.x;

    // ---- 1. load the block (rows of B0 cells are contiguous in HBM) ----
    const int rowlen = B0 * NN;
    const int nrows = B1 * B2;
    const int nload = NPOP * nrows * rowlen;
    for (int idx = tid; idx < nload; idx += nth) {
        const int e = idx % rowlen;
        const int t = idx / rowlen;
        const int row = t % nrows;
        const int pop = t / nrows;
        const int ly = row % B1, lz = row / B1;
        const long long g = (long long)pop * I.nodes
            + (((long long)(z0 + lz) * (D > 1 ? I.n[1] : 1) + (y0 + ly)) * I.n[0] + x0) * NN + e;
        s[(pop * bcells + row * B0) * NN + e] = f[g];
    }
    __syncthreads();

    const T* __restrict__ coef = static_cast<const T*>(I.coef);
    int ia[3];
    int total = 0;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        ia[a] = items_per_axis<D>(I, a, NP, M);
        total += ia[a];
    }

    // ---- 2. transport of every (population, line) of the block ----
    if (I.mode == 0) {
        const T* __restrict__ sig = static_cast<const T*>(I.sig_in);
        const T* __restrict__ raw = static_cast<const T*>(I.raw_in);
        for (int item = tid; item < total; item += nth) {
            int a = 0, it = item;
            while (it >= ia[a]) { it -= ia[a]; ++a; }
            const int lines = ia[a] / (2 * M);
            const int pl = it / lines;
            const int line = it % lines;
            const int sgn = pl / M, v = pl % M;
            const int pop = (2 * a + sgn) * M + v;
            const LineGeom<D, NP> G = line_geom<D, NP>(I, a, line, bx, by, bz);
            const int bidx = a == 0 ? bx : (a == 1 ? by : bz);
            const int nbk = I.nblk[a];
            const int q = sgn == 0 ? bidx : nbk - 1 - bidx;   // downwind block order
            const int nb = I.nb[a], NS = I.NS[a];
            const int S = q / nb, r = q % nb;
            const T* rec = coef + (2 * a + sgn) * kCoefStride;
            const T RB = ldc(rec + kOffRhoB);
            const long long pbase = (long long)pop * I.sig_stride + G.gline;
            // inflow of the final iterate (see the header comment)
            int s0 = (S - I.iters) % NS;
            if (s0 < 0) s0 += NS;
            T t = raw[pbase + (long long)(s0 * nb + nb - 1) * G.glines];
            for (int jj = 1; jj < I.iters; ++jj) {
                int sj = (S - I.iters + jj) % NS;
                if (sj < 0) sj += NS;
                for (int rr = 0; rr < nb; ++rr)
                    t = fma(RB, t, sig[pbase + (long long)(sj * nb + rr) * G.glines]);
            }
            for (int rr = 0; rr < r; ++rr)
                t = fma(RB, t, sig[pbase + (long long)(S * nb + rr) * G.glines]);

            T Pm[NP][NP], g[NP];
#pragma unroll
            for (int i = 0; i < NP; ++i) {
                g[i] = ldc(rec + kOffG + i);
#pragma unroll
                for (int j = 0; j < NP; ++j) Pm[i][j] = ldc(rec + i * NP + j);
            }
            const int Ba = I.B[a];
            T* line_p = s + pop * bcells * NN + G.base;
            for (int cc = 0; cc < Ba; ++cc) {
                const int c = sgn == 0 ? cc : Ba - 1 - cc;
                T* p = line_p + c * G.cs;
                T u[NP], dlt[NP];
#pragma unroll
                for (int j = 0; j < NP; ++j) u[j] = p[j * G.ns];
#pragma unroll
                for (int i = 0; i < NP; ++i) {
                    T acc = g[i] * t;
#pragma unroll
                    for (int j = 0; j < NP; ++j) acc = fma(Pm[i][j], u[j], acc);
                    dlt[i] = acc;     // f* - f^n at node i
                }
                t = sgn == 0 ? u[NP - 1] + dlt[NP - 1] : u[0] + dlt[0];
#pragma unroll
                for (int i = 0; i < NP; ++i) p[i * G.ns] = fma(T(2), dlt[i], u[i]);
            }
        }
        __syncthreads();

        // ---- 3. relaxation at every node (eq. over_relaxation) ----
        const int nnodes = bcells * NN;
        const T omega = T(I.omega);
        const T inv2d = T(1.0 / (2.0 * D));
        const T inv2l = T(1.0 / (2.0 * I.lambda));
        for (int nd = tid; nd < nnodes; nd += nth) {
            T fk[NPOP];
#pragma unroll
            for (int pp = 0; pp < NPOP; ++pp) fk[pp] = s[pp * bcells * NN + nd];
            T W[M];
#pragma unroll
            for (int v = 0; v < M; ++v) {
                Acc<T> acc;
#pragma unroll
                for (int k = 0; k < NV; ++k) acc.add(fk[k * M + v]);
                W[v] = acc.s;
            }
#pragma unroll
            for (int a = 0; a < D; ++a) {
                T Q[M];
                flux<D, SYS, T>(I, W, a, Q);
#pragma unroll
                for (int v = 0; v < M; ++v) {
                    const T base = W[v] * inv2d;
                    const T half = Q[v] * inv2l;
                    const T mp = base + half, mm = base - half;
                    T& fp = fk[(2 * a) * M + v];
                    T& fm = fk[(2 * a + 1) * M + v];
                    if (I.omega == 2.0) {
                        fp = fma(T(2), mp, -fp);
                        fm = fma(T(2), mm, -fm);
                    } else {
                        fp = omega * mp + (T(1) - omega) * fp;
                        fm = omega * mm + (T(1) - omega) * fm;
                    }
                }
            }
#pragma unroll
            for (int pp = 0; pp < NPOP; ++pp) s[pp * bcells * NN + nd] = fk[pp];
        }
        __syncthreads();
    }

    // ---- 4. block summaries of the (relaxed) state for the next step ----
    {
        T* __restrict__ sig = static_cast<T*>(I.sig_out);
        T* __restrict__ raw = static_cast<T*>(I.raw_out);
        for (int item = tid; item < total; item += nth) {
            int a = 0, it = item;
            while (it >= ia[a]) { it -= ia[a]; ++a; }
            const int lines = ia[a] / (2 * M);
            const int pl = it / lines;
            const int line = it % lines;
            const int sgn = pl / M, v = pl % M;
            const int pop = (2 * a + sgn) * M + v;
            const LineGeom<D, NP> G = line_geom<D, NP>(I, a, line, bx, by, bz);
            const int bidx = a == 0 ? bx : (a == 1 ? by : bz);
            const int q = sgn == 0 ? bidx : I.nblk[a] - 1 - bidx;
            const T* rec = coef + (2 * a + sgn) * kCoefStride;
            T prow[NP];
#pragma unroll
            for (int j = 0; j < NP; ++j) prow[j] = ldc(rec + kOffProw + j);
            const T rho = ldc(rec + kOffRho);
            const int Ba = I.B[a];
            const T* line_p = s + pop * bcells * NN + G.base;
            T t = 0, last = 0;
            for (int cc = 0; cc < Ba; ++cc) {
                const int c = sgn == 0 ? cc : Ba - 1 - cc;
                const T* p = line_p + c * G.cs;
                T acc = rho * t;
#pragma unroll
                for (int j = 0; j < NP; ++j) acc = fma(prow[j], p[j * G.ns], acc);
                t = acc;
                last = sgn == 0 ? p[(NP - 1) * G.ns] : p[0];
            }
            const long long o = (long long)pop * I.sig_stride + (long long)q * G.glines + G.gline;
            sig[o] = t;
            raw[o] = last;
        }
    }
    (void)TN;

    // ---- 5. store f^{n+1} ----
    if (I.mode == 0) {
        for (int idx = tid; idx < nload; idx += nth) {
            const int e = idx % rowlen;
            const int t = idx / rowlen;
            const int row = t % nrows;
            const int pop = t / nrows;
            const int ly = row % B1, lz = row / B1;
            const long long g = (long long)pop * I.nodes
                + (((long long)(z0 + lz) * (D > 1 ? I.n[1] : 1) + (y0 + ly)) * I.n[0] + x0) * NN + e;
            f[g] = s[(pop * bcells + row * B0) * NN + e];
        }
    }
}

template <int D, int P, int SYS, typename T>
__global__ void __launch_bounds__(kThreads) step_kernel(Inst I)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* s = reinterpret_cast<T*>(smem_raw);
    const int b = blockIdx.x;
    const int bx = b % I.nblk[0];
    const int by = (b / I.nblk[0]) % I.nblk[1];
    const int bz = b / (I.nblk[0] * I.nblk[1]);
    step_block<D, P, SYS, T>(I, bx, by, bz, s);
}

}  // namespace kin
