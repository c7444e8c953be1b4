// kin_device.cuh -- device-side pieces of the kinetic DG step (internal).
//
// One thread block owns a box of B[0] x B[1] x B[2] cells ("cell block") and
// every population on it.  A step launch does, per cell block:
//   1. load f^n of all populations of the block into shared memory (bulk
//      copies of the contiguous rows of B[0] cells, completing on an
//      mbarrier);
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
//   5. store f^{n+1} (bulk copies).
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
// blocks of S applied to that.  In downwind block order this is one flat
// chain: start from the raw value of the block just before the first block
// of subdomain S-K+1 and fold in the sigma of every block up to the current
// one.  This is the same linear algebra as K Jacobi sweeps, so f moves
// through HBM once per step (read + write) instead of K times.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "kin_tma.cuh"

namespace kin {

constexpr int kAdvection = 0;
constexpr int kEuler = 1;
constexpr int kMaxwell = 2;        // 3D only: W = (E, H) (Sec. 6.1.1)
// conserved variables m of a system in D dimensions
__host__ __device__ constexpr int nvars(int D, int SYS) { return SYS == kAdvection ? 1 : (SYS == kMaxwell ? 6 : D + 2); }
constexpr int kCoefStride = 32;    // coefficient slots per (axis, sign)
constexpr int kMaxPop = 36;        // populations at most (axis velocities: 2d x m, Maxwell 6 x 6)
constexpr int kThreads = 256;      // upper bound on threads per block

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

// error word bits (Inst::err)
constexpr int kErrLoadTimeout = 1;

struct AxisInfo {
    FastDiv lines;      // lines of one population inside a block: (cells / B_a) * NP^{d-1}
    FastDiv e1;         // block extent along the first transverse axis
    long long glines;   // lines of one population in the whole mesh
};

struct __align__(16) Inst {
    void* f;                 // T*: [pop][cells][nodes], updated in place
    const void* sig_in;      // T*: block summaries of the current state
    const void* raw_in;
    void* sig_out;           // T*: summaries of the state this launch writes
    void* raw_out;
    int* err;                // device error word (OR of kErr* bits)
    long long nodes;         // cells * nodes per cell
    long long sig_stride;    // elements per population in sig: [block q][line]
    long long raw_stride;    // elements per population in raw: [S][line]
    long long wait_cycles;   // bound on the bulk-load wait, in SM clocks
    int n[3];                // cells per axis
    int B[3];                // cell-block extents
    int nblk[3];             // blocks per axis
    int nb[3];               // blocks per subdomain along each axis
    int NS[3];               // subdomains along each axis
    AxisInfo ax[3];
    FastDiv fd_nblk0;        // nblk[0]
    FastDiv fd_nblk01;       // nblk[0] * nblk[1]
    FastDiv fd_nb[3];        // nb[a]
    FastDiv fd_nrows;        // B[1] * B[2]
    FastDiv fd_B1;           // B[1]
    FastDiv fd_rowlen;       // B[0] * nodes per cell
    int iters;               // K
    int mode;                // 0: full step, 1: summaries only (no transport, no store)
    int tma;                 // 1: rows moved by bulk copies (alignment checked on the host)
    int stages;              // shared-memory tile buffers per thread block (1 or 2)
    int debug_stall;         // test hook: the load barrier expects 16 bytes that never arrive
    double lambda, gamma, omega;
    double mu;               // Maxwell: conductivity source factor (1 - sigma dt/2) / (1 + sigma dt/2)
    int inflow[3];           // 1: axis a has inflow boundaries instead of being periodic
    // look-back depth per (axis, sign): only the last lbdepth blocks of a walk
    // are folded; every earlier contribution reaches the inflow damped by
    // rho^B per block, i.e. by at most rho^(B lbdepth), which the host keeps
    // below 2^-36 (FP32) or 2^-72 (FP64) -- far below the rounding of the
    // result, so the truncated walk returns the same inflow up to rounding
    int lbdepth[6];
    // T*: inflow boundaries: per population the value across the
    // domain-boundary face it enters through, M_k(W_b)[v] of that face's state
    const void* bnd;
    double adv[3];
    // block-inverse coefficients (computed in FP64 on the device once per
    // context), carried in the launch parameters: read from the constant bank
    double cd[6][kCoefStride];
    float cf[6][kCoefStride];
};

template <typename T>
__device__ __forceinline__ const T* coef_rec(const Inst& I, int dir);
template <>
__device__ __forceinline__ const float* coef_rec<float>(const Inst& I, int dir) { return I.cf[dir]; }
template <>
__device__ __forceinline__ const double* coef_rec<double>(const Inst& I, int dir) { return I.cd[dir]; }

// One coefficient by direct member access (constant-bank operand when the
// indices are compile-time and I is the kernel parameter).
__device__ __forceinline__ float coef_of(const Inst& I, int dir, int k, float) { return I.cf[dir][k]; }
__device__ __forceinline__ double coef_of(const Inst& I, int dir, int k, double) { return I.cd[dir][k]; }

// Inflow of the final subdomain iterate for the line 'gline' of population
// 'pop' (axis a, sign sgn) entering block 'bidx' (see the header comment): the
// raw outflow value of subdomain S-K, then in downwind order the blocks of the
// K-1 whole subdomains S-K+1 .. S-1 and the blocks of S upwind of this one.
// Summaries are stored [block q (downwind order)][line], raw values
// [subdomain][line]; every load is coalesced across consecutive lines.
template <typename T>
__device__ __forceinline__ T bnd_of(const Inst& I, int pop)
{
    return __ldg(static_cast<const T*>(I.bnd) + pop);
}

template <typename T>
__device__ __forceinline__ T chain_inflow(const Inst& I, int a, int sgn, int bidx, int pop, long long gline)
{
    const int nbk = I.nblk[a], nb = I.nb[a], NS = I.NS[a], K = I.iters;
    const int q = sgn == 0 ? bidx : nbk - 1 - bidx;
    const int S = q / nb, r = q - (q / nb) * nb;
    const long long gl = I.ax[a].glines;
    const T* __restrict__ sig = static_cast<const T*>(I.sig_in) + (long long)pop * I.sig_stride + gline;
    const T* __restrict__ raw = static_cast<const T*>(I.raw_in) + (long long)pop * I.raw_stride + gline;
    const T RB = coef_of(I, 2 * a + sgn, kOffRhoB, T(0));
    int s0 = S - K;
    int cnt, q0;
    const bool from_bnd = I.inflow[a] && s0 < 0;
    if (from_bnd) {
        // the walk reaches the domain boundary within K subdomains: it starts
        // there from the boundary value (the same in every iteration) and
        // folds every block from the first one
        cnt = S * nb + r;
        q0 = 0;
    } else {
        while (s0 < 0) s0 += NS;
        cnt = (K - 1) * nb + r;
        q0 = (s0 + 1 == NS) ? 0 : (s0 + 1) * nb;
    }
    T t;
    const int depth = I.lbdepth[2 * a + sgn];
    if (cnt > depth) {
        // only the last 'depth' blocks matter (see Inst::lbdepth)
        q0 = (q0 + cnt - depth) % nbk;
        cnt = depth;
        t = T(0);
    } else {
        t = from_bnd ? bnd_of<T>(I, pop) : __ldg(raw + (long long)s0 * gl);
    }
    const T* p = sig + (long long)q0 * gl;
    // walk the summaries of blocks q0, q0+1, ... (periodic) by pointer stride
    const T* const end = sig + (long long)nbk * gl;
#pragma unroll 4
    for (int j = 0; j < cnt; ++j) {
        t = fma(RB, t, __ldg(p));
        p += gl;
        if (p == end) p = sig;
    }
    return t;
}

// Write the summaries of this block for line 'gline': sigma always, raw only
// for the downwind-most block of its subdomain.
template <typename T>
__device__ __forceinline__ void write_summary(const Inst& I, int a, int sgn, int bidx, int pop, long long gline,
                                              T sigma, T last)
{
    const int nbk = I.nblk[a], nb = I.nb[a];
    const int q = sgn == 0 ? bidx : nbk - 1 - bidx;
    const int S = q / nb, r = q - (q / nb) * nb;
    const long long gl = I.ax[a].glines;
    T* sig = static_cast<T*>(I.sig_out) + (long long)pop * I.sig_stride;
    T* raw = static_cast<T*>(I.raw_out) + (long long)pop * I.raw_stride;
    sig[(long long)q * gl + gline] = sigma;
    if (r == nb - 1) raw[(long long)S * gl + gline] = last;
}

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

// Geometry of one line of axis A inside the block.
template <int D, int NP, int A>
struct Line {
    int base;          // shared-memory offset of the line's first element (population 0)
    long long gline;   // global line id within a population's summary slab
};

template <int D, int NP, int A>
__device__ __forceinline__ Line<D, NP, A> line_of(const Inst& I, int line, int org0, int org1, int org2)
{
    constexpr int NN = ipow(NP, D);
    constexpr int TN = ipow(NP, D - 1);
    constexpr int T1 = A == 0 ? 1 : 0;                  // first transverse axis
    constexpr int T2 = A == 2 ? 1 : 2;                  // second transverse axis
    const int tnode = line % TN;
    const int tcell = line / TN;
    const int jt1 = tnode % NP, jt2 = tnode / NP;
    Line<D, NP, A> L;
    if (D == 1) {
        L.base = 0;
        L.gline = 0;
        return L;
    }
    const unsigned c2 = D == 3 ? fdiv((unsigned)tcell, I.ax[A].e1) : 0u;
    const unsigned c1 = (unsigned)tcell - c2 * I.ax[A].e1.d;
    const int B0 = I.B[0], B1 = I.B[1];
    const int cstr1 = T1 == 0 ? 1 : (T1 == 1 ? B0 : B0 * B1);
    const int cstr2 = T2 == 1 ? B0 : B0 * B1;
    constexpr int nstr1 = T1 == 0 ? 1 : (T1 == 1 ? NP : NP * NP);
    constexpr int nstr2 = T2 == 1 ? NP : NP * NP;
    L.base = ((int)c1 * cstr1 + (D == 3 ? (int)c2 * cstr2 : 0)) * NN + jt1 * nstr1 + (D == 3 ? jt2 * nstr2 : 0);
    const int org1v = T1 == 0 ? org0 : (T1 == 1 ? org1 : org2);
    const int org2v = T2 == 1 ? org1 : org2;
    long long gt;
    if (D == 3) gt = (long long)(org2v + (int)c2) * I.n[T1] + (org1v + (int)c1);
    else gt = org1v + (int)c1;
    L.gline = gt * TN + tnode;
    return L;
}

// Items of axis A: (population of axis A, line) pairs, line fastest.
template <int D, int P, int SYS, int A>
__device__ __forceinline__ int items_of_axis(const Inst& I)
{
    constexpr int M = nvars(D, SYS);
    return 2 * M * (int)I.ax[A].lines.d;
}

// Inflow traces of the final subdomain iterate for every item of axis A,
// folded from the block summaries of the previous launch, into tin[].  These
// loads do not depend on the tile's own data, so they run while the tile is
// still being copied in.
template <int D, int P, int SYS, typename T, int A>
__device__ __forceinline__ void chain_axis(const Inst& I, int bx, int by, int bz, T* tin)
{
    constexpr int NP = P + 1;
    constexpr int M = nvars(D, SYS);
    const int B0 = I.B[0], B1 = D > 1 ? I.B[1] : 1, B2 = D > 2 ? I.B[2] : 1;
    const int org0 = bx * B0, org1 = by * B1, org2 = bz * B2;
    const int Lp = (int)I.ax[A].lines.d;
    const int items = 2 * M * Lp;
    const int bidx = A == 0 ? bx : (A == 1 ? by : bz);
    for (int it = threadIdx.x; it < items; it += blockDim.x) {
        const int pl = (int)fdiv((unsigned)it, I.ax[A].lines);
        const int line = it - pl * Lp;
        const int sgn = pl / M, v = pl - (pl / M) * M;
        const int pop = (2 * A + sgn) * M + v;
        const Line<D, NP, A> G = line_of<D, NP, A>(I, line, org0, org1, org2);
        const T t = chain_inflow<T>(I, A, sgn, bidx, pop, G.gline);
        tin[it] = t;
    }
}

// Transport (phase 2) or summaries (phase 4) of every line of axis A.
template <int D, int P, int SYS, typename T, int A, bool SUMMARY>
__device__ __forceinline__ void lines_axis(const Inst& I, int bx, int by, int bz, T* s, const T* tin)
{
    constexpr int NP = P + 1;
    constexpr int NN = ipow(NP, D);
    constexpr int M = nvars(D, SYS);
    const int B0 = I.B[0], B1 = D > 1 ? I.B[1] : 1, B2 = D > 2 ? I.B[2] : 1;
    const int bcells = B0 * B1 * B2;
    const int org0 = bx * B0, org1 = by * B1, org2 = bz * B2;
    const int Lp = (int)I.ax[A].lines.d;
    const int items = 2 * M * Lp;
    const int cs = (A == 0 ? 1 : (A == 1 ? B0 : B0 * B1)) * NN;
    constexpr int ns = A == 0 ? 1 : (A == 1 ? NP : NP * NP);
    const int Ba = I.B[A];
    const int bidx = A == 0 ? bx : (A == 1 ? by : bz);

    for (int it = threadIdx.x; it < items; it += blockDim.x) {
        const int pl = (int)fdiv((unsigned)it, I.ax[A].lines);
        const int line = it - pl * Lp;
        const int sgn = pl / M, v = pl - (pl / M) * M;
        const int pop = (2 * A + sgn) * M + v;
        const Line<D, NP, A> G = line_of<D, NP, A>(I, line, org0, org1, org2);
        const T* rec = coef_rec<T>(I, 2 * A + sgn);
        T* line_p = s + pop * bcells * NN + G.base;

        if (!SUMMARY) {
            T t = tin[it];
            T Pm[NP][NP];
#pragma unroll
            for (int i = 0; i < NP; ++i)
#pragma unroll
                for (int j = 0; j < NP; ++j) Pm[i][j] = rec[i * NP + j];
#pragma unroll 4
            for (int cc = 0; cc < Ba; ++cc) {
                const int c = sgn == 0 ? cc : Ba - 1 - cc;
                T* p = line_p + c * cs;
                T u[NP], du[NP], dlt[NP];
#pragma unroll
                for (int j = 0; j < NP; ++j) {
                    u[j] = p[j * ns];
                    du[j] = u[j] - t;
                }
                // f* - f^n at node i in difference form: (P - I) u + g t
                // = (P - I)(u - t 1), because (P - I) 1 + g = 0 (A 1 = W 1 +
                // nu e_in: the derivative of a constant vanishes).  A constant
                // state then stays exactly constant whatever the rounding of
                // the coefficients, which removes the systematic FP32 drift.
#pragma unroll
                for (int i = 0; i < NP; ++i) {
                    T acc = Pm[i][0] * du[0];
#pragma unroll
                    for (int j = 1; j < NP; ++j) acc = fma(Pm[i][j], du[j], acc);
                    dlt[i] = acc;
                }
                t = sgn == 0 ? u[NP - 1] + dlt[NP - 1] : u[0] + dlt[0];
#pragma unroll
                for (int i = 0; i < NP; ++i) p[i * ns] = fma(T(2), dlt[i], u[i]);
            }
        } else {
            T prow[NP];
#pragma unroll
            for (int j = 0; j < NP; ++j) prow[j] = rec[kOffProw + j];
            const T rho = rec[kOffRho];
            T t = 0, last = 0;
#pragma unroll 4
            for (int cc = 0; cc < Ba; ++cc) {
                const int c = sgn == 0 ? cc : Ba - 1 - cc;
                const T* p = line_p + c * cs;
                T u[NP];
#pragma unroll
                for (int j = 0; j < NP; ++j) u[j] = p[j * ns];
                T acc = prow[0] * u[0];
#pragma unroll
                for (int j = 1; j < NP; ++j) acc = fma(prow[j], u[j], acc);
                t = fma(rho, t, acc);
                last = sgn == 0 ? u[NP - 1] : u[0];
            }
            write_summary<T>(I, A, sgn, bidx, pop, G.gline, t, last);
        }
    }
}

template <int D, int P, int SYS, typename T>
__device__ __forceinline__ void chain_all(const Inst& I, int bx, int by, int bz, T* tin)
{
    chain_axis<D, P, SYS, T, 0>(I, bx, by, bz, tin);
    if constexpr (D > 1) chain_axis<D, P, SYS, T, 1>(I, bx, by, bz, tin + items_of_axis<D, P, SYS, 0>(I));
    if constexpr (D > 2)
        chain_axis<D, P, SYS, T, 2>(I, bx, by, bz,
                                    tin + items_of_axis<D, P, SYS, 0>(I) + items_of_axis<D, P, SYS, 1>(I));
}

template <int D, int P, int SYS, typename T, bool SUMMARY>
__device__ __forceinline__ void lines_all(const Inst& I, int bx, int by, int bz, T* s, const T* tin)
{
    lines_axis<D, P, SYS, T, 0, SUMMARY>(I, bx, by, bz, s, tin);
    if constexpr (D > 1)
        lines_axis<D, P, SYS, T, 1, SUMMARY>(I, bx, by, bz, s, tin + items_of_axis<D, P, SYS, 0>(I));
    if constexpr (D > 2)
        lines_axis<D, P, SYS, T, 2, SUMMARY>(I, bx, by, bz, s,
                                              tin + items_of_axis<D, P, SYS, 0>(I) + items_of_axis<D, P, SYS, 1>(I));
}

struct TileXYZ {
    int bx, by, bz;
};

__device__ __forceinline__ TileXYZ tile_xyz(const Inst& I, int t)
{
    TileXYZ c;
    c.bz = (int)fdiv((unsigned)t, I.fd_nblk01);
    const int rem = t - c.bz * (int)I.fd_nblk01.d;
    c.by = (int)fdiv((unsigned)rem, I.fd_nblk0);
    c.bx = rem - c.by * (int)I.fd_nblk0.d;
    return c;
}

// W / (2d), the equilibrium's isotropic part.  1/(2d) is exact in binary for
// d = 1, 2.  For d = 3 a product with the rounded 1/6 would carry the same
// relative error at every node and step: sum_k M_k = 6 base would then
// differ from W by a fixed factor, and with omega = 2 the moments would
// drift by 2 x 3e-8 per step in FP32.  The quotient is therefore corrected
// with its exact residual (one FMA each), which leaves an unbiased rounding.
template <int D, typename T>
__device__ __forceinline__ T div2d(T w)
{
    if constexpr (D == 3) {
        const T q = w * T(1.0 / 6.0);
        return fma(fma(T(-6), q, w), T(1.0 / 6.0), q);
    } else {
        return w * T(1.0 / (2.0 * D));
    }
}

// Maxwell flux Q(W, e_a) = (-e_a x H, e_a x E) of W = (E, H) (Sec. 6.1.1):
// with (a, j, k) a cyclic permutation of the axes, e_a x X = (X_j e_k - X_k e_j).
template <typename V>
__device__ __forceinline__ void maxwell_flux(const V* W, int a, V* Q, V zero)
{
    const int j = (a + 1) % 3, k = (a + 2) % 3;
    Q[a] = zero;
    Q[k] = -W[3 + j];
    Q[j] = W[3 + k];
    Q[3 + a] = zero;
    Q[3 + k] = W[j];
    Q[3 + j] = -W[k];
}

// Relaxation of one node of Maxwell's equations with a uniform conductivity
// (Sec. 2.3, Sec. 6.4): the Crank-Nicolson source step on the moments
// (W+ = (mu E, H)), then the non-equilibrium part relaxed about the new
// equilibrium, f <- M(W+) + (1 - omega) (f - M(W-)), on the six axis
// velocities stored as fk[(2a + s) * 6 + v] (s = 0 for +lambda e_a).
template <typename T>
__device__ __forceinline__ void maxwell_relax_node(T* fk, const T* W, T mu, T om1, T inv2l)
{
    constexpr int M = 6;
    T Wp[M];
#pragma unroll
    for (int v = 0; v < M; ++v) Wp[v] = v < 3 ? mu * W[v] : W[v];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        T Qm[M], Qp[M];
        maxwell_flux(W, a, Qm, T(0));
        maxwell_flux(Wp, a, Qp, T(0));
#pragma unroll
        for (int v = 0; v < M; ++v) {
            // Q^a has no component along E_a and H_a
            const bool z = v == a || v == 3 + a;
            const T bm = div2d<3>(W[v]), hm = z ? T(0) : Qm[v] * inv2l;
            const T bp = div2d<3>(Wp[v]), hp = z ? T(0) : Qp[v] * inv2l;
            T& fp = fk[(2 * a) * M + v];
            T& fm = fk[(2 * a + 1) * M + v];
            fp = fma(om1, fp - (z ? bm : bm + hm), z ? bp : bp + hp);
            fm = fma(om1, fm - (z ? bm : bm - hm), z ? bp : bp - hp);
        }
    }
}

// Relaxation at every node of the block (eq. over_relaxation) with the 2d
// velocity equilibria M_{a,+-} = W/(2d) +- Q^a(W)/(2 lambda).
template <int D, int P, int SYS, typename T>
__device__ __forceinline__ void relax_block(const Inst& I, T* s, int bcells)
{
    constexpr int NP = P + 1;
    constexpr int NN = ipow(NP, D);
    constexpr int M = nvars(D, SYS);
    constexpr int NV = 2 * D;
    constexpr int NPOP = NV * M;
    const int nnodes = bcells * NN;
    const int pstride = bcells * NN;
    const T omega = T(I.omega);
    const bool two = I.omega == 2.0;
    const T inv2l = T(1.0 / (2.0 * I.lambda));
    const T gm1 = T(I.gamma - 1.0);
    for (int nd = threadIdx.x; nd < nnodes; nd += blockDim.x) {
        T fk[NPOP];
#pragma unroll
        for (int pp = 0; pp < NPOP; ++pp) fk[pp] = s[pp * pstride + nd];
        T W[M];
#pragma unroll
        for (int v = 0; v < M; ++v) {
            Acc<T> acc;
#pragma unroll
            for (int k = 0; k < NV; ++k) acc.add(fk[k * M + v]);
            W[v] = acc.s;
        }
        if constexpr (SYS == kMaxwell) {
            maxwell_relax_node(fk, W, T(I.mu), T(1) - omega, inv2l);
#pragma unroll
            for (int pp = 0; pp < NPOP; ++pp) s[pp * pstride + nd] = fk[pp];
            continue;
        }
        T inv = 0, pr = 0;
        if (SYS == kEuler) {
            inv = T(1) / W[0];
            T ke = 0;
#pragma unroll
            for (int b = 0; b < D; ++b) ke = fma(W[1 + b], W[1 + b], ke);
            pr = gm1 * (W[1 + D] - T(0.5) * ke * inv);
        }
#pragma unroll
        for (int a = 0; a < D; ++a) {
            T Q[M];
            if (SYS == kAdvection) {
                Q[0] = T(I.adv[a]) * W[0];
            } else {
                const T ua = W[1 + a] * inv;
                Q[0] = W[1 + a];
#pragma unroll
                for (int b = 0; b < D; ++b) Q[1 + b] = W[1 + b] * ua + (b == a ? pr : T(0));
                Q[1 + D] = (W[1 + D] + pr) * ua;
            }
#pragma unroll
            for (int v = 0; v < M; ++v) {
                const T base = div2d<D>(W[v]);
                const T half = Q[v] * inv2l;
                T& fp = fk[(2 * a) * M + v];
                T& fm = fk[(2 * a + 1) * M + v];
                if (two) {
                    fp = fma(T(2), base + half, -fp);
                    fm = fma(T(2), base - half, -fm);
                } else {
                    fp = omega * (base + half) + (T(1) - omega) * fp;
                    fm = omega * (base - half) + (T(1) - omega) * fm;
                }
            }
        }
#pragma unroll
        for (int pp = 0; pp < NPOP; ++pp) s[pp * pstride + nd] = fk[pp];
    }
}

// Global offset of row 'row' of population 'pop' of this block.
template <int D, int NN>
__device__ __forceinline__ long long row_offset(const Inst& I, int pop, int row, int x0, int y0, int z0)
{
    int ly = 0, lz = 0;
    if (D == 2) ly = row;
    if (D == 3) {
        lz = (int)fdiv((unsigned)row, I.fd_B1);
        ly = row - lz * (int)I.fd_B1.d;
    }
    const long long cellrow = ((long long)(z0 + lz) * (D > 1 ? I.n[1] : 1) + (y0 + ly)) * I.n[0] + x0;
    return (long long)pop * I.nodes + cellrow * NN;
}

// Bulk loads of every row of tile t into s, completing on bar (warp 0 only).
template <int D, int P, int SYS, typename T>
__device__ __forceinline__ void issue_tile_load(const Inst& I, int t, T* s, uint64_t* bar)
{
    constexpr int NN = ipow(P + 1, D);
    constexpr int NPOP = 2 * D * (nvars(D, SYS));
    const int B0 = I.B[0], B1 = D > 1 ? I.B[1] : 1, B2 = D > 2 ? I.B[2] : 1;
    const int bcells = B0 * B1 * B2, rowlen = B0 * NN, nrows = B1 * B2, nchunks = NPOP * nrows;
    const TileXYZ c = tile_xyz(I, t);
    const int lane = threadIdx.x;
    const T* f = static_cast<const T*>(I.f);
    if (lane == 0)
        mbar_arrive_expect_tx(bar, (unsigned)(nchunks * rowlen * sizeof(T)) + (I.debug_stall ? 16u : 0u));
    __syncwarp();
    for (int ch = lane; ch < nchunks; ch += 32) {
        const int pop = (int)fdiv((unsigned)ch, I.fd_nrows);
        const int row = ch - pop * nrows;
        bulk_g2s(s + (pop * bcells + row * B0) * NN,
                 f + row_offset<D, NN>(I, pop, row, c.bx * B0, c.by * B1, c.bz * B2),
                 (unsigned)(rowlen * sizeof(T)), bar);
    }
}

// Bulk stores of every row of tile t from s (warp 0 only; one bulk group per lane).
template <int D, int P, int SYS, typename T>
__device__ __forceinline__ void issue_tile_store(const Inst& I, int t, const T* s)
{
    constexpr int NN = ipow(P + 1, D);
    constexpr int NPOP = 2 * D * (nvars(D, SYS));
    const int B0 = I.B[0], B1 = D > 1 ? I.B[1] : 1, B2 = D > 2 ? I.B[2] : 1;
    const int bcells = B0 * B1 * B2, rowlen = B0 * NN, nrows = B1 * B2, nchunks = NPOP * nrows;
    const TileXYZ c = tile_xyz(I, t);
    T* f = static_cast<T*>(I.f);
    for (int ch = threadIdx.x; ch < nchunks; ch += 32) {
        const int pop = (int)fdiv((unsigned)ch, I.fd_nrows);
        const int row = ch - pop * nrows;
        bulk_s2g(f + row_offset<D, NN>(I, pop, row, c.bx * B0, c.by * B1, c.bz * B2),
                 s + (pop * bcells + row * B0) * NN, (unsigned)(rowlen * sizeof(T)));
    }
    bulk_commit();
}

// Element-wise load / store of a tile (used when rows are not 16-byte aligned).
template <int D, int P, int SYS, typename T, bool LOAD>
__device__ __forceinline__ void copy_tile_generic(const Inst& I, int t, T* s)
{
    constexpr int NN = ipow(P + 1, D);
    constexpr int NPOP = 2 * D * (nvars(D, SYS));
    const int B0 = I.B[0], B1 = D > 1 ? I.B[1] : 1, B2 = D > 2 ? I.B[2] : 1;
    const int bcells = B0 * B1 * B2, rowlen = B0 * NN, nrows = B1 * B2;
    const int nload = NPOP * nrows * rowlen;
    const TileXYZ c = tile_xyz(I, t);
    T* f = static_cast<T*>(I.f);
    for (int idx = threadIdx.x; idx < nload; idx += blockDim.x) {
        const int ch = (int)fdiv((unsigned)idx, I.fd_rowlen);
        const int e = idx - ch * rowlen;
        const int pop = (int)fdiv((unsigned)ch, I.fd_nrows);
        const int row = ch - pop * nrows;
        const long long g = row_offset<D, NN>(I, pop, row, c.bx * B0, c.by * B1, c.bz * B2) + e;
        T& sv = s[(pop * bcells + row * B0) * NN + e];
        if (LOAD) sv = f[g];
        else f[g] = sv;
    }
}

// Phases 2-4 on a loaded tile; ends after the summaries (no trailing barrier).
template <int D, int P, int SYS, typename T>
__device__ __forceinline__ void compute_tile(const Inst& I, int t, T* s, const T* tin)
{
    const TileXYZ c = tile_xyz(I, t);
    const int bcells = I.B[0] * (D > 1 ? I.B[1] : 1) * (D > 2 ? I.B[2] : 1);
    if (I.mode == 0) {
        lines_all<D, P, SYS, T, false>(I, c.bx, c.by, c.bz, s, tin);   // 2. transport
        __syncthreads();
        relax_block<D, P, SYS, T>(I, s, bcells);                       // 3. relaxation
        __syncthreads();
    }
    lines_all<D, P, SYS, T, true>(I, c.bx, c.by, c.bz, s, tin);        // 4. summaries
}

template <int D, int P, int SYS, typename T>
__device__ __forceinline__ void chain_tile(const Inst& I, int t, T* tin)
{
    if (I.mode != 0) return;
    const TileXYZ c = tile_xyz(I, t);
    chain_all<D, P, SYS, T>(I, c.bx, c.by, c.bz, tin);
}

// Persistent step kernel: each thread block walks the tiles blockIdx.x,
// blockIdx.x + gridDim.x, ...  With bulk copies and two shared-memory stages
// the load of the next tile and the store of the previous one run while the
// current tile is computed.
template <int D, int P, int SYS, typename T>
__global__ void __launch_bounds__(kThreads) step_kernel(const __grid_constant__ Inst I)
{
    constexpr int NN = ipow(P + 1, D);
    constexpr int NPOP = 2 * D * (nvars(D, SYS));
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ int flag;
    const int bcells = I.B[0] * (D > 1 ? I.B[1] : 1) * (D > 2 ? I.B[2] : 1);
    T* buf0 = reinterpret_cast<T*>(smem_raw);
    T* buf1 = buf0 + NPOP * bcells * NN;
    T* tin = buf0 + I.stages * NPOP * bcells * NN;     // inflow traces of the current tile
    const int ntiles = I.nblk[0] * I.nblk[1] * I.nblk[2];
    const int tid = threadIdx.x;
    const bool warp0 = tid < 32;

    if (!I.tma) {
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
            chain_tile<D, P, SYS, T>(I, t, tin);
            copy_tile_generic<D, P, SYS, T, true>(I, t, buf0);
            __syncthreads();
            compute_tile<D, P, SYS, T>(I, t, buf0, tin);
            if (I.mode == 0) {
                __syncthreads();
                copy_tile_generic<D, P, SYS, T, false>(I, t, buf0);
            }
            __syncthreads();
        }
        return;
    }

    int t = blockIdx.x;
    if (t >= ntiles) return;
    const bool two = I.stages == 2;
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (warp0) issue_tile_load<D, P, SYS, T>(I, t, buf0, &bar[0]);

    for (int i = 0; t < ntiles; ++i, t += gridDim.x) {
        const int st = two ? (i & 1) : 0;
        T* cur = st ? buf1 : buf0;
        const int tn = t + gridDim.x;
        if (two && tn < ntiles && warp0) {
            bulk_wait_read();      // stores of the tile that last used the other stage have read it
            __syncwarp();
            issue_tile_load<D, P, SYS, T>(I, tn, st ? buf0 : buf1, &bar[st ^ 1]);
        }
        chain_tile<D, P, SYS, T>(I, t, tin);    // overlaps the bulk loads in flight
        const unsigned parity = two ? ((i >> 1) & 1) : (i & 1);
        if (tid == 0) flag = mbar_wait_bounded(&bar[st], parity, I.wait_cycles) ? 1 : 0;
        __syncthreads();
        if (flag == 0) {
            // give up: report the error, then wait once more (bounded) for the
            // bulk loads this block issued into its own shared memory -- the
            // stalled stage's and, with two stages, the next tile's: a bulk
            // copy cannot be cancelled, and the block's shared memory must
            // not be released while one may still write it -- and for the
            // block's bulk stores (bulk_wait_all); then leave.  A load that
            // has still not landed after the second bound is beyond repair
            // here; the error word makes the host poison the context.
            if (tid == 0) {
                if (I.err) atomicOr(I.err, kErrLoadTimeout);
                mbar_wait_bounded(&bar[st], parity, I.wait_cycles);
                if (two && tn < ntiles) mbar_wait_bounded(&bar[st ^ 1], ((i + 1) >> 1) & 1, I.wait_cycles);
            }
            if (warp0) bulk_wait_all();
            return;
        }
        (void)mbar_try_wait(&bar[st], parity);   // completed phase: acquire for every thread

        compute_tile<D, P, SYS, T>(I, t, cur, tin);

        if (I.mode == 0) {
            fence_proxy_async_smem();
            __syncthreads();
            if (warp0) issue_tile_store<D, P, SYS, T>(I, t, cur);
        } else {
            __syncthreads();
        }
        if (!two && tn < ntiles && warp0) {
            bulk_wait_read();
            __syncwarp();
            issue_tile_load<D, P, SYS, T>(I, tn, buf0, &bar[0]);
        }
    }
    if (warp0) bulk_wait_all();
}

}  // namespace kin
