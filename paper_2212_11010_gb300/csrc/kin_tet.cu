// kin_tet.cu -- the kinetic DG step on tetrahedral meshes (the paper's
// setting: Sec. 3.1 with tetrahedral cells, Sec. 3.2 downwind order, Sec. 5.1
// subdomain iteration).
//
// Basis: P1 Lagrange functions of each cell's four vertices, every integral
// exact: mass |L|/20 (1 + delta_ij); volume term (V . grad psi_i) |L|/4; face
// mass |F|/12 (1 + delta_ij) on the face's three vertices.  The implicit half
// step of Crank-Nicolson (tau = dt/2) of one cell reads
//   A f* = M f^n + tau sum_{inflow faces} |V.N| F f_R,
//   A = M + tau (-K + sum_{outflow faces} (V.N) F),
// and f^{n+1} = 2 f* - f^n.  Since A 1 = M 1 + tau sum_in |V.N| F 1 (the weak
// form of a constant), the kernels solve it in difference form about the
// cell's first node value r: f* - r 1 = A^{-1} [M (f^n - r 1) + tau sum_in
// |V.N| F (f_R - r 1)], exact for constant states whatever the rounding of
// A^{-1} (as on the Cartesian path).
//
// Downwind order (Sec. 3.2): for each velocity the host orients the faces,
// and inside every subdomain sorts the cells breadth-first into levels
// (cells of one level have no upwind neighbour in the same level).  A step
// is K launches of the sweep kernel -- one block per (subdomain, velocity),
// walking the levels with a barrier between them, every thread one (cell,
// variable) pair of the level -- and one pointwise launch for the
// Crank-Nicolson extrapolation and the relaxation.  Iteration p reads the
// neighbour's iterate p-1 across a subdomain interface (a face to another
// subdomain, or across the periodic boundary) and the current iterate
// inside (eq. ibvp); iterate 0 is f^n.
#include "kin_aux.h"
#include "kin_device.cuh"

#include <algorithm>
#include <type_traits>

namespace kin {

// ---------------------------------------------------------------------------
// FP64 setup: per (velocity, cell) the record
//   [0, 16)  A^{-1} (row-major)      [16]  |L| / 20
//   [17, 21) tau |V.N_a| |F_a| / 12 on inflow faces a, else 0
// ---------------------------------------------------------------------------

__global__ void tet_setup_kernel(TetSetupArgs A)
{
    const long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (id >= (long long)A.ncells * A.nvel) return;
    const int k = (int)(id / A.ncells);
    const int c = (int)(id - (long long)k * A.ncells);
    const double* x = A.xyz + (size_t)c * 12;
    const double V[3] = {A.vel[k][0], A.vel[k][1], A.vel[k][2]};
    double e[3][3];
    for (int b = 0; b < 3; ++b)
        for (int i = 0; i < 3; ++i) e[b][i] = x[3 * (b + 1) + i] - x[i];
    auto cross = [](const double* a, const double* b, double* r) {
        r[0] = a[1] * b[2] - a[2] * b[1];
        r[1] = a[2] * b[0] - a[0] * b[2];
        r[2] = a[0] * b[1] - a[1] * b[0];
    };
    double c12[3], c20[3], c01[3];
    cross(e[1], e[2], c12);
    cross(e[2], e[0], c20);
    cross(e[0], e[1], c01);
    const double det = e[0][0] * c12[0] + e[0][1] * c12[1] + e[0][2] * c12[2];
    const double vol = fabs(det) / 6.0;
    double grad[4][3];
    for (int i = 0; i < 3; ++i) {
        grad[1][i] = c12[i] / det;
        grad[2][i] = c20[i] / det;
        grad[3][i] = c01[i] / det;
        grad[0][i] = -(grad[1][i] + grad[2][i] + grad[3][i]);
    }
    double area[4];
    for (int a = 0; a < 4; ++a) {
        // |F_a| = 3 |L| |grad psi_a|: the face opposite vertex a
        const double g2 = grad[a][0] * grad[a][0] + grad[a][1] * grad[a][1] + grad[a][2] * grad[a][2];
        area[a] = 3.0 * vol * sqrt(g2);
    }
    const double tau = 0.5 * A.dt;
    double M[4][8];
    for (int i = 0; i < 4; ++i) {
        const double vg = V[0] * grad[i][0] + V[1] * grad[i][1] + V[2] * grad[i][2];
        for (int j = 0; j < 4; ++j) {
            M[i][j] = vol / 20.0 * (i == j ? 2.0 : 1.0) - tau * vg * vol / 4.0;
            M[i][4 + j] = i == j ? 1.0 : 0.0;
        }
    }
    const unsigned char ft = A.ftype[(size_t)k * A.ncells + c];
    double cin[4] = {0, 0, 0, 0};
    for (int a = 0; a < 4; ++a) {
        const int t = (ft >> (2 * a)) & 3;          // 1 inflow, 2 outflow, 0 parallel
        if (t == 0) continue;
        // V.N_a with N_a = -grad psi_a / |grad psi_a|
        const double gl = sqrt(grad[a][0] * grad[a][0] + grad[a][1] * grad[a][1] + grad[a][2] * grad[a][2]);
        const double vn = -(V[0] * grad[a][0] + V[1] * grad[a][1] + V[2] * grad[a][2]) / gl;
        if (t == 2) {
            for (int i = 0; i < 4; ++i)
                for (int j = 0; j < 4; ++j)
                    if (i != a && j != a) M[i][j] += tau * vn * area[a] / 12.0 * (i == j ? 2.0 : 1.0);
        } else {
            cin[a] = tau * fabs(vn) * area[a] / 12.0;
        }
    }
    // Gauss-Jordan inverse with partial pivoting
    for (int col = 0; col < 4; ++col) {
        int p = col;
        for (int r = col + 1; r < 4; ++r)
            if (fabs(M[r][col]) > fabs(M[p][col])) p = r;
        if (p != col)
            for (int j = 0; j < 8; ++j) {
                const double t = M[col][j];
                M[col][j] = M[p][j];
                M[p][j] = t;
            }
        const double d = 1.0 / M[col][col];
        for (int j = 0; j < 8; ++j) M[col][j] *= d;
        for (int r = 0; r < 4; ++r) {
            if (r == col) continue;
            const double l = M[r][col];
            for (int j = 0; j < 8; ++j) M[r][j] -= l * M[col][j];
        }
    }
    // records in the velocity's level order: a level reads consecutive records
    const size_t pos = (size_t)A.rank[(size_t)k * A.ncells + c];
    double* rec = A.c64 + ((size_t)k * A.ncells + pos) * kTetRec;
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) rec[i * 4 + j] = M[i][4 + j];
    rec[16] = vol / 20.0;
    for (int a = 0; a < 4; ++a) rec[17 + a] = cin[a];
    if (A.c32) {
        float* r32 = A.c32 + ((size_t)k * A.ncells + pos) * kTetRec;
        for (int q = 0; q < kTetRec; ++q) r32[q] = (float)rec[q];
    }
}

// ---------------------------------------------------------------------------
// sweep: one block per (subdomain, velocity), levels in order
// ---------------------------------------------------------------------------

// The four node values of a cell as one vector access (FP32: 16 bytes; the
// cell's nodes are contiguous and every population slab starts 16-byte
// aligned).
template <typename T>
__device__ __forceinline__ void load4(const T* p, T (&u)[4])
{
    if constexpr (sizeof(T) == 4) {
        const float4 q = *reinterpret_cast<const float4*>(p);
        u[0] = q.x;
        u[1] = q.y;
        u[2] = q.z;
        u[3] = q.w;
    } else {
        const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
        u[0] = a.x;
        u[1] = a.y;
        u[2] = b.x;
        u[3] = b.y;
    }
}

template <typename T>
__device__ __forceinline__ void store4(T* p, const T (&u)[4])
{
    if constexpr (sizeof(T) == 4) {
        *reinterpret_cast<float4*>(p) = make_float4(u[0], u[1], u[2], u[3]);
    } else {
        reinterpret_cast<double2*>(p)[0] = make_double2(u[0], u[1]);
        reinterpret_cast<double2*>(p)[1] = make_double2(u[2], u[3]);
    }
}

// Every thread takes one (cell, variable) pair of the level: the m threads
// of a cell read the same coefficient record (one broadcast), and a level of
// c cells offers c m independent solves.  The inflow faces are resolved
// ahead of time, per position of the velocity's level order, one word per
// face: the neighbour cell R << 7, the neighbour's local index of each of
// the face's three vertices (2 bits at bits 5, 3, 1), and bit 0 set when the
// face is a subdomain interface (the value comes from the previous iterate,
// else from the current one); -1 on the faces that are not inflow faces.
// A thread's first pair of a level has its cell and face references loaded
// during the level before,
// so a level waits for one round of loads (the cell's f^n and record and the
// neighbour values, issued together: the face types come from the
// references) rather than for a chain of dependent ones.
template <typename T>
__global__ void __launch_bounds__(kTetSweepThreads, 2) tet_sweep_kernel(TetArgs A, const T* __restrict__ prev, T* cur)
{
    const int s = blockIdx.x, k = blockIdx.y;
    const int* __restrict__ order = A.order + (size_t)k * A.ncells;
    const int* __restrict__ fref = A.fref + (size_t)k * A.ncells * 4;
    const int lb = A.lstart[k * (A.nsub + 1) + s], le = A.lstart[k * (A.nsub + 1) + s + 1];
    const T* __restrict__ coef = static_cast<const T*>(A.coef) + (size_t)k * A.ncells * kTetRec;
    const T* __restrict__ fn = static_cast<const T*>(A.f);
    const long long nodes = A.nodes;
    const int m = A.m;
    const int tid = threadIdx.x, nt = blockDim.x;

    auto solve = [&](int pos, int v, int c, const int4 nr) {
        const T* rec = coef + (size_t)pos * kTetRec;
        const long long pop = (long long)(k * m + v) * nodes;
        T u[4];
        load4(fn + pop + (size_t)c * 4, u);
        const T r = u[0];
        T du[4], sum = T(0);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            du[i] = u[i] - r;
            sum += du[i];
        }
        const T m20 = rec[16];
        T rhs[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) rhs[i] = m20 * (sum + du[i]);
        const int fw[4] = {nr.x, nr.y, nr.z, nr.w};
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            // (the face type comes from the references, already in registers,
            // so the neighbour loads need not wait for the record)
            const int wd = fw[a];
            if (wd < 0) continue;
            const T ca = rec[17 + a];
            const T* src = ((wd & 1) ? prev : cur) + pop + (size_t)(wd >> 7) * 4;
            // the neighbour's values at this cell's face vertices (j != a, ascending)
            T g[4] = {T(0), T(0), T(0), T(0)};
            T gs = T(0);
            int jj = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (j == a) continue;
                g[j] = src[(wd >> (5 - 2 * jj)) & 3] - r;
                gs += g[j];
                ++jj;
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (i != a) rhs[i] = fma(ca, gs + g[i], rhs[i]);
        }
        T x[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            T acc = rec[i * 4] * rhs[0];
#pragma unroll
            for (int j = 1; j < 4; ++j) acc = fma(rec[i * 4 + j], rhs[j], acc);
            x[i] = acc + r;
        }
        store4(cur + pop + (size_t)c * 4, x);
    };
    auto refs = [&](int pos) { return reinterpret_cast<const int4*>(fref)[pos]; };

    // this thread's first pair of the coming level: cell and face references
    int cn = 0;
    int4 nrn = make_int4(-1, -1, -1, -1);
    if (lb < le && tid < (A.bounds[lb + 1] - A.bounds[lb]) * m) {
        const int pos = A.bounds[lb] + tid / m;
        cn = order[pos];
        nrn = refs(pos);
    }
    for (int l = lb; l < le; ++l) {
        const int p0 = A.bounds[l], p1 = A.bounds[l + 1];
        const int items = (p1 - p0) * m;
        const int cc = cn;
        const int4 nrc = nrn;
        if (l + 1 < le && tid < (A.bounds[l + 2] - p1) * m) {
            const int pos = p1 + tid / m;
            cn = order[pos];
            nrn = refs(pos);
        }
        if (tid < items) solve(p0 + tid / m, tid % m, cc, nrc);
        for (int it = tid + nt; it < items; it += nt) {
            const int pos = p0 + it / m;
            solve(pos, it % m, order[pos], refs(pos));
        }
        __syncthreads();     // the next level reads this level's cells
    }
}

// ---------------------------------------------------------------------------
// equilibria and relaxation at the nodes
// ---------------------------------------------------------------------------

// Q^a(W) of the system (Euler, scalar advection or Maxwell).
template <int SYS, typename V>
__device__ __forceinline__ void tet_flux(const TetArgs& A, const V* W, int a, V* Q)
{
    if constexpr (SYS == kAdvection) {
        Q[0] = V(A.adv[a]) * W[0];
    } else if constexpr (SYS == kMaxwell) {
        maxwell_flux(W, a, Q, V(0));
    } else {
        V ke = V(0);
#pragma unroll
        for (int b = 0; b < 3; ++b) ke = fma(W[1 + b], W[1 + b], ke);
        const V inv = V(1) / W[0];
        const V pr = V(A.gamma - 1.0) * (W[4] - V(0.5) * ke * inv);
        const V ua = W[1 + a] * inv;
        Q[0] = W[1 + a];
#pragma unroll
        for (int b = 0; b < 3; ++b) Q[1 + b] = W[1 + b] * ua + (b == a ? pr : V(0));
        Q[4] = (W[4] + pr) * ua;
    }
}

// Equilibria of all populations: D3Q6 M_{a+-} = W/6 +- Q^a/(2 lambda);
// D3Q4 (cube diagonals V_k = lambda s_k, Sec. 6.1.3)
// M_k = W/4 + sum_a s_k^a Q^a / (4 lambda), which solves eq. maxwell_def.
template <int SYS, int VS, typename V>
__device__ __forceinline__ void tet_equilibria(const TetArgs& A, const V* W, V* M)
{
    constexpr int m = nvars(3, SYS);
    V Q[3][m];
#pragma unroll
    for (int a = 0; a < 3; ++a) tet_flux<SYS>(A, W, a, Q[a]);
    if constexpr (VS == 1) {
        constexpr int sg[4][3] = {{1, 1, 1}, {1, -1, -1}, {-1, 1, -1}, {-1, -1, 1}};
        const V il = V(1.0 / (4.0 * A.lambda));
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int v = 0; v < m; ++v) {
                V q = V(sg[k][0]) * Q[0][v];
                q = fma(V(sg[k][1]), Q[1][v], q);
                q = fma(V(sg[k][2]), Q[2][v], q);
                M[k * m + v] = fma(q, il, W[v] * V(0.25));
            }
    } else {
        const V il = V(1.0 / (2.0 * A.lambda));
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int v = 0; v < m; ++v) {
                const V base = div2d<3>(W[v]);
                M[(2 * a) * m + v] = base + Q[a][v] * il;
                M[(2 * a + 1) * m + v] = base - Q[a][v] * il;
            }
    }
}

// f^{n+1} = 2 f* - f^n, then W = sum_k f_k (Kahan in FP32) and the
// relaxation f <- omega M(W) + (1 - omega) f (eq. over_relaxation); Maxwell
// with conductivity relaxes about the equilibrium after the source step,
// f <- M(W+) + (1 - omega)(f - M(W-)).  Compiled per system and velocity
// set, so that every population stays in registers.
template <int SYS, int VS, typename T>
__global__ void __launch_bounds__(256) tet_relax_kernel(TetArgs A, const T* __restrict__ star)
{
    constexpr int m = nvars(3, SYS), NV = VS == 1 ? 4 : 6, NPOP = NV * m;
    T* f = static_cast<T*>(A.f);
    const long long nodes = A.nodes;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nodes;
         i += (long long)gridDim.x * blockDim.x) {
        T fk[NPOP];
#pragma unroll
        for (int p = 0; p < NPOP; ++p) fk[p] = fma(T(2), star[p * nodes + i], -f[p * nodes + i]);
        T W[m];
#pragma unroll
        for (int v = 0; v < m; ++v) {
            Acc<T> acc;
#pragma unroll
            for (int k = 0; k < NV; ++k) acc.add(fk[k * m + v]);
            W[v] = acc.s;
        }
        T Mm[NPOP];
        tet_equilibria<SYS, VS>(A, W, Mm);
        const T om = T(A.omega);
        if constexpr (SYS == kMaxwell) {
            T Wp[m], Mp[NPOP];
#pragma unroll
            for (int v = 0; v < m; ++v) Wp[v] = v < 3 ? T(A.mu) * W[v] : W[v];
            tet_equilibria<SYS, VS>(A, Wp, Mp);
#pragma unroll
            for (int p = 0; p < NPOP; ++p) f[p * nodes + i] = fma(T(1) - om, fk[p] - Mm[p], Mp[p]);
        } else {
            if (A.omega == 2.0) {
#pragma unroll
                for (int p = 0; p < NPOP; ++p) f[p * nodes + i] = fma(T(2), Mm[p], -fk[p]);
            } else {
#pragma unroll
                for (int p = 0; p < NPOP; ++p) f[p * nodes + i] = om * Mm[p] + (T(1) - om) * fk[p];
            }
        }
    }
}

// f = M(W) from the FP64 macroscopic state (Sec. 2.2 initialisation).
template <int SYS, int VS, typename T>
__global__ void tet_init_kernel(TetArgs A, const double* __restrict__ W0)
{
    constexpr int m = nvars(3, SYS), NPOP = (VS == 1 ? 4 : 6) * m;
    T* f = static_cast<T*>(A.f);
    const long long nodes = A.nodes;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nodes;
         i += (long long)gridDim.x * blockDim.x) {
        double W[m], M[NPOP];
#pragma unroll
        for (int v = 0; v < m; ++v) W[v] = W0[v * nodes + i];
        tet_equilibria<SYS, VS>(A, W, M);
#pragma unroll
        for (int p = 0; p < NPOP; ++p) f[p * nodes + i] = (T)M[p];
    }
}

// Launch a (system, velocity set, precision) instance of a pointwise kernel.
template <template <int, int, typename> class K, typename... Args>
static cudaError_t tet_dispatch(const TetArgs& a, int prec, unsigned grid, cudaStream_t st, Args... args)
{
    auto go = [&](auto sys, auto vs) {
        constexpr int S = decltype(sys)::value, V = decltype(vs)::value;
        if (prec == 1) K<S, V, float>::launch(a, grid, st, args...);
        else K<S, V, double>::launch(a, grid, st, args...);
    };
    using I0 = std::integral_constant<int, 0>;
    using I1 = std::integral_constant<int, 1>;
    using I2 = std::integral_constant<int, 2>;
    const bool d3q4 = a.velset == 1;
    switch (a.system) {
    case kAdvection: d3q4 ? go(I0{}, I1{}) : go(I0{}, I0{}); break;
    case kEuler: d3q4 ? go(I1{}, I1{}) : go(I1{}, I0{}); break;
    default: d3q4 ? go(I2{}, I1{}) : go(I2{}, I0{}); break;
    }
    return cudaGetLastError();
}

template <int S, int V, typename T>
struct RelaxLaunch {
    static void launch(const TetArgs& a, unsigned grid, cudaStream_t st, const void* star)
    {
        tet_relax_kernel<S, V, T><<<grid, 256, 0, st>>>(a, static_cast<const T*>(star));
    }
};

template <int S, int V, typename T>
struct InitLaunch {
    static void launch(const TetArgs& a, unsigned grid, cudaStream_t st, const double* W)
    {
        tet_init_kernel<S, V, T><<<grid, 256, 0, st>>>(a, W);
    }
};

cudaError_t tet_launch_setup(const TetSetupArgs& a, cudaStream_t st)
{
    const long long n = (long long)a.ncells * a.nvel;
    tet_setup_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t tet_launch_sweep(const TetArgs& a, const void* prev, void* cur, int prec, cudaStream_t st)
{
    const dim3 grid(a.nsub, a.nvel);
    if (prec == 1)
        tet_sweep_kernel<float><<<grid, kTetSweepThreads, 0, st>>>(a, static_cast<const float*>(prev),
                                                                  static_cast<float*>(cur));
    else
        tet_sweep_kernel<double><<<grid, kTetSweepThreads, 0, st>>>(a, static_cast<const double*>(prev),
                                                                   static_cast<double*>(cur));
    return cudaGetLastError();
}

cudaError_t tet_launch_relax(const TetArgs& a, const void* star, int prec, cudaStream_t st)
{
    const unsigned grid = (unsigned)std::min<long long>((a.nodes + 255) / 256, 152LL * 8);
    return tet_dispatch<RelaxLaunch>(a, prec, grid, st, star);
}

cudaError_t tet_launch_init(const TetArgs& a, const double* W, int prec, cudaStream_t st)
{
    const unsigned grid = (unsigned)std::min<long long>((a.nodes + 255) / 256, 152LL * 8);
    return tet_dispatch<InitLaunch>(a, prec, grid, st, W);
}

}  // namespace kin
