// kin_simplex.cu -- the paper's d + 1 velocity sets (D2Q3, Sec. 2.4; D3Q4,
// Sec. 6.1.3).  Their velocities are not aligned with the mesh: a cell has an
// inflow face on every axis with V_a != 0, the downwind order is a true
// anti-diagonal wavefront (Sec. 3.2), and subdomains meet at corners
// (Sec. 5.1, the three-iteration case).  The transport is done by the
// subdomain iteration of eq. ibvp as written, K sweeps per step:
//   sweep        one launch per iterate (per velocity when a velocity alone
//                fills the GPU): a thread block streams (variable, subdomain)
//                problems through the subdomain's columns, one cell per lane
//                and wave, lanes skewed so that every upwind neighbour is done
//                the wave before (sx_sweep_velocity); each cell solves its
//                full local block (eq. dg_imp, CN half step) with inflow from
//                its own previous cell, the neighbouring lane, or across the
//                interface (f^n on iterate 1, else the previous iterate's
//                traces); downwind boundary cells write this iterate's traces;
//                the last iterate writes f^{n+1} = 2 f* - f^n; with K = 1 a
//                trace pass first copies iterate 0;
//   relaxation   W = sum_k f_k and f_k <- omega M_k(W) + (1 - omega) f_k with
//                M from the moment system eq. maxwell_def (its inverse is
//                precomputed in FP64).
#include "kin_aux.h"
#include "kin_device.cuh"
#include "kin_tma.cuh"

#include <math.h>
#include <string.h>

namespace kin {

// ---------------------------------------------------------------------------
// FP64 preprocessing: velocity, block inverse and face operators per velocity
// ---------------------------------------------------------------------------

__device__ static void sx_velocity(int dim, int k, double lam, double V[3])
{
    V[0] = V[1] = V[2] = 0.0;
    if (dim == 2) {
        V[0] = lam * cos(2.0 * M_PI * k / 3.0);
        V[1] = lam * sin(2.0 * M_PI * k / 3.0);
    } else {
        const double s[4][3] = {{1, 1, 1}, {1, -1, -1}, {-1, 1, -1}, {-1, -1, 1}};
        for (int a = 0; a < 3; ++a) V[a] = lam * s[k][a];
    }
}

__device__ static void sx_gll(int p, double* xi, double* w)
{
    for (int j = 0; j <= p; ++j) {
        double x = -cos(M_PI * j / p);
        double Pv = 1.0;
        if (j > 0 && j < p) {
            for (int it = 0; it < 60; ++it) {
                double a = 1.0, b = x;
                for (int k = 1; k < p; ++k) {
                    double c = ((2 * k + 1) * x * b - k * a) / (k + 1);
                    a = b;
                    b = c;
                }
                double dP = p * (a - x * b) / (1.0 - x * x);
                double d2P = (2.0 * x * dP - p * (p + 1.0) * b) / (1.0 - x * x);
                double step = dP / d2P;
                x -= step;
                if (fabs(step) < 1e-17) break;
            }
            double a = 1.0, b = x;
            for (int k = 1; k < p; ++k) {
                double c = ((2 * k + 1) * x * b - k * a) / (k + 1);
                a = b;
                b = c;
            }
            Pv = b;
        } else {
            Pv = (j == 0 && (p % 2)) ? -1.0 : 1.0;
        }
        xi[j] = (j == 0) ? 0.0 : (j == p ? 1.0 : 0.5 * (x + 1.0));
        w[j] = 1.0 / (p * (p + 1.0) * Pv * Pv);
    }
}

// One thread per velocity.  Record layout (NN^2 + NN + d TN elements):
//   [0, NN*NN)                 A^{-1}   (row-major)
//   [NN*NN, NN*NN + NN)        W_cell   (tensor Gauss-Lobatto weights)
//   [NN*NN + NN + a*TN, ...)   nu_a W_perp on the inflow face of axis a (0 if V_a = 0)
// with A = W_cell + sum_a nu_a (S_a at axis a, W at the others),
// S_a = Q + e_0 e_0^T (V_a > 0) or -Q + e_p e_p^T (V_a < 0), nu_a = |V_a| dt / (2 h_a),
// so that the CN half step of eq. dg_imp is f* = A^{-1} (W_cell f^n + sum_a nu_a E_a W_perp tr_a),
// E_a the injection onto the inflow face nodes of axis a.
// Thread 0 also writes the inverse of the moment matrix [1...1; V_0 ... V_d].
__global__ void sx_setup_kernel(SxSetupArgs A)
{
    const int k = threadIdx.x;
    const int d = A.dim, p = A.degree, np = p + 1;
    int nn = 1, tn = 1;
    for (int a = 0; a < d; ++a) nn *= np;
    for (int a = 1; a < d; ++a) tn *= np;
    double xi[kMaxNP], w[kMaxNP];
    sx_gll(p, xi, w);
    if (k == 0) {
        // moment matrix and its inverse (Gauss-Jordan), nvel = d + 1
        const int nv = d + 1;
        double M[4][8];
        for (int j = 0; j < nv; ++j) {
            double V[3];
            sx_velocity(d, j, A.lambda, V);
            M[0][j] = 1.0;
            for (int a = 0; a < d; ++a) M[1 + a][j] = V[a];
        }
        for (int i = 0; i < nv; ++i)
            for (int j = 0; j < nv; ++j) M[i][nv + j] = (i == j) ? 1.0 : 0.0;
        for (int c = 0; c < nv; ++c) {
            int piv = c;
            for (int r = c + 1; r < nv; ++r)
                if (fabs(M[r][c]) > fabs(M[piv][c])) piv = r;
            for (int j = 0; j < 2 * nv; ++j) {
                double t = M[c][j];
                M[c][j] = M[piv][j];
                M[piv][j] = t;
            }
            const double inv = 1.0 / M[c][c];
            for (int j = 0; j < 2 * nv; ++j) M[c][j] *= inv;
            for (int r = 0; r < nv; ++r)
                if (r != c) {
                    const double l = M[r][c];
                    for (int j = 0; j < 2 * nv; ++j) M[r][j] -= l * M[c][j];
                }
        }
        for (int i = 0; i < nv; ++i)
            for (int j = 0; j < nv; ++j) A.minv[i * nv + j] = M[i][nv + j];
    }
    if (k > d) return;
    double V[3];
    sx_velocity(d, k, A.lambda, V);
    // 1D pieces
    double bw[kMaxNP], Dm[kMaxNP][kMaxNP];
    for (int i = 0; i < np; ++i) {
        double prod = 1.0;
        for (int j = 0; j < np; ++j)
            if (j != i) prod *= xi[i] - xi[j];
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
    double S[3][kMaxNP][kMaxNP], nu[3];
    for (int a = 0; a < d; ++a) {
        nu[a] = fabs(V[a]) * 0.5 * A.dt / A.h[a];
        for (int i = 0; i < np; ++i)
            for (int j = 0; j < np; ++j) {
                const double q = w[i] * Dm[i][j];
                double v = 0.0;
                if (V[a] > 0) v = q + ((i == 0 && j == 0) ? 1.0 : 0.0);
                else if (V[a] < 0) v = -q + ((i == p && j == p) ? 1.0 : 0.0);
                S[a][i][j] = v;
            }
    }
    // assemble A (nn x nn) and invert; node index = ix + np iy + np^2 iz
    double* Mx = A.work + (size_t)k * 2 * kSxMaxNN * kSxMaxNN;   // [nn][2nn]
    const int w2 = 2 * nn;
    for (int i = 0; i < nn; ++i) {
        int ii[3] = {i % np, (i / np) % np, i / (np * np)};
        for (int j = 0; j < nn; ++j) {
            int jj[3] = {j % np, (j / np) % np, j / (np * np)};
            bool diag = true;
            double wprod = 1.0;
            for (int b = 0; b < d; ++b) {
                if (ii[b] != jj[b]) diag = false;
                wprod *= w[ii[b]];
            }
            double v = diag ? wprod : 0.0;
            for (int a = 0; a < d; ++a) {
                bool same = true;
                double wt = 1.0;
                for (int b = 0; b < d; ++b) {
                    if (b == a) continue;
                    if (ii[b] != jj[b]) same = false;
                    wt *= w[ii[b]];
                }
                if (same) v += nu[a] * S[a][ii[a]][jj[a]] * wt;
            }
            Mx[i * w2 + j] = v;
            Mx[i * w2 + nn + j] = (i == j) ? 1.0 : 0.0;
        }
    }
    for (int c = 0; c < nn; ++c) {
        int piv = c;
        for (int r = c + 1; r < nn; ++r)
            if (fabs(Mx[r * w2 + c]) > fabs(Mx[piv * w2 + c])) piv = r;
        if (piv != c)
            for (int j = 0; j < w2; ++j) {
                const double t = Mx[c * w2 + j];
                Mx[c * w2 + j] = Mx[piv * w2 + j];
                Mx[piv * w2 + j] = t;
            }
        const double inv = 1.0 / Mx[c * w2 + c];
        for (int j = 0; j < w2; ++j) Mx[c * w2 + j] *= inv;
        for (int r = 0; r < nn; ++r) {
            if (r == c) continue;
            const double l = Mx[r * w2 + c];
            if (l != 0.0)
                for (int j = 0; j < w2; ++j) Mx[r * w2 + j] -= l * Mx[c * w2 + j];
        }
    }
    double* rec = A.c64 + (size_t)k * A.stride;
    for (int i = 0; i < nn; ++i)
        for (int j = 0; j < nn; ++j) rec[i * nn + j] = Mx[i * w2 + nn + j];
    for (int j = 0; j < nn; ++j) {
        int jj[3] = {j % np, (j / np) % np, j / (np * np)};
        double wj = 1.0;
        for (int b = 0; b < d; ++b) wj *= w[jj[b]];
        rec[nn * nn + j] = wj;
    }
    for (int a = 0; a < d; ++a)
        for (int t = 0; t < tn; ++t) {
            // transverse node t enumerates the other axes, lowest first
            double wt = 1.0;
            int r = t;
            for (int b = 0; b < d; ++b) {
                if (b == a) continue;
                wt *= w[r % np];
                r /= np;
            }
            rec[nn * nn + nn + a * tn + t] = V[a] == 0.0 ? 0.0 : nu[a] * wt;
        }
}

// ---------------------------------------------------------------------------
// trace pass and sweeps
// ---------------------------------------------------------------------------

// Global line id of the face node (transverse cell, transverse node) of axis a.
__device__ __forceinline__ long long sx_gline(const SxArgs& S, int a, const int c[3], const int j[3], int np)
{
    int t1 = -1, t2 = -1;
    for (int b = 0; b < S.dim; ++b) {
        if (b == a) continue;
        if (t1 < 0) t1 = b;
        else t2 = b;
    }
    long long gt = 0, tnode = 0;
    if (t2 >= 0) {
        gt = (long long)c[t2] * S.n[t1] + c[t1];
        tnode = j[t1] + np * j[t2];
    } else if (t1 >= 0) {
        gt = c[t1];
        tnode = j[t1];
    }
    long long tn = 1;
    for (int b = 1; b < S.dim; ++b) tn *= np;
    return gt * tn + tnode;
}

// Iterate 0 of eq. ibvp: the f^n values on the outflow face of every
// subdomain's downwind boundary, per (population, axis with V_a != 0).
template <typename T>
__global__ void sx_trace0_kernel(SxArgs S)
{
    const int np = S.degree + 1;
    const T* f = static_cast<const T*>(S.f);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < S.trace_total;
         e += (long long)gridDim.x * blockDim.x) {
        long long r = e;
        int pop = 0, a = 0;
        // entries: pop-major, then axis, then [NS_a][glines_a]
        for (;;) {
            const int k = pop / S.m;
            bool done = false;
            for (a = 0; a < S.dim; ++a) {
                if (S.vsgn[k][a] == 0) continue;
                const long long cnt = (long long)S.NS[a] * S.glines[a];
                if (r < cnt) {
                    done = true;
                    break;
                }
                r -= cnt;
            }
            if (done) break;
            ++pop;
        }
        const int k = pop / S.m, sg = S.vsgn[k][a];
        const int sa = (int)(r / S.glines[a]);
        const long long gl = r % S.glines[a];
        // decode gline -> transverse cell and node
        long long tn = 1;
        for (int b = 1; b < S.dim; ++b) tn *= np;
        const long long gt = gl / tn;
        const int tnode = (int)(gl % tn);
        int c[3] = {0, 0, 0}, j[3] = {0, 0, 0};
        int t1 = -1, t2 = -1;
        for (int b = 0; b < S.dim; ++b) {
            if (b == a) continue;
            if (t1 < 0) t1 = b;
            else t2 = b;
        }
        if (t2 >= 0) {
            c[t1] = (int)(gt % S.n[t1]);
            c[t2] = (int)(gt / S.n[t1]);
            j[t1] = tnode % np;
            j[t2] = tnode / np;
        } else if (t1 >= 0) {
            c[t1] = (int)gt;
            j[t1] = tnode;
        }
        c[a] = sa * S.L[a] + (sg > 0 ? S.L[a] - 1 : 0);
        j[a] = sg > 0 ? np - 1 : 0;
        const long long cell = ((long long)c[2] * S.n[1] + c[1]) * S.n[0] + c[0];
        const int node = j[0] + np * j[1] + np * np * j[2];
        T* out = static_cast<T*>(S.tr_out[a]);
        out[(long long)pop * S.NS[a] * S.glines[a] + r] = f[(long long)pop * S.nodes + cell * S.nn + node];
    }
}

// Sign of V_k along axis a for the d + 1 sets (D2Q3: 0, 120 and 240 degrees;
// D3Q4: the cube diagonals (1,1,1), (1,-1,-1), (-1,1,-1), (-1,-1,1)).
__host__ __device__ constexpr int sx_sign(int D, int k, int a)
{
    if (D == 2) {
        if (a == 0) return k == 0 ? 1 : -1;
        if (a == 1) return k == 0 ? 0 : (k == 1 ? 1 : -1);
        return 0;
    }
    if (a == 0) return k < 2 ? 1 : -1;
    if (a == 1) return (k == 0 || k == 2) ? 1 : -1;
    if (a == 2) return (k == 0 || k == 3) ? 1 : -1;
    return 0;
}

// Cell node with index ja along axis a and transverse node tt (the other
// axes, lowest first); node = j0 + NP j1 + NP^2 j2.
template <int D, int NP>
__host__ __device__ constexpr int sx_node(int a, int ja, int tt)
{
    int j[3] = {0, 0, 0};
    int r = tt;
    for (int b = 0; b < D; ++b) {
        if (b == a) continue;
        j[b] = r % NP;
        r /= NP;
    }
    j[a] = ja;
    return j[0] + NP * j[1] + NP * NP * j[2];
}

// Division by an invariant divisor d >= 1 for dividends below 2^31
// (Granlund and Montgomery, "Division by invariant integers using
// multiplication", 1994, the round-up multiplier): l = ceil(log2 d),
// m = floor(2^32 (2^l - d) / d) + 1, q = (mulhi(m, n) + n) >> l.
struct SxDiv {
    unsigned m;
    int l;
};

static inline SxDiv sx_div_make(int d)
{
    SxDiv r;
    int l = 0;
    while ((1LL << l) < d) ++l;
    r.l = l;
    r.m = (unsigned)((((1ULL << 32) * ((1ULL << l) - (unsigned long long)d)) / (unsigned long long)d) + 1);
    return r;
}

__device__ __forceinline__ int sx_div(int n, SxDiv d)
{
    return (int)(((unsigned long long)__umulhi(d.m, (unsigned)n) + (unsigned)n) >> d.l);
}

// Launch parameters of one sweep.  The block inverse, the cell weights and
// the face weights of every velocity travel in the parameter block, so the
// fully unrolled cell solve takes them as constant-bank operands.
template <int D, int P, typename T>
struct SxWave {
    static constexpr int NP = P + 1, NN = ipow(NP, D), TN = ipow(NP, D - 1), NV = D + 1;
    SxArgs S;
    int bpv;            // thread blocks per velocity
    int k0;             // first velocity of this launch
    SxDiv div_nsub, div_ns0, div_ns1;
    T ainv[NV][NN * NN];
    T wcell[NN];
    T face[NV][D][TN];
};

// Prefetch rings of the sweep, filled by cp.async kSxRing - 1 waves ahead:
// per lane and wave, the cell's f^n (NN values) and its interface inflow
// along the stepping axis (TN values); per wave and boundary lane of a
// transverse axis, that axis' interface inflow (TN values).  Each lane owns
// NEP contiguous elements per variable and slot (NEP = NN + TN rounded up so
// that NEP / CW is odd: lanes then fall in distinct banks for scalar (CW = 1)
// and 16-byte (CW > 1) accesses).  The exchange of outflow faces between
// lanes uses the same rule with TN.
__host__ __device__ constexpr int sx_pad_odd(int n, int cw)
{
    return ((n + cw - 1) / cw) % 2 ? (n + cw - 1) / cw * cw : ((n + cw - 1) / cw + 1) * cw;
}

template <int D, int P, typename T>
struct SxRing {
    static constexpr int NN = ipow(P + 1, D), TN = ipow(P + 1, D - 1);
    static constexpr int C = 16 / (int)sizeof(T);
    static constexpr int CW = (NN % C == 0 && TN % C == 0) ? C : 1;
    static constexpr int NEP = sx_pad_odd(NN + TN, CW);   // f^n of the cell + inflow along DEP
    static constexpr int TNP = sx_pad_odd(TN, CW);
};
constexpr int kSxRing = 2;            // slots; waves in flight = kSxRing - 1

// Position of one lane in the stream of problems: q counts the lane's cells
// (q = wave - skew), od is the oriented coordinate along the stepping axis.
struct SxTrack {
    int q, od, i, pop;
    int s[3], g[3];
    bool valid;
};

template <int NN, typename T>
__device__ __forceinline__ void sx_st(T* p, const T* u)
{
    if constexpr ((NN * sizeof(T)) % 16 == 0) {
        if constexpr (sizeof(T) == 4) {
#pragma unroll
            for (int k = 0; k < NN / 4; ++k)
                reinterpret_cast<float4*>(p)[k] = make_float4(u[4 * k], u[4 * k + 1], u[4 * k + 2], u[4 * k + 3]);
        } else {
#pragma unroll
            for (int k = 0; k < NN / 2; ++k) reinterpret_cast<double2*>(p)[k] = make_double2(u[2 * k], u[2 * k + 1]);
        }
    } else {
#pragma unroll
        for (int i = 0; i < NN; ++i) p[i] = u[i];
    }
}

// N values from / to shared memory, 16 bytes at a time when VEC (the address
// is then 16-byte aligned and N a multiple of 16 / sizeof(T)).
template <int N, bool VEC, typename T>
__device__ __forceinline__ void sx_lds(const T* p, T* v)
{
    if constexpr (VEC && sizeof(T) == 4) {
#pragma unroll
        for (int k = 0; k < N / 4; ++k) {
            const float4 q = reinterpret_cast<const float4*>(p)[k];
            v[4 * k] = q.x;
            v[4 * k + 1] = q.y;
            v[4 * k + 2] = q.z;
            v[4 * k + 3] = q.w;
        }
    } else if constexpr (VEC) {
#pragma unroll
        for (int k = 0; k < N / 2; ++k) {
            const double2 q = reinterpret_cast<const double2*>(p)[k];
            v[2 * k] = q.x;
            v[2 * k + 1] = q.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < N; ++i) v[i] = p[i];
    }
}

template <int N, bool VEC, typename T>
__device__ __forceinline__ void sx_sts(T* p, const T* v)
{
    if constexpr (VEC && sizeof(T) == 4) {
#pragma unroll
        for (int k = 0; k < N / 4; ++k)
            reinterpret_cast<float4*>(p)[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
    } else if constexpr (VEC) {
#pragma unroll
        for (int k = 0; k < N / 2; ++k) reinterpret_cast<double2*>(p)[k] = make_double2(v[2 * k], v[2 * k + 1]);
    } else {
#pragma unroll
        for (int i = 0; i < N; ++i) p[i] = v[i];
    }
}

// Transverse cell id of the face of axis a (the other axes, lowest first).
template <int D>
__device__ __forceinline__ int sx_face_cell(const SxArgs& S, int a, const int g[3])
{
    if (D == 2) return a == 0 ? g[1] : g[0];
    const int b1 = a == 0 ? 1 : 0, b2 = a == 2 ? 1 : 2;
    return g[b2] * S.n[b1] + g[b1];
}

template <int D, int KV>
__device__ __forceinline__ constexpr int sx_sg(int a)
{
    return a == 0 ? sx_sign(D, KV, 0) : (a == 1 ? sx_sign(D, KV, 1) : sx_sign(D, KV, 2));
}

// One velocity's part of a sweep (iterate it of eq. ibvp).  A thread block
// streams the problems (variable, subdomain) lb, lb + bpv, ... of velocity
// KV.  Its lanes are the subdomain's columns along the stepping axis DEP (the last axis with
// V_a != 0), indexed by the oriented transverse coordinates; lane o visits
// its column's cells one per wave, delayed by skew = sum of its oriented
// transverse coordinates, so that at every wave the cell of each lane has its
// upwind neighbours (Sec. 3.2) already done: along DEP the lane's own previous
// cell, along a transverse axis the previous wave of the neighbouring lane,
// which passes its outflow face through shared memory.  Consecutive
// problems follow each other in the column without a gap, so every lane is
// busy except during the first and last skew waves.  Cells on a subdomain's
// upwind boundary take their inflow from the previous iterate's traces (from
// f^n itself on iterate 1); cells on its downwind boundary write this
// iterate's traces.  The cell solve is the CN half step of eq. dg_imp in
// shifted form: with t = f^n at node 0,
//   f* = t + A^{-1} (W_cell (f^n - t) + sum_a nu_a E_a W_perp (tr_a - t)),
// which keeps constant states exactly.  The last iterate writes
// f^{n+1} = 2 f* - f^n in place.
template <int D, int P, int KV, typename T>
__device__ __forceinline__ void sx_sweep_velocity(const SxWave<D, P, T>& A, const int lb, T* xs, T* ring)
{
    constexpr int NP = P + 1, NN = ipow(NP, D), TN = ipow(NP, D - 1);
    using RG = SxRing<D, P, T>;
    constexpr int CW = RG::CW, NEP = RG::NEP, TNP = RG::TNP;
    constexpr int PF = kSxRing - 1;
    constexpr int DEP = D == 3 ? 2 : (KV == 0 ? 0 : 1);
    constexpr int TA0 = D == 3 ? 0 : 1 - DEP;
    constexpr int TA1 = D == 3 ? 1 : 0;          // only used when D == 3
    constexpr bool X0 = sx_sign(D, KV, TA0) != 0;
    constexpr bool X1 = D == 3 && sx_sign(D, KV, TA1) != 0;
    constexpr int SGD = sx_sign(D, KV, DEP);
    // node 0 receives face inflow iff some axis enters at index 0
    constexpr bool R0 = sx_sign(D, KV, 0) > 0 || sx_sign(D, KV, 1) > 0 || sx_sign(D, KV, 2) > 0;

    const SxArgs& S = A.S;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int n0 = S.L[TA0], n1 = D == 3 ? S.L[TA1] : 1;
    const int Ld = S.L[DEP];
    const bool active = tid < n0 * n1;
    const int ot1 = D == 3 ? tid / n0 : 0, ot0 = tid - ot1 * n0;
    const int lt0 = sx_sign(D, KV, TA0) < 0 ? n0 - 1 - ot0 : ot0;
    const int lt1 = (D == 3 && sx_sign(D, KV, TA1) < 0) ? n1 - 1 - ot1 : ot1;
    const int skew = (X0 ? ot0 : 0) + (X1 ? ot1 : 0);
    const int maxskew = (X0 ? n0 - 1 : 0) + (X1 ? n1 - 1 : 0);
    const int nsub = S.NS[0] * S.NS[1] * S.NS[2];
    const int nprob = S.m * nsub;                // (variable, subdomain)
    const int nb = lb < nprob ? (nprob - lb + A.bpv - 1) / A.bpv : 0;
    const int span = nb * Ld;
    const int total = nb > 0 ? span + maxskew : 0;
    T* f = static_cast<T*>(S.f);

    auto advance = [&](SxTrack& t) {
        ++t.q;
        t.valid = false;
        if (t.q < 0 || t.q >= span) return;
        bool fresh = false;
        if (t.q == 0) {
            t.od = 0;
            t.i = 0;
            fresh = true;
        } else if (++t.od == Ld) {
            t.od = 0;
            ++t.i;
            fresh = true;
        }
        if (fresh) {
            const int pid = lb + t.i * A.bpv;
            const int v = sx_div(pid, A.div_nsub), s = pid - v * nsub;
            const int s12 = sx_div(s, A.div_ns0), s2 = sx_div(s12, A.div_ns1);
            t.pop = KV * S.m + v;
            t.s[0] = s - s12 * S.NS[0];
            t.s[1] = s12 - s2 * S.NS[1];
            t.s[2] = s2;
            t.g[TA0] = t.s[TA0] * S.L[TA0] + lt0;
            if (D == 3) t.g[TA1] = t.s[TA1] * S.L[TA1] + lt1;
            else t.g[2] = 0;
        }
        t.g[DEP] = t.s[DEP] * Ld + (SGD < 0 ? Ld - 1 - t.od : t.od);
        t.valid = active;
    };

    // interface inflow is needed on the upwind boundary of the subdomain
    auto at_inflow = [&](const SxTrack& t, int a) {
        return a == DEP ? t.od == 0 : (a == TA0 ? ot0 == 0 : ot1 == 0);
    };
    auto at_outflow = [&](const SxTrack& t, int a) {
        return a == DEP ? t.od == Ld - 1 : (a == TA0 ? ot0 == n0 - 1 : ot1 == n1 - 1);
    };
    // this lane's elements in ring slot r
    auto slot = [&](int r) -> T* { return ring + (r * nt + tid) * NEP; };
    // transverse inflow of boundary lane b of axis ax in slot r
    T* tring = ring + kSxRing * nt * NEP;
    const int nbm = D == 2 ? 1 : (n0 > n1 ? n0 : n1);
    auto tslot = [&](int r, int ax, int b) -> T* { return tring + ((r * 2 + ax) * nbm + b) * TNP; };
    const int bidx0 = ot1, bidx1 = ot0;          // boundary index of this lane on TA0 / TA1
    // exchange [parity][axis][lane][TNP]
    auto xslot = [&](int par, int ax) -> T* { return xs + ((par * 2 + ax) * nt + tid) * TNP; };

    // issue the copies of the wave tracked by t into ring slot r
    auto fetch = [&](const SxTrack& t, int r) {
        if (t.valid) {
            T* dst = slot(r);
            const int cell = (t.g[2] * S.n[1] + t.g[1]) * S.n[0] + t.g[0];
            const T* src = f + (long long)t.pop * S.nodes + (long long)cell * NN;
            if constexpr (CW > 1) {
#pragma unroll
                for (int e = 0; e < NN; e += CW) cp16_g2s(dst + e, src + e);
            } else {
#pragma unroll
                for (int e = 0; e < NN; ++e) cp_small_g2s<sizeof(T)>(dst + e, src + e);
            }
#pragma unroll
            for (int a = 0; a < D; ++a) {
                const int sg = sx_sg<D, KV>(a);
                if (sg == 0 || !at_inflow(t, a)) continue;
                T* dbase = a == DEP ? dst + NN : tslot(r, a == TA0 ? 0 : 1, a == TA0 ? bidx0 : bidx1);
                if (S.from_f) {
                    // iterate 0 of eq. ibvp: f^n on the outflow face of the upwind cell
                    int gu[3] = {t.g[0], t.g[1], t.g[2]};
                    gu[a] -= sg;
                    if (gu[a] < 0) gu[a] += S.n[a];
                    if (gu[a] >= S.n[a]) gu[a] -= S.n[a];
                    const T* up = f + (long long)t.pop * S.nodes
                        + (long long)((gu[2] * S.n[1] + gu[1]) * S.n[0] + gu[0]) * NN;
                    const int out = sg > 0 ? P : 0;
#pragma unroll
                    for (int tt = 0; tt < TN; ++tt)
                        cp_small_g2s<sizeof(T)>(dbase + tt, up + sx_node<D, NP>(a, out, tt));
                } else {
                    int sup = t.s[a] - sg;
                    if (sup < 0) sup += S.NS[a];
                    if (sup >= S.NS[a]) sup -= S.NS[a];
                    const T* tr = static_cast<const T*>(S.tr_in[a]) + ((long long)t.pop * S.NS[a] + sup) * S.glines[a]
                        + (long long)sx_face_cell<D>(S, a, t.g) * TN;
                    if constexpr (CW > 1) {
#pragma unroll
                        for (int tt = 0; tt < TN; tt += CW) cp16_g2s(dbase + tt, tr + tt);
                    } else {
#pragma unroll
                        for (int tt = 0; tt < TN; ++tt) cp_small_g2s<sizeof(T)>(dbase + tt, tr + tt);
                    }
                }
            }
        }
        cp_commit();
    };

    T pd[TN];                                   // own outflow face along DEP (previous wave)
#pragma unroll
    for (int tt = 0; tt < TN; ++tt) pd[tt] = T(0);

    auto compute = [&](int W, const SxTrack& t, int rs) {
        if (!t.valid) return;
        const int par = W & 1;
        const T* sl = slot(rs);
        // where each axis' inflow comes from: the interface (ring), the own
        // previous cell (registers) or the upwind lane (exchange)
        const T* isrc[3] = {nullptr, nullptr, nullptr};
        bool fromreg[3] = {false, false, false};
#pragma unroll
        for (int a = 0; a < D; ++a) {
            const int sg = sx_sg<D, KV>(a);
            if (sg == 0) continue;
            if (a == DEP) {
                if (at_inflow(t, a)) isrc[a] = sl + NN;
                else fromreg[a] = true;
            } else {
                const int ax = a == TA0 ? 0 : 1;
                isrc[a] = at_inflow(t, a) ? tslot(rs, ax, ax == 0 ? bidx0 : bidx1)
                                          : xslot(par ^ 1, ax) - (a == TA0 ? 1 : n0) * TNP;
            }
        }
        T u[NN];
        sx_lds<NN, (CW > 1)>(sl, u);
        const T tref = u[0];
        T r[NN];
        r[0] = T(0);
#pragma unroll
        for (int j = 1; j < NN; ++j) r[j] = A.wcell[j] * (u[j] - tref);
#pragma unroll
        for (int a = 0; a < D; ++a) {
            const int sg = sx_sg<D, KV>(a);
            if (sg == 0) continue;
            const int in = sg > 0 ? 0 : P;
            T tv[TN];
            if (a == DEP && fromreg[a]) {
#pragma unroll
                for (int tt = 0; tt < TN; ++tt) tv[tt] = pd[tt];
            } else {
                sx_lds<TN, (CW > 1)>(isrc[a], tv);
            }
#pragma unroll
            for (int tt = 0; tt < TN; ++tt) {
                const int j = sx_node<D, NP>(a, in, tt);
                r[j] = fma(A.face[KV][a][tt], tv[tt] - tref, r[j]);
            }
        }
        // x = A^{-1} r by columns: each step is NN independent FMAs
        T x[NN];
#pragma unroll
        for (int i = 0; i < NN; ++i) x[i] = R0 ? A.ainv[KV][i * NN] * r[0] : A.ainv[KV][i * NN + 1] * r[1];
#pragma unroll
        for (int j = R0 ? 1 : 2; j < NN; ++j)
#pragma unroll
            for (int i = 0; i < NN; ++i) x[i] = fma(A.ainv[KV][i * NN + j], r[j], x[i]);
#pragma unroll
        for (int i = 0; i < NN; ++i) x[i] += tref;
        // outflow faces: transverse ones to the next lanes, DEP kept here
#pragma unroll
        for (int a = 0; a < D; ++a) {
            const int sg = sx_sg<D, KV>(a);
            if (sg == 0) continue;
            const int out = sg > 0 ? P : 0;
            T o[TN];
#pragma unroll
            for (int tt = 0; tt < TN; ++tt) o[tt] = x[sx_node<D, NP>(a, out, tt)];
            if (a == DEP) {
#pragma unroll
                for (int tt = 0; tt < TN; ++tt) pd[tt] = o[tt];
            } else {
                sx_sts<TN, (CW > 1)>(xslot(par, a == TA0 ? 0 : 1), o);
            }
            if (!S.final_iter && at_outflow(t, a)) {
                T* tr = static_cast<T*>(S.tr_out[a]) + ((long long)t.pop * S.NS[a] + t.s[a]) * S.glines[a]
                    + (long long)sx_face_cell<D>(S, a, t.g) * TN;
                sx_st<TN>(tr, o);
            }
        }
        if (S.final_iter) {
            const int cell = (t.g[2] * S.n[1] + t.g[1]) * S.n[0] + t.g[0];
#pragma unroll
            for (int i = 0; i < NN; ++i) x[i] = fma(T(2), x[i], -u[i]);
            sx_st<NN>(f + (long long)t.pop * S.nodes + (long long)cell * NN, x);
        }
    };

    SxTrack tp, tc;
    tp.q = tc.q = -skew - 1;
    tp.od = tc.od = tp.i = tc.i = tp.pop = tc.pop = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) tp.s[a] = tc.s[a] = tp.g[a] = tc.g[a] = 0;
    tp.valid = tc.valid = false;
    for (int k = 0; k < PF; ++k) {
        advance(tp);
        fetch(tp, k);
    }
    for (int W = 0; W < total; ++W) {
        // with one wave in flight the prefetch position of the last wave is
        // this wave's: copy it rather than advance a second tracker
        if constexpr (PF == 1) tc = tp;
        advance(tp);
        fetch(tp, (W + PF) % kSxRing);             // wave W + PF
        cp_wait_group<PF>();                        // wave W has landed
        if constexpr (PF != 1) advance(tc);
        compute(W, tc, W % kSxRing);
        __syncthreads();
    }
    cp_wait_group<0>();
}

// One sweep over every population: blockIdx.x / bpv + k0 is the velocity.
// MAXT bounds the block size (the subdomain's columns), which bounds
// registers.
template <int D, int P, typename T, int MAXT>
__global__ void __launch_bounds__(MAXT) sx_wave_kernel(const __grid_constant__ SxWave<D, P, T> A)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T* xs = reinterpret_cast<T*>(smem_raw);
    const int k = A.k0 + (int)blockIdx.x / A.bpv, lb = (int)blockIdx.x % A.bpv;
    T* ring = xs + 4 * SxRing<D, P, T>::TNP * blockDim.x;
    if (k == 0) sx_sweep_velocity<D, P, 0, T>(A, lb, xs, ring);
    else if (k == 1) sx_sweep_velocity<D, P, 1, T>(A, lb, xs, ring);
    else if (k == 2) sx_sweep_velocity<D, P, 2, T>(A, lb, xs, ring);
    else if (D == 3) sx_sweep_velocity<D, P, 3, T>(A, lb, xs, ring);
}

// Relaxation with the d + 1 velocity equilibria: M_{k,v} = sum_j Minv[k][j] rhs_j,
// rhs = (W_v, Q^1_v, ..., Q^d_v) (eq. maxwell_def).
template <int D, int SYS, typename T>
__global__ void sx_relax_kernel(SxArgs S)
{
    constexpr int M = nvars(D, SYS);
    constexpr int NV = D + 1;
    T* f = static_cast<T*>(S.f);
    const T omega = T(S.omega);
    const T gm1 = T(S.gamma - 1.0);
    T minv[NV][NV];
#pragma unroll
    for (int i = 0; i < NV; ++i)
#pragma unroll
        for (int j = 0; j < NV; ++j) minv[i][j] = T(S.minv[i * NV + j]);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < S.nodes;
         i += (long long)gridDim.x * blockDim.x) {
        T fk[NV * M];
#pragma unroll
        for (int p = 0; p < NV * M; ++p) fk[p] = f[(long long)p * S.nodes + i];
        T W[M];
#pragma unroll
        for (int v = 0; v < M; ++v) {
            Acc<T> acc;
#pragma unroll
            for (int kk = 0; kk < NV; ++kk) acc.add(fk[kk * M + v]);
            W[v] = acc.s;
        }
        T Q[D][M];
        if (SYS == kAdvection) {
#pragma unroll
            for (int a = 0; a < D; ++a) Q[a][0] = T(S.adv[a]) * W[0];
        } else {
            const T inv = T(1) / W[0];
            T ke = 0;
#pragma unroll
            for (int b = 0; b < D; ++b) ke = fma(W[1 + b], W[1 + b], ke);
            const T pr = gm1 * (W[1 + D] - T(0.5) * ke * inv);
#pragma unroll
            for (int a = 0; a < D; ++a) {
                const T ua = W[1 + a] * inv;
                Q[a][0] = W[1 + a];
#pragma unroll
                for (int b = 0; b < D; ++b) Q[a][1 + b] = W[1 + b] * ua + (b == a ? pr : T(0));
                Q[a][1 + D] = (W[1 + D] + pr) * ua;
            }
        }
#pragma unroll
        for (int kk = 0; kk < NV; ++kk)
#pragma unroll
            for (int v = 0; v < M; ++v) {
                T mk = minv[kk][0] * W[v];
#pragma unroll
                for (int a = 0; a < D; ++a) mk = fma(minv[kk][1 + a], Q[a][v], mk);
                T& fv = fk[kk * M + v];
                fv = (S.omega == 2.0) ? fma(T(2), mk, -fv) : omega * mk + (T(1) - omega) * fv;
            }
#pragma unroll
        for (int p = 0; p < NV * M; ++p) f[(long long)p * S.nodes + i] = fk[p];
    }
}

// f = M(W) for the d + 1 sets (initialisation), FP64 in.
template <int D, int SYS, typename T>
__global__ void sx_init_kernel(SxArgs S, const double* __restrict__ Wd)
{
    constexpr int M = nvars(D, SYS);
    constexpr int NV = D + 1;
    T* f = static_cast<T*>(S.f);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < S.nodes;
         i += (long long)gridDim.x * blockDim.x) {
        double W[M], Q[D][M];
        for (int v = 0; v < M; ++v) W[v] = Wd[(long long)v * S.nodes + i];
        if (SYS == kAdvection) {
            for (int a = 0; a < D; ++a) Q[a][0] = S.adv[a] * W[0];
        } else {
            double ke = 0.0;
            for (int b = 0; b < D; ++b) ke += W[1 + b] * W[1 + b];
            const double pr = (S.gamma - 1.0) * (W[1 + D] - 0.5 * ke / W[0]);
            for (int a = 0; a < D; ++a) {
                const double ua = W[1 + a] / W[0];
                Q[a][0] = W[1 + a];
                for (int b = 0; b < D; ++b) Q[a][1 + b] = W[1 + b] * ua + (b == a ? pr : 0.0);
                Q[a][1 + D] = (W[1 + D] + pr) * ua;
            }
        }
        for (int kk = 0; kk < NV; ++kk)
            for (int v = 0; v < M; ++v) {
                double mk = S.minv[kk * NV] * W[v];
                for (int a = 0; a < D; ++a) mk += S.minv[kk * NV + 1 + a] * Q[a][v];
                f[(long long)(kk * M + v) * S.nodes + i] = (T)mk;
            }
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

cudaError_t sx_launch_setup(const SxSetupArgs& a, cudaStream_t st)
{
    sx_setup_kernel<<<1, 32, 0, st>>>(a);
    return cudaGetLastError();
}

static int sx_grid(long long n)
{
    long long g = (n + 255) / 256;
    if (g > 152 * 8) g = 152 * 8;
    return (int)(g < 1 ? 1 : g);
}

constexpr int kSxNarrow = 256;     // block sizes up to this use the register-rich instance

template <int D, int P, typename T>
static const void* wave_fn(int nt)
{
    return nt <= kSxNarrow ? (const void*)sx_wave_kernel<D, P, T, kSxNarrow> : (const void*)sx_wave_kernel<D, P, T, 1024>;
}

template <typename T>
static const void* wave_pick(int dim, int degree, int nt)
{
    if (dim == 2) {
        if (degree == 1) return wave_fn<2, 1, T>(nt);
        if (degree == 2) return wave_fn<2, 2, T>(nt);
        if (degree == 3) return wave_fn<2, 3, T>(nt);
    } else if (dim == 3) {
        if (degree == 1) return wave_fn<3, 1, T>(nt);
        if (degree == 2) return wave_fn<3, 2, T>(nt);
    }
    return nullptr;
}

static int sx_lanes(const SxArgs& a)
{
    if (a.dim == 2) return a.L[0] > a.L[1] ? a.L[0] : a.L[1];
    return a.L[0] * a.L[1];
}

// boundary lanes per transverse axis, at most (the larger transverse extent
// over the velocities' lane layouts)
static int sx_boundary_lanes(const SxArgs& a)
{
    if (a.dim == 2) return 1;
    return a.L[0] > a.L[1] ? a.L[0] : a.L[1];
}

template <int D, int P, typename T>
static size_t wave_smem_of(int nt, int nbm)
{
    using RG = SxRing<D, P, T>;
    // exchange [2 parities][2 axes][nt][TNP] + ring [kSxRing][nt][NEP]
    // + transverse inflow [kSxRing][2 axes][nbm][TNP]
    return (((size_t)4 * RG::TNP + (size_t)kSxRing * RG::NEP) * nt + (size_t)kSxRing * 2 * nbm * RG::TNP) * sizeof(T);
}

template <typename T>
static size_t wave_smem(int dim, int degree, int nt, int nbm)
{
    if (dim == 2) {
        if (degree == 1) return wave_smem_of<2, 1, T>(nt, nbm);
        if (degree == 2) return wave_smem_of<2, 2, T>(nt, nbm);
        if (degree == 3) return wave_smem_of<2, 3, T>(nt, nbm);
    } else if (dim == 3) {
        if (degree == 1) return wave_smem_of<3, 1, T>(nt, nbm);
        if (degree == 2) return wave_smem_of<3, 2, T>(nt, nbm);
    }
    return 0;
}

int sx_sweep_shape(const SxArgs& a, int prec, SxPlan* plan)
{
    const int nt = (sx_lanes(a) + 31) / 32 * 32;
    const void* fn = prec == 1 ? wave_pick<float>(a.dim, a.degree, nt) : wave_pick<double>(a.dim, a.degree, nt);
    const int nbm = sx_boundary_lanes(a);
    const size_t sm = prec == 1 ? wave_smem<float>(a.dim, a.degree, nt, nbm) : wave_smem<double>(a.dim, a.degree, nt, nbm);
    if (!fn || nt > 1024 || sm > 227 * 1024) return 0;
    plan->threads = nt;
    plan->smem = sm;
    return 1;
}

cudaError_t sx_sweep_plan(const SxArgs& a, int prec, SxPlan* plan)
{
    if (!sx_sweep_shape(a, prec, plan)) return cudaErrorInvalidValue;
    const void* fn = prec == 1 ? wave_pick<float>(a.dim, a.degree, plan->threads)
                               : wave_pick<double>(a.dim, a.degree, plan->threads);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plan->smem);
    if (e != cudaSuccess) return e;
    int occ = 0, dev = 0, nsm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, plan->threads, plan->smem);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    // one resident wave of blocks, each streaming ceil(problems / blocks)
    // problems.  When one velocity's problems alone fill that wave, the
    // velocities go in separate launches (an SM then runs one velocity's
    // code at a time); otherwise one launch takes them all.
    const int nprob = a.m * a.NS[0] * a.NS[1] * a.NS[2];
    const int slots = occ * nsm;
    plan->split = nprob >= slots;
    int b = plan->split ? slots : slots / a.nvel;
    if (b < 1) b = 1;
    if (b > nprob) b = nprob;
    const int per = (nprob + b - 1) / b;
    plan->bpv = (nprob + per - 1) / per;
    plan->occupancy = occ;
    return cudaSuccess;
}

template <int D, int P, typename T>
static cudaError_t wave_launch(const SxArgs& a, const double* hrec, int rstride, const SxPlan& plan,
                               cudaStream_t st)
{
    using WA = SxWave<D, P, T>;
    static_assert(sizeof(WA) <= 32000, "sweep parameters exceed the kernel parameter limit");
    constexpr int NN = WA::NN, TN = WA::TN, NV = WA::NV;
    WA w;
    memset(&w, 0, sizeof w);
    w.S = a;
    w.bpv = plan.bpv;
    w.k0 = 0;
    w.div_nsub = sx_div_make(a.NS[0] * a.NS[1] * a.NS[2]);
    w.div_ns0 = sx_div_make(a.NS[0]);
    w.div_ns1 = sx_div_make(a.NS[1]);
    for (int k = 0; k < NV; ++k) {
        const double* rec = hrec + (size_t)k * rstride;
        for (int e = 0; e < NN * NN; ++e) w.ainv[k][e] = (T)rec[e];
        for (int ax = 0; ax < D; ++ax)
            for (int t = 0; t < TN; ++t) w.face[k][ax][t] = (T)rec[NN * NN + NN + ax * TN + t];
    }
    for (int j = 0; j < NN; ++j) w.wcell[j] = (T)hrec[NN * NN + j];
    const void* fn = wave_fn<D, P, T>(plan.threads);
    void* p[] = {&w};
    if (!plan.split)
        return cudaLaunchKernel(fn, dim3(a.nvel * plan.bpv), dim3(plan.threads), p, plan.smem, st);
    for (int k = 0; k < a.nvel; ++k) {
        w.k0 = k;
        const cudaError_t e = cudaLaunchKernel(fn, dim3(plan.bpv), dim3(plan.threads), p, plan.smem, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <typename T>
static cudaError_t wave_dispatch(const SxArgs& a, const double* hrec, int rstride, const SxPlan& plan,
                                 cudaStream_t st)
{
    if (a.dim == 2) {
        if (a.degree == 1) return wave_launch<2, 1, T>(a, hrec, rstride, plan, st);
        if (a.degree == 2) return wave_launch<2, 2, T>(a, hrec, rstride, plan, st);
        if (a.degree == 3) return wave_launch<2, 3, T>(a, hrec, rstride, plan, st);
    } else if (a.dim == 3) {
        if (a.degree == 1) return wave_launch<3, 1, T>(a, hrec, rstride, plan, st);
        if (a.degree == 2) return wave_launch<3, 2, T>(a, hrec, rstride, plan, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t sx_launch_sweep(const SxArgs& a, int prec, const double* hrec, int rstride, const SxPlan& plan,
                            cudaStream_t st)
{
    return prec == 1 ? wave_dispatch<float>(a, hrec, rstride, plan, st)
                     : wave_dispatch<double>(a, hrec, rstride, plan, st);
}

cudaError_t sx_launch_trace0(const SxArgs& a, int prec, cudaStream_t st)
{
    const int g = sx_grid(a.trace_total);
    if (prec == 1) sx_trace0_kernel<float><<<g, 256, 0, st>>>(a);
    else sx_trace0_kernel<double><<<g, 256, 0, st>>>(a);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t relax_dispatch(const SxArgs& a, cudaStream_t st, bool init, const double* W)
{
    const int g = sx_grid(a.nodes);
#define KIN_SX(DD, SY)                                                                     \
    if (a.dim == DD && a.system == SY) {                                                   \
        if (init) sx_init_kernel<DD, SY, T><<<g, 256, 0, st>>>(a, W);                      \
        else sx_relax_kernel<DD, SY, T><<<g, 256, 0, st>>>(a);                             \
        return cudaGetLastError();                                                         \
    }
    KIN_SX(2, kAdvection)
    KIN_SX(2, kEuler)
    KIN_SX(3, kAdvection)
    KIN_SX(3, kEuler)
#undef KIN_SX
    return cudaErrorInvalidValue;
}

cudaError_t sx_launch_relax(const SxArgs& a, int prec, cudaStream_t st)
{
    return prec == 1 ? relax_dispatch<float>(a, st, false, nullptr) : relax_dispatch<double>(a, st, false, nullptr);
}

cudaError_t sx_launch_init(const SxArgs& a, const double* W, int prec, cudaStream_t st)
{
    return prec == 1 ? relax_dispatch<float>(a, st, true, W) : relax_dispatch<double>(a, st, true, W);
}

}  // namespace kin
