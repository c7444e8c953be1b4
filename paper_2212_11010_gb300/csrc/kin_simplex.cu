// kin_simplex.cu -- the paper's d + 1 velocity sets (D2Q3, Sec. 2.4; D3Q4,
// Sec. 6.1.3).  Their velocities are not aligned with the mesh: a cell has an
// inflow face on every axis with V_a != 0, the downwind order is a true
// anti-diagonal wavefront (Sec. 3.2), and subdomains meet at corners
// (Sec. 5.1, the three-iteration case).  The transport is done by the
// subdomain iteration of eq. ibvp as written:
//   trace pass   iterate 0: outflow faces of f^n on every subdomain boundary;
//   K sweeps     one thread block per (population, subdomain) holds the
//                subdomain in shared memory and visits its cells by wavefronts;
//                each cell solves its full local block (eq. dg_imp, CN half
//                step) with inflow from upwind faces inside the subdomain
//                (shared memory) or across the interface (previous iterate's
//                traces); the sweep writes this iterate's outflow traces and,
//                on the last iterate, f^{n+1} = 2 f* - f^n;
//   relaxation   W = sum_k f_k and f_k <- omega M_k(W) + (1 - omega) f_k with
//                M from the moment system eq. maxwell_def (its inverse is
//                precomputed in FP64).
#include "kin_aux.h"
#include "kin_device.cuh"

#include <math.h>

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

// One thread per velocity.  Record layout (sx_coef_stride elements):
//   [0, NN*NN)                 Pm = A^{-1} W_cell - I   (row-major)
//   [NN*NN + a*NN*TN, ...)     G_a = nu_a A^{-1} (e_in,a x W_perp)  (NN x TN)
// with A = W_cell + sum_a nu_a (S_a at axis a, W at the others),
// S_a = Q + e_0 e_0^T (V_a > 0) or -Q + e_p e_p^T (V_a < 0), nu_a = |V_a| dt / (2 h_a).
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
    int in_node[3];
    for (int a = 0; a < d; ++a) {
        nu[a] = fabs(V[a]) * 0.5 * A.dt / A.h[a];
        in_node[a] = V[a] > 0 ? 0 : p;
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
        for (int j = 0; j < nn; ++j) {
            int jj[3] = {j % np, (j / np) % np, j / (np * np)};
            double wj = 1.0;
            for (int b = 0; b < d; ++b) wj *= w[jj[b]];
            rec[i * nn + j] = Mx[i * w2 + nn + j] * wj - (i == j ? 1.0 : 0.0);
        }
    for (int a = 0; a < d; ++a) {
        double* G = rec + nn * nn + a * nn * tn;
        for (int i = 0; i < nn; ++i)
            for (int t = 0; t < tn; ++t) G[i * tn + t] = 0.0;
        if (V[a] == 0.0) continue;
        // inflow face of axis a: nodes with index in_node[a] along a; the
        // transverse node index t enumerates the other axes (lowest first)
        for (int j = 0; j < nn; ++j) {
            int jj[3] = {j % np, (j / np) % np, j / (np * np)};
            if (jj[a] != in_node[a]) continue;
            double wt = 1.0;
            int t = 0, mul = 1;
            for (int b = 0; b < d; ++b) {
                if (b == a) continue;
                wt *= w[jj[b]];
                t += jj[b] * mul;
                mul *= np;
            }
            for (int i = 0; i < nn; ++i) G[i * tn + t] += nu[a] * Mx[i * w2 + nn + j] * wt;
        }
    }
    if (A.c32)
        for (int e = 0; e < A.stride; ++e) A.c32[(size_t)k * A.stride + e] = (float)rec[e];
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

// One (population, subdomain) per thread block: wavefront sweep of iterate p.
template <int D, int P, typename T>
__global__ void __launch_bounds__(kSxThreads) sx_sweep_kernel(SxArgs S)
{
    constexpr int NP = P + 1;
    constexpr int NN = ipow(NP, D);
    constexpr int TN = ipow(NP, D - 1);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* tile = reinterpret_cast<T*>(smem_raw);             // L0 L1 L2 cells x NN
    T* cf = tile + (size_t)S.L[0] * S.L[1] * S.L[2] * NN;  // coefficients of this velocity
    const int nsub = S.NS[0] * S.NS[1] * S.NS[2];
    const int pop = blockIdx.x / nsub, sub = blockIdx.x % nsub;
    const int k = pop / S.m;
    const int s[3] = {sub % S.NS[0], (sub / S.NS[0]) % S.NS[1], sub / (S.NS[0] * S.NS[1])};
    const int L0 = S.L[0], L1 = S.L[1], L2 = S.L[2];
    const int org[3] = {s[0] * L0, s[1] * L1, s[2] * L2};
    T* f = static_cast<T*>(S.f);
    const long long fbase = (long long)pop * S.nodes;
    const int tid = threadIdx.x, nth = blockDim.x;

    // load the subdomain (rows of L0 cells are contiguous) and the coefficients
    const int rowlen = L0 * NN, nrows = L1 * L2;
    for (int idx = tid; idx < nrows * rowlen; idx += nth) {
        const int row = idx / rowlen, e = idx - (idx / rowlen) * rowlen;
        const int ly = row % L1, lz = row / L1;
        const long long g = fbase + (((long long)(org[2] + lz) * S.n[1] + (org[1] + ly)) * S.n[0] + org[0]) * NN + e;
        tile[idx] = f[g];
    }
    const T* crec = static_cast<const T*>(S.coef) + (size_t)k * S.coef_stride;
    for (int e = tid; e < S.coef_stride; e += nth) cf[e] = crec[e];
    __syncthreads();

    const int* sg = S.vsgn[k];
    // wavefront structure: the dependent axis is the last one with V_a != 0
    int dep = 0;
    for (int a = 0; a < D; ++a)
        if (sg[a] != 0) dep = a;
    int nwave = 1, ncand = 1;
    for (int a = 0; a < D; ++a) {
        if (sg[a] != 0) nwave += S.L[a] - 1;
        if (a != dep) ncand *= S.L[a];
    }
    for (int wv = 0; wv < nwave; ++wv) {
        for (int cand = tid; cand < ncand; cand += nth) {
            // oriented coordinates of the non-dependent axes, then the dependent one
            int o[3] = {0, 0, 0}, rem = cand, sumo = 0;
            for (int a = 0; a < D; ++a) {
                if (a == dep) continue;
                o[a] = rem % S.L[a];
                rem /= S.L[a];
                if (sg[a] != 0) sumo += o[a];
            }
            o[dep] = wv - sumo;
            if (o[dep] < 0 || o[dep] >= S.L[dep]) continue;
            int c[3] = {0, 0, 0};
            for (int a = 0; a < D; ++a) c[a] = sg[a] < 0 ? S.L[a] - 1 - o[a] : o[a];
            T* cell = tile + ((c[2] * L1 + c[1]) * L0 + c[0]) * NN;
            T u[NN], dl[NN];
#pragma unroll
            for (int i = 0; i < NN; ++i) u[i] = cell[i];
#pragma unroll
            for (int i = 0; i < NN; ++i) {
                T acc = 0;
#pragma unroll
                for (int j = 0; j < NN; ++j) acc = fma(cf[i * NN + j], u[j], acc);
                dl[i] = acc;
            }
            for (int a = 0; a < D; ++a) {
                if (sg[a] == 0) continue;
                const int in_node = sg[a] > 0 ? 0 : NP - 1;     // inflow face node along a
                const int up_node = sg[a] > 0 ? NP - 1 : 0;     // matching node of the upwind cell
                T t[TN];
                if (o[a] > 0) {
                    int cu[3] = {c[0], c[1], c[2]};
                    cu[a] -= sg[a];
                    const T* ucell = tile + ((cu[2] * L1 + cu[1]) * L0 + cu[0]) * NN;
#pragma unroll
                    for (int tt = 0; tt < TN; ++tt) {
                        // transverse node tt -> cell node with index up_node along a
                        int jn[3] = {0, 0, 0}, r2 = tt;
                        for (int b = 0; b < D; ++b) {
                            if (b == a) continue;
                            jn[b] = r2 % NP;
                            r2 /= NP;
                        }
                        jn[a] = up_node;
                        t[tt] = ucell[jn[0] + NP * jn[1] + NP * NP * jn[2]];
                    }
                } else {
                    // across the interface: the upwind subdomain's previous iterate
                    int sup = s[a] - sg[a];
                    if (sup < 0) sup += S.NS[a];
                    if (sup >= S.NS[a]) sup -= S.NS[a];
                    const T* tin = static_cast<const T*>(S.tr_in[a]) + (long long)pop * S.NS[a] * S.glines[a]
                        + (long long)sup * S.glines[a];
                    int cg[3] = {org[0] + c[0], org[1] + c[1], org[2] + c[2]};
#pragma unroll
                    for (int tt = 0; tt < TN; ++tt) {
                        int jn[3] = {0, 0, 0}, r2 = tt;
                        for (int b = 0; b < D; ++b) {
                            if (b == a) continue;
                            jn[b] = r2 % NP;
                            r2 /= NP;
                        }
                        t[tt] = tin[sx_gline(S, a, cg, jn, NP)];
                    }
                    (void)in_node;
                }
                const T* G = cf + NN * NN + a * NN * TN;
#pragma unroll
                for (int i = 0; i < NN; ++i)
#pragma unroll
                    for (int tt = 0; tt < TN; ++tt) dl[i] = fma(G[i * TN + tt], t[tt], dl[i]);
            }
#pragma unroll
            for (int i = 0; i < NN; ++i) cell[i] = u[i] + dl[i];      // f* replaces f^n
        }
        __syncthreads();
    }

    // outflow traces of this iterate on the subdomain's downwind faces
    for (int a = 0; a < D; ++a) {
        if (sg[a] == 0) continue;
        int ext[3] = {L0, L1, L2};
        ext[a] = 1;
        const int nface = ext[0] * ext[1] * ext[2] * TN;
        T* tout = static_cast<T*>(S.tr_out[a]) + (long long)pop * S.NS[a] * S.glines[a] + (long long)s[a] * S.glines[a];
        for (int e = tid; e < nface; e += nth) {
            const int tt = e % TN, fc = e / TN;
            int c[3] = {fc % ext[0], (fc / ext[0]) % ext[1], fc / (ext[0] * ext[1])};
            c[a] = sg[a] > 0 ? S.L[a] - 1 : 0;
            int jn[3] = {0, 0, 0}, r2 = tt;
            for (int b = 0; b < D; ++b) {
                if (b == a) continue;
                jn[b] = r2 % NP;
                r2 /= NP;
            }
            jn[a] = sg[a] > 0 ? NP - 1 : 0;
            const T v = tile[((c[2] * L1 + c[1]) * L0 + c[0]) * NN + jn[0] + NP * jn[1] + NP * NP * jn[2]];
            int cg[3] = {org[0] + c[0], org[1] + c[1], org[2] + c[2]};
            tout[sx_gline(S, a, cg, jn, NP)] = v;
        }
    }
    // last iterate: f^{n+1} = 2 f* - f^n, in place
    if (S.final_iter) {
        for (int idx = tid; idx < nrows * rowlen; idx += nth) {
            const int row = idx / rowlen, e = idx - (idx / rowlen) * rowlen;
            const int ly = row % L1, lz = row / L1;
            const long long g = fbase + (((long long)(org[2] + lz) * S.n[1] + (org[1] + ly)) * S.n[0] + org[0]) * NN + e;
            f[g] = T(2) * tile[idx] - f[g];
        }
    }
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

template <typename T>
static cudaError_t sweep_dispatch(const SxArgs& a, cudaStream_t st, size_t smem, int grid)
{
    const void* fn = nullptr;
    if (a.dim == 2) {
        if (a.degree == 1) fn = (const void*)sx_sweep_kernel<2, 1, T>;
        if (a.degree == 2) fn = (const void*)sx_sweep_kernel<2, 2, T>;
        if (a.degree == 3) fn = (const void*)sx_sweep_kernel<2, 3, T>;
    } else if (a.dim == 3) {
        if (a.degree == 1) fn = (const void*)sx_sweep_kernel<3, 1, T>;
        if (a.degree == 2) fn = (const void*)sx_sweep_kernel<3, 2, T>;
    }
    if (!fn) return cudaErrorInvalidValue;
    cudaError_t e = cudaSuccess;
    if (smem > 48 * 1024) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    SxArgs args = a;
    void* p[] = {&args};
    return cudaLaunchKernel(fn, dim3(grid), dim3(kSxThreads), p, smem, st);
}

cudaError_t sx_launch_sweep(const SxArgs& a, int prec, size_t smem, cudaStream_t st)
{
    const int grid = a.npop * a.NS[0] * a.NS[1] * a.NS[2];
    return prec == 1 ? sweep_dispatch<float>(a, st, smem, grid) : sweep_dispatch<double>(a, st, smem, grid);
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
