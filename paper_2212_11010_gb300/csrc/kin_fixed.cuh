// kin_fixed.cuh -- the fused step kernel for a compile-time cell-block shape.
//
// Same computation as the generic kernel of kin_device.cuh (look-back
// inflow, tile load, downwind sweeps, relaxation, tile store, block
// summaries), specialised on the block extents B0 x B1 x B2 and the thread
// count NTH so that every loop has a constant trip count and every
// shared-memory offset is an immediate.  Differences in the schedule:
//   * the look-back runs first, split over two thread halves (one per
//     velocity sign), then the tile moves as 16-byte cp.async chunks from
//     every thread; stores are 16-byte vector stores;
//   * shared memory rows and population slabs are padded (by a multiple of 16
//     bytes, which keeps the vector copies legal) with the padding that
//     minimises bank conflicts of the sweep and relaxation access patterns,
//     chosen at compile time (degree 3 in 2D: grouped sweeps, pm_group4);
//   * a sweep item is one (axis, variable, line) for both velocity signs;
//     the relaxation works on node pairs with packed FP32 instructions.
#pragma once

#include <type_traits>

#include "kin_device.cuh"

namespace kin {

// ---------------------------------------------------------------------------
// compile-time layout
// ---------------------------------------------------------------------------

template <int D, int P, int SYS, typename T, int B0, int B1, int B2>
struct Shape {
    static constexpr int NP = P + 1;
    static constexpr int NN = ipow(NP, D);
    static constexpr int TN = ipow(NP, D - 1);
    static constexpr int M = nvars(D, SYS);
    static constexpr int NPOP = 2 * D * M;
    static constexpr int NROWS = B1 * B2;
    static constexpr int ROWLEN = B0 * NN;
    static constexpr int CELLS = B0 * B1 * B2;
    static constexpr int NODES = CELLS * NN;
    static constexpr int VEC = 16 / (int)sizeof(T);      // elements per 16 bytes
    static constexpr int ext(int a) { return a == 0 ? B0 : (a == 1 ? B1 : B2); }
    static constexpr int lines(int a) { return (CELLS / ext(a)) * TN; }   // per population
    static constexpr int t1(int a) { return a == 0 ? 1 : 0; }
    static constexpr int t2(int a) { return a == 2 ? 1 : 2; }
    static constexpr int nstep(int a) { return a == 0 ? 1 : (a == 1 ? NP : NP * NP); }

    // shared-memory offset of (cell x, y, z, node) for given row / slab pads
    static constexpr int rstr(int rp) { return ROWLEN + rp; }
    static constexpr int pstr(int rp, int pp) { return NROWS * rstr(rp) + pp; }
    static constexpr int cell_off(int rp, int x, int y, int z) { return (z * B1 + y) * rstr(rp) + x * NN; }
    static constexpr int cstep(int rp, int a) { return a == 0 ? NN : (a == 1 ? rstr(rp) : B1 * rstr(rp)); }

    // smem offset of the first element of (axis a, population-local pl, line)
    static constexpr int line_base(int rp, int pp, int a, int pl_pop, int line)
    {
        const int tnode = line % TN, tcell = line / TN;
        const int j1 = tnode % NP, j2 = tnode / NP;
        const int e1 = ext(t1(a));
        const int c1 = D > 1 ? tcell % e1 : 0, c2 = D > 2 ? tcell / e1 : 0;
        int c[3] = {0, 0, 0}, j[3] = {0, 0, 0};
        if (D > 1) {
            c[t1(a)] = c1;
            j[t1(a)] = j1;
        }
        if (D > 2) {
            c[t2(a)] = c2;
            j[t2(a)] = j2;
        }
        return pl_pop * pstr(rp, pp) + cell_off(rp, c[0], c[1], c[2]) + j[0] + j[1] * NP + j[2] * NP * NP;
    }

    // worst bank multiplicity of one warp access (32 consecutive items)
    static constexpr int banks_of(int words_per_elem, const int* addr, int n)
    {
        // 32 banks of 4 bytes; an 8-byte element occupies two banks
        int cnt[32] = {};
        int worst = 0;
        for (int i = 0; i < n; ++i) {
            for (int w = 0; w < words_per_elem; ++w) {
                const int b = (addr[i] * words_per_elem + w) % 32;
                ++cnt[b];
                if (cnt[b] > worst) worst = cnt[b];
            }
        }
        return worst;
    }

    static constexpr int conflict_cost(int rp, int pp)
    {
        const int wpe = (int)sizeof(T) / 4;
        int cost = 0;
        // sweeps: the first warp of each axis's items (lines fastest, then populations)
        for (int a = 0; a < D; ++a) {
            int addr[32] = {};
            for (int i = 0; i < 32; ++i) {
                const int pl = i / lines(a), line = i % lines(a);
                addr[i] = line_base(rp, pp, a, pl, line);
            }
            cost += banks_of(wpe, addr, 32);
        }
        // relaxation: 32 consecutive nodes of population 0 and 1
        for (int pop = 0; pop < 2; ++pop) {
            int addr[32] = {};
            for (int i = 0; i < 32; ++i) {
                const int nd = i % NODES;
                addr[i] = pop * pstr(rp, pp) + (nd / ROWLEN) * rstr(rp) + nd % ROWLEN;
            }
            cost += banks_of(wpe, addr, 32);
        }
        return cost;
    }

    static constexpr int best_pad(bool want_rp)
    {
        int best_rp = 0, best_pp = 0, best = 1 << 30;
        for (int rp = 0; rp < 32; rp += VEC)
            for (int pp = 0; pp < 32; pp += VEC) {
                const int c = conflict_cost(rp, pp) * 1024 + rp + pp;   // prefer small pads on ties
                if (c < best) {
                    best = c;
                    best_rp = rp;
                    best_pp = pp;
                }
            }
        return want_rp ? best_rp : best_pp;
    }

    // Degree 3 in 2D (FP32): a cell row of nodes is one 16-byte word, and
    // lines are swept four at a time with 16-byte shared-memory accesses
    // (pm_group4).  Row pad 4 makes the word index of consecutive cell rows
    // odd apart, and the slab pad makes consecutive populations one word
    // apart modulo 8, so the 8 words of a quarter warp hit distinct bank
    // groups for both axes.
    static constexpr bool G4 = D == 2 && NP == 4 && sizeof(T) == 4 && B1 % 8 == 0 && B0 % 2 == 0 && M == 4;
    static constexpr int g4_pp()
    {
        for (int pp = 0; pp < 32; pp += 4)
            if (((NROWS * (ROWLEN + 4) + pp) / 4) % 8 == 1) return pp;
        return 0;
    }
    static constexpr int RP = G4 ? 4 : best_pad(true);
    static constexpr int PP = G4 ? g4_pp() : best_pad(false);
    static constexpr int RSTR = rstr(RP);
    static constexpr int PSTR = pstr(RP, PP);
    static constexpr int TILE = NPOP * PSTR;                        // elements per tile buffer
    static constexpr size_t SMEM = sizeof(T) * (size_t)TILE;
    // line items of the tile, axis by axis: (variable, line) pairs; each
    // item stands for the + and the - population of its line
    static constexpr int E0 = M * lines(0);
    static constexpr int E1 = E0 + (D > 1 ? M * lines(1) : 0);
    static constexpr int ITEMS = E1 + (D > 2 ? M * lines(2) : 0);
    static constexpr int eoff(int a) { return a == 0 ? 0 : (a == 1 ? E0 : E1); }
    // inflow traces of the tile (shared memory after the tile buffers): [sign][item]
    static constexpr size_t TIN_BYTES = sizeof(T) * (size_t)(((2 * ITEMS * sizeof(T) + 15) / 16) * 16 / sizeof(T));
    // lines of one sign of axis a handled by each thread of a sign half
    static constexpr int kpt(int a, int half) { return (M * lines(a) + half - 1) / half; }
    static constexpr int kpt_max(int half)
    {
        return kpt(0, half) > (D > 1 ? kpt(1, half) : 0)
                   ? (kpt(0, half) > (D > 2 ? kpt(2, half) : 0) ? kpt(0, half) : kpt(2, half))
                   : ((D > 1 ? kpt(1, half) : 0) > (D > 2 ? kpt(2, half) : 0) ? kpt(1, half) : kpt(2, half));
    }
};

// ---------------------------------------------------------------------------
// kernel pieces
// ---------------------------------------------------------------------------

// Global line id (summary slab index) of a line of axis A in the tile at org.
template <int D, int NP, int A, int B0, int B1>
__device__ __forceinline__ long long fixed_gline(const Inst& I, int line, int org0, int org1, int org2)
{
    constexpr int TN = ipow(NP, D - 1);
    constexpr int T1 = A == 0 ? 1 : 0;
    constexpr int T2 = A == 2 ? 1 : 2;
    constexpr int E1 = T1 == 0 ? B0 : B1;
    const int tnode = line % TN, tcell = line / TN;
    if (D == 1) return 0;
    const int c1 = tcell % E1, c2 = D > 2 ? tcell / E1 : 0;
    const int o1 = T1 == 0 ? org0 : (T1 == 1 ? org1 : org2);
    const int o2 = T2 == 1 ? org1 : org2;
    long long gt;
    if (D == 3) gt = (long long)(o2 + c2) * I.n[T1] + (o1 + c1);
    else gt = o1 + c1;
    return gt * TN + tnode;
}

// Coefficient k of direction dir: from the launch parameters (one problem
// per launch), or for batched launches from a shared-memory copy when one is
// given, else from the instance's launch record in global memory.
template <bool BATCH, typename T>
__device__ __forceinline__ T cget(const Inst& I, const T* csm, int dir, int k)
{
    if constexpr (BATCH)
        return csm ? csm[dir * kCoefStride + k] : coef_of(I, dir, k, T(0));
    else
        return coef_of(I, dir, k, T(0));
}

// Sweep (MODE 1) or block summaries (MODE 2) of one line item of axis A:
// variable v, line 'line', for both velocity signs of the axis.  The
// look-back inflows come from tin[sign][item].
template <int D, int P, int SYS, typename T, int B0, int B1, int B2, int A, int MODE, bool BATCH>
__device__ __forceinline__ void pm_item(const Inst& I, int local, int org0, int org1, int org2, int bidx, T* s,
                                        const T* tin, const T* csm)
{
    using S = Shape<D, P, SYS, T, B0, B1, B2>;
    constexpr int NP = S::NP, M = S::M, LP = S::lines(A), BA = S::ext(A);
    constexpr int CST = S::cstep(S::RP, A), NS = S::nstep(A);
    const int v = local / LP, line = local - (local / LP) * LP;
    const int popP = (2 * A) * M + v;
    T* const sp = s + S::line_base(S::RP, S::PP, A, popP, line);     // + population
    T* const sm = sp + M * S::PSTR;                                    // - population (pop + M)
    // the two directions one after the other: the + line upward, then the -
    // line downward (packing the two into FP32 pair instructions measured
    // slower: the operand pairs had to be assembled from separate words)
#pragma unroll
    for (int sg = 0; sg < 2; ++sg) {
        const int dir = 2 * A + sg;
        T* const base = sg == 0 ? sp : sm;
        if (MODE == 1) {
            T t = tin[sg * S::ITEMS + S::eoff(A) + local];
#pragma unroll
            for (int cc = 0; cc < BA; ++cc) {
                T* const p = base + (sg == 0 ? cc : BA - 1 - cc) * CST;
                T u[NP], du[NP], dlt[NP];
#pragma unroll
                for (int j = 0; j < NP; ++j) {
                    u[j] = p[j * NS];
                    du[j] = u[j] - t;
                }
                // difference form (P - I)(u - t 1) of (P - I) u + g t: exact
                // for constant states whatever the coefficients' rounding
#pragma unroll
                for (int i = 0; i < NP; ++i) {
                    T acc = cget<BATCH>(I, csm, dir, i * NP) * du[0];
#pragma unroll
                    for (int j = 1; j < NP; ++j) acc = fma(cget<BATCH>(I, csm, dir, i * NP + j), du[j], acc);
                    dlt[i] = acc;
                }
                t = sg == 0 ? u[NP - 1] + dlt[NP - 1] : u[0] + dlt[0];
#pragma unroll
                for (int i = 0; i < NP; ++i) p[i * NS] = fma(T(2), dlt[i], u[i]);
            }
        } else {
            const T rho = cget<BATCH>(I, csm, dir, kOffRho);
            T t = 0;
#pragma unroll
            for (int cc = 0; cc < BA; ++cc) {
                const T* const p = base + (sg == 0 ? cc : BA - 1 - cc) * CST;
                T acc = cget<BATCH>(I, csm, dir, kOffProw) * p[0];
#pragma unroll
                for (int j = 1; j < NP; ++j) acc = fma(cget<BATCH>(I, csm, dir, kOffProw + j), p[j * NS], acc);
                t = fma(rho, t, acc);
            }
            const T last = sg == 0 ? sp[(BA - 1) * CST + (NP - 1) * NS] : sm[0];
            const int nbk = I.nblk[A], nbs = I.nb[A];
            const int q = sg == 0 ? bidx : nbk - 1 - bidx;
            const int Sd = (int)fdiv((unsigned)q, I.fd_nb[A]);
            const long long gl = I.ax[A].glines;
            const long long gline = fixed_gline<D, NP, A, B0, B1>(I, line, org0, org1, org2);
            const int pop = popP + sg * M;
            static_cast<T*>(I.sig_out)[(long long)pop * I.sig_stride + (long long)q * gl + gline] = t;
            if (q - Sd * nbs == nbs - 1)
                static_cast<T*>(I.raw_out)[(long long)pop * I.raw_stride + (long long)Sd * gl + gline] = last;
        }
    }
}

// Every line item of the tile, axis after axis, spread over all threads
// (items it, it + NTH, ...).  Axis boundaries fall on warp boundaries for
// the compiled shapes, so the axis branch does not split a warp.
// Sweep (MODE 1) or block summaries (MODE 2) of a group of four lines for
// degree 3 in 2D (Shape::G4).  Group items: first the x groups
// ((sign, variable) major, y-cell row c1 fastest: the four lines of one row
// of cells, y-nodes j1 = 0..3), then the y groups ((sign, x-cell) major,
// variable fastest: the four lines of one column of cells, x-nodes
// j0 = 0..3).  Every shared-memory access moves one 16-byte word: the four
// x-nodes of one line of a cell (x groups), or one y-node of all four lines
// (y groups).  Inflows and summaries of the four lines are consecutive.
template <int D, int P, int SYS, typename T, int B0, int B1, int B2, int MODE, bool BATCH>
__device__ __forceinline__ void pm_group4(const Inst& I, int git, int org0, int org1, int bx, int by, T* s,
                                          const T* tin, const T* csm)
{
    using S = Shape<D, P, SYS, T, B0, B1, B2>;
    constexpr int M = S::M, NN = 16;
    constexpr int GX = 2 * M * B1;
    const bool xa = git < GX;
    int sg, v, c, A;
    if (xa) {
        A = 0;
        sg = git / (M * B1);
        v = (git / B1) % M;
        c = git % B1;                   // y-cell row
    } else {
        const int gy = git - GX;
        A = 1;
        v = gy % M;
        c = (gy / M) % B0;              // x-cell column
        sg = gy / (M * B0);
    }
    const int dir = 2 * A + sg;
    const int pop = dir * M + v;
    T* const slab = s + pop * S::PSTR;
    const int lineoff = v * S::lines(A) + c * 4;            // item index of line 0 of the group
    float4* const tin4 = (float4*)(tin + sg * S::ITEMS + S::eoff(A) + lineoff);
    const int BA = xa ? B0 : B1;
    auto word = [&](int cc, int j) -> float4* {
        // cell cc along the sweep axis (already in sweep order), word j
        const int cell = sg == 0 ? cc : BA - 1 - cc;
        const int off = xa ? c * S::RSTR + cell * NN : cell * S::RSTR + c * NN;
        return reinterpret_cast<float4*>(slab + off + 4 * j);
    };
    if (MODE == 1) {
        float Pm[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) Pm[i][j] = cget<BATCH>(I, csm, dir, i * 4 + j);
        const float4 t0 = *tin4;
        float t[4] = {t0.x, t0.y, t0.z, t0.w};
        // the cell loop is unrolled per axis so that every offset is an immediate
        auto cellstep = [&](int cc) {
            float u[4][4];              // u[line][node along the line]
            float4 w[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) w[j] = *word(cc, j);
#pragma unroll
            for (int l = 0; l < 4; ++l)
#pragma unroll
                for (int n = 0; n < 4; ++n) {
                    // x groups: word l holds the nodes of line l; y groups: word n holds node n of all lines
                    const float4 q = xa ? w[l] : w[n];
                    const int e = xa ? n : l;
                    u[l][n] = e == 0 ? q.x : (e == 1 ? q.y : (e == 2 ? q.z : q.w));
                }
            float nw[4][4];
#pragma unroll
            for (int l = 0; l < 4; ++l) {
                float dlt[4], du[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) du[j] = u[l][j] - t[l];
                // difference form, as in pm_item
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    float acc = Pm[i][0] * du[0];
#pragma unroll
                    for (int j = 1; j < 4; ++j) acc = fmaf(Pm[i][j], du[j], acc);
                    dlt[i] = acc;
                }
                t[l] = sg == 0 ? u[l][3] + dlt[3] : u[l][0] + dlt[0];
#pragma unroll
                for (int i = 0; i < 4; ++i) nw[l][i] = fmaf(2.0f, dlt[i], u[l][i]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j)
                *word(cc, j) = xa ? make_float4(nw[j][0], nw[j][1], nw[j][2], nw[j][3])
                                  : make_float4(nw[0][j], nw[1][j], nw[2][j], nw[3][j]);
        };
        if (xa) {
#pragma unroll
            for (int cc = 0; cc < B0; ++cc) cellstep(cc);
        } else {
#pragma unroll
            for (int cc = 0; cc < B1; ++cc) cellstep(cc);
        }
    } else {
        float prow[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) prow[j] = cget<BATCH>(I, csm, dir, kOffProw + j);
        const float rho = cget<BATCH>(I, csm, dir, kOffRho);
        float t[4] = {0.f, 0.f, 0.f, 0.f}, last[4];
        auto cellsum = [&](int cc, bool final_cell) {
            float4 w[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) w[j] = *word(cc, j);
#pragma unroll
            for (int l = 0; l < 4; ++l) {
                float u[4];
#pragma unroll
                for (int n = 0; n < 4; ++n) {
                    const float4 q = xa ? w[l] : w[n];
                    const int e = xa ? n : l;
                    u[n] = e == 0 ? q.x : (e == 1 ? q.y : (e == 2 ? q.z : q.w));
                }
                float acc = prow[0] * u[0];
#pragma unroll
                for (int j = 1; j < 4; ++j) acc = fmaf(prow[j], u[j], acc);
                t[l] = fmaf(rho, t[l], acc);
                if (final_cell) last[l] = sg == 0 ? u[3] : u[0];
            }
        };
        if (xa) {
#pragma unroll
            for (int cc = 0; cc < B0; ++cc) cellsum(cc, cc == B0 - 1);
        } else {
#pragma unroll
            for (int cc = 0; cc < B1; ++cc) cellsum(cc, cc == B1 - 1);
        }
        const int nbk = I.nblk[A], nbs = I.nb[A];
        const int bidx = xa ? bx : by;
        const int q = sg == 0 ? bidx : nbk - 1 - bidx;
        const int Sd = (int)fdiv((unsigned)q, I.fd_nb[A]);
        const long long gl = I.ax[A].glines;
        // lines (cell c of the transverse axis, node 0..3): glines 4 (origin + c) + 0..3
        const long long gline0 = 4LL * ((xa ? org1 : org0) + c);
        *reinterpret_cast<float4*>(static_cast<float*>(I.sig_out) + (long long)pop * I.sig_stride +
                                   (long long)q * gl + gline0) = make_float4(t[0], t[1], t[2], t[3]);
        if (q - Sd * nbs == nbs - 1)
            *reinterpret_cast<float4*>(static_cast<float*>(I.raw_out) + (long long)pop * I.raw_stride +
                                       (long long)Sd * gl + gline0) = make_float4(last[0], last[1], last[2], last[3]);
    }
}

template <int D, int P, int SYS, typename T, int B0, int B1, int B2, int NTH, int MODE, bool BATCH>
__device__ __forceinline__ void fixed_pm_all(const Inst& I, int org0, int org1, int org2, int bx, int by, int bz,
                                             T* s, const T* tin, const T* csm)
{
    using S = Shape<D, P, SYS, T, B0, B1, B2>;
    if constexpr (S::G4) {
        constexpr int NG = 2 * S::M * (B0 + B1);
#pragma unroll
        for (int k = 0; k < (NG + NTH - 1) / NTH; ++k) {
            const int git = threadIdx.x + k * NTH;
            if (NG % NTH != 0 && git >= NG) break;
            pm_group4<D, P, SYS, T, B0, B1, B2, MODE, BATCH>(I, git, org0, org1, bx, by, s, tin, csm);
        }
        return;
    }
#pragma unroll
    for (int k = 0; k < (S::ITEMS + NTH - 1) / NTH; ++k) {
        const int it = threadIdx.x + k * NTH;
        if (S::ITEMS % NTH != 0 && it >= S::ITEMS) break;
        if (it < S::E0) {
            pm_item<D, P, SYS, T, B0, B1, B2, 0, MODE, BATCH>(I, it, org0, org1, org2, bx, s, tin, csm);
        } else if (D == 2 || it < S::E1) {
            if constexpr (D > 1) pm_item<D, P, SYS, T, B0, B1, B2, 1, MODE, BATCH>(I, it - S::E0, org0, org1, org2, by, s, tin, csm);
        } else {
            if constexpr (D > 2) pm_item<D, P, SYS, T, B0, B1, B2, 2, MODE, BATCH>(I, it - S::E1, org0, org1, org2, bz, s, tin, csm);
        }
    }
}

// Look-back plan of one axis for this thread's sign: the block index q,
// subdomain S and the start of the walk over the summary blocks are the same
// for every line of the (axis, sign); the raw value of subdomain S-K starts
// every line's fold (see chain_inflow for the meaning).  off[k] receives the
// 32-bit element offset of line k's summaries (block 0).
template <int D, int P, int SYS, typename T, int B0, int B1, int B2, int NTH, int A, int KM>
__device__ __forceinline__ void chain_setup(const Inst& I, int hid, int sgn, int org0, int org1, int org2,
                                            int bidx, T (&tr)[KM], int (&off)[KM], int& qj, int& cnt, T& RB)
{
    using S = Shape<D, P, SYS, T, B0, B1, B2>;
    constexpr int NP = S::NP, M = S::M, HALF = NTH / 2;
    constexpr int LP = S::lines(A);
    constexpr int ITEMS = M * LP;
    constexpr int KPT = S::kpt(A, HALF);
    const int nbk = I.nblk[A], nbs = I.nb[A], NSa = I.NS[A], K = I.iters;
    const int q = sgn == 0 ? bidx : nbk - 1 - bidx;
    const int Sd = (int)fdiv((unsigned)q, I.fd_nb[A]);
    const int r = q - Sd * nbs;
    int s0 = Sd - K;
    // an inflow axis whose walk reaches the domain boundary starts there from
    // the boundary value and folds every block from the first one
    const bool from_bnd = I.inflow[A] && s0 < 0;
    while (s0 < 0) s0 += NSa;
    const long long gl = I.ax[A].glines;
    cnt = from_bnd ? Sd * nbs + r : (K - 1) * nbs + r;
    qj = from_bnd ? 0 : ((s0 + 1 == NSa) ? 0 : (s0 + 1) * nbs);
    // only the last lbdepth blocks of the walk matter (see Inst::lbdepth):
    // a longer walk starts that many blocks upstream from a zero inflow
    const int depth = I.lbdepth[2 * A + sgn];
    const bool trunc = cnt > depth;
    if (trunc) {
        qj = (qj + cnt - depth) % nbk;
        cnt = depth;
    }
    RB = coef_of(I, 2 * A + sgn, kOffRhoB, T(0));
    const T* __restrict__ raw = static_cast<const T*>(I.raw_in) + (long long)s0 * gl;
#pragma unroll
    for (int k = 0; k < KM; ++k) {
        const int it = hid + k * HALF;
        if (k >= KPT || (ITEMS % HALF != 0 && it >= ITEMS)) {
            off[k] = 0;       // a valid address; the item's result is never used
            tr[k] = T(0);
            continue;
        }
        const int v = it / LP, line = it % LP;
        const long long gline = fixed_gline<D, NP, A, B0, B1>(I, line, org0, org1, org2);
        const int pop = (2 * A + sgn) * M + v;
        off[k] = (int)((long long)pop * I.sig_stride + gline);   // fits: checked on the host
        tr[k] = trunc ? T(0)
                      : __ldg(from_bnd ? static_cast<const T*>(I.bnd) + pop
                                       : raw + (long long)pop * I.raw_stride + gline);
    }
}

// Look-back inflows of all lines of this thread (every axis of its sign),
// folded before the tile's copies are issued.  The walks of all axes advance
// together one summary block per step: every line keeps the 32-bit element
// index of its next summary, which moves by the line count of its axis and
// wraps (periodically) after the last block; the unrolled steps let the
// loads of several steps be in flight at once.
template <int D, int P, int SYS, typename T, int B0, int B1, int B2, int NTH>
__device__ __forceinline__ void fixed_chain(const Inst& I, int org0, int org1, int org2, int bx, int by, int bz,
                                            T* tin)
{
    using S = Shape<D, P, SYS, T, B0, B1, B2>;
    constexpr int HALF = NTH / 2;
    constexpr int KM = S::kpt_max(HALF);
    T tr[3][KM];
    constexpr int KP[3] = {S::kpt(0, HALF), D > 1 ? S::kpt(1, HALF) : 0, D > 2 ? S::kpt(2, HALF) : 0};
    const int tid = threadIdx.x;
    const int sgn = tid < HALF ? 0 : 1;
    const int hid = tid - sgn * HALF;
    int idx[3][KM];
    int qj[3] = {0, 0, 0}, cnt[3] = {0, 0, 0};
    T RB[3] = {T(0), T(0), T(0)};
    chain_setup<D, P, SYS, T, B0, B1, B2, NTH, 0, KM>(I, hid, sgn, org0, org1, org2, bx, tr[0], idx[0], qj[0],
                                                      cnt[0], RB[0]);
    if constexpr (D > 1)
        chain_setup<D, P, SYS, T, B0, B1, B2, NTH, 1, KM>(I, hid, sgn, org0, org1, org2, by, tr[1], idx[1],
                                                          qj[1], cnt[1], RB[1]);
    if constexpr (D > 2)
        chain_setup<D, P, SYS, T, B0, B1, B2, NTH, 2, KM>(I, hid, sgn, org0, org1, org2, bz, tr[2], idx[2],
                                                          qj[2], cnt[2], RB[2]);
    const T* __restrict__ sig = static_cast<const T*>(I.sig_in);
    int gl[3], left[3], wrap[3];
    int maxcnt = 0;
#pragma unroll
    for (int A = 0; A < D; ++A) {
        gl[A] = (int)I.ax[A].glines;
        left[A] = I.nblk[A] - qj[A];            // steps before the walk wraps to block 0
        wrap[A] = I.nblk[A] * gl[A];
#pragma unroll
        for (int k = 0; k < KM; ++k)
            if (k < KP[A]) idx[A][k] += qj[A] * gl[A];
        maxcnt = cnt[A] > maxcnt ? cnt[A] : maxcnt;
    }
#pragma unroll 4
    for (int j = 0; j < maxcnt; ++j) {
#pragma unroll
        for (int A = 0; A < D; ++A) {
            if (j < cnt[A]) {
                const bool w = --left[A] == 0;
                const int step = w ? gl[A] - wrap[A] : gl[A];
                left[A] = w ? I.nblk[A] : left[A];
#pragma unroll
                for (int k = 0; k < KM; ++k)
                    if (k < KP[A]) {
                        tr[A][k] = fma(RB[A], tr[A][k], __ldg(sig + idx[A][k]));
                        idx[A][k] += step;
                    }
            }
        }
    }
    // tin[sign][item]; item = offset of the axis + (variable, line) index
#pragma unroll
    for (int A = 0; A < D; ++A)
#pragma unroll
        for (int k = 0; k < KM; ++k) {
            const int it = hid + k * HALF;
            if (k < KP[A] && it < S::M * S::lines(A)) tin[sgn * S::ITEMS + S::eoff(A) + it] = tr[A][k];
        }
}

template <int D, int P, int SYS, typename T, int B0, int B1, int B2, int NTH>
__device__ __forceinline__ void fixed_relax(const Inst& I, T* s)
{
    using S = Shape<D, P, SYS, T, B0, B1, B2>;
    constexpr int M = S::M, NV = 2 * D, NPOP = S::NPOP;
    const T omega = T(I.omega);
    const bool two = I.omega == 2.0;
    const T inv2l = T(1.0 / (2.0 * I.lambda));
    const T gm1 = T(I.gamma - 1.0);
#pragma unroll
    for (int k = 0; k < (S::NODES + NTH - 1) / NTH; ++k) {
        const int nd = threadIdx.x + k * NTH;
        if (S::NODES % NTH != 0 && nd >= S::NODES) break;
        const int o = (nd / S::ROWLEN) * S::RSTR + nd % S::ROWLEN;
        T fk[NPOP];
#pragma unroll
        for (int pp = 0; pp < NPOP; ++pp) fk[pp] = s[pp * S::PSTR + o];
        T W[M];
#pragma unroll
        for (int v = 0; v < M; ++v) {
            Acc<T> acc;
#pragma unroll
            for (int kk = 0; kk < NV; ++kk) acc.add(fk[kk * M + v]);
            W[v] = acc.s;
        }
        if constexpr (SYS == kMaxwell) {
            maxwell_relax_node(fk, W, T(I.mu), T(1) - omega, inv2l);
#pragma unroll
            for (int pp = 0; pp < NPOP; ++pp) s[pp * S::PSTR + o] = fk[pp];
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
        for (int pp = 0; pp < NPOP; ++pp) s[pp * S::PSTR + o] = fk[pp];
    }
}

// Packed FP32 pairs (two lanes per instruction; each lane is the scalar IEEE
// operation of the same name).
__device__ __forceinline__ float2 f2(float x) { return make_float2(x, x); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// div2d on a node pair
template <int D>
__device__ __forceinline__ float2 div2d2(float2 w)
{
    if constexpr (D == 3) {
        const float2 q = __fmul2_rn(w, f2(1.0f / 6.0f));
        return __ffma2_rn(__ffma2_rn(f2(-6.0f), q, w), f2(1.0f / 6.0f), q);
    } else {
        return __fmul2_rn(w, f2((float)(1.0 / (2.0 * D))));
    }
}

// The relaxation of fixed_relax on two neighbouring nodes at a time (FP32,
// rows of even length): the populations of a node pair are one 8-byte
// shared-memory word each, and every step is a packed pair operation.
template <int D, int P, int SYS, int B0, int B1, int B2, int NTH>
__device__ __forceinline__ void fixed_relax_pairs(const Inst& I, float* s)
{
    using S = Shape<D, P, SYS, float, B0, B1, B2>;
    constexpr int M = S::M, NV = 2 * D, NPOP = S::NPOP;
    constexpr int NPAIR = S::NODES / 2;
    static_assert(S::ROWLEN % 2 == 0 && S::RSTR % 2 == 0 && S::PSTR % 2 == 0, "node pairs must be 8-byte words");
    const bool two = I.omega == 2.0;
    const float2 om = f2((float)I.omega), omc = f2(1.0f - (float)I.omega);
    const float2 inv2l = f2((float)(1.0 / (2.0 * I.lambda)));
    const float2 gm1 = f2((float)(I.gamma - 1.0));
    const float2 twof = f2(2.0f);
#pragma unroll
    for (int k = 0; k < (NPAIR + NTH - 1) / NTH; ++k) {
        const int pr = threadIdx.x + k * NTH;
        if (NPAIR % NTH != 0 && pr >= NPAIR) break;
        const int nd = 2 * pr;
        const int o = (nd / S::ROWLEN) * S::RSTR + nd % S::ROWLEN;
        // W = sum_k f_k, compensated (the first term starts the sum exactly);
        // with many populations the pairs are read again for the update
        // instead of being held in registers
        constexpr bool HOLD = NPOP < 16;
        float2 fk[HOLD ? NPOP : 1];
        const unsigned sbase = (unsigned)__cvta_generic_to_shared(s + o);
        auto ld = [&](int pp) {
            if constexpr (HOLD) {
                return *reinterpret_cast<const float2*>(s + pp * S::PSTR + o);
            } else {
                // a fresh read each time (kept out of registers between the passes)
                float2 v;
                asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];"
                             : "=f"(v.x), "=f"(v.y)
                             : "r"(sbase + (unsigned)(pp * S::PSTR * 4))
                             : "memory");
                return v;
            }
        };
        if constexpr (HOLD) {
#pragma unroll
            for (int pp = 0; pp < NPOP; ++pp) fk[pp] = ld(pp);
        }
        auto get = [&](int pp) { if constexpr (HOLD) return fk[pp]; else return ld(pp); };
        float2 W[M];
#pragma unroll
        for (int v = 0; v < M; ++v) {
            float2 sum = get(v), c = f2(0.0f);
#pragma unroll
            for (int kk = 1; kk < NV; ++kk) {
                const float2 y = kk == 1 ? get(kk * M + v) : sub2(get(kk * M + v), c);
                const float2 t = add2(sum, y);
                c = sub2(sub2(t, sum), y);
                sum = t;
            }
            W[v] = sum;
        }
        if constexpr (SYS == kMaxwell) {
            // maxwell_relax_node on node pairs
            const float2 mu = f2((float)I.mu), zero = f2(0.0f);
            auto neg2 = [](float2 x) { return make_float2(-x.x, -x.y); };
            float2 Wp[M];
#pragma unroll
            for (int v = 0; v < M; ++v) Wp[v] = v < 3 ? mul2(mu, W[v]) : W[v];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const int j = (a + 1) % 3, kk = (a + 2) % 3;
                float2 Qm[M], Qp[M];
                Qm[a] = zero; Qm[kk] = neg2(W[3 + j]); Qm[j] = W[3 + kk];
                Qm[3 + a] = zero; Qm[3 + kk] = W[j]; Qm[3 + j] = neg2(W[kk]);
                Qp[a] = zero; Qp[kk] = neg2(Wp[3 + j]); Qp[j] = Wp[3 + kk];
                Qp[3 + a] = zero; Qp[3 + kk] = Wp[j]; Qp[3 + j] = neg2(Wp[kk]);
#pragma unroll
                for (int v = 0; v < M; ++v) {
                    const bool z = v == a || v == 3 + a;
                    const float2 bm = div2d2<D>(W[v]), bp = div2d2<D>(Wp[v]);
                    const float2 hm = z ? zero : mul2(Qm[v], inv2l), hp = z ? zero : mul2(Qp[v], inv2l);
                    const int ip = (2 * a) * M + v, im = (2 * a + 1) * M + v;
                    const float2 fp = get(ip), fm = get(im);
                    const float2 np_ = fma2(omc, sub2(fp, z ? bm : add2(bm, hm)), z ? bp : add2(bp, hp));
                    const float2 nm_ = fma2(omc, sub2(fm, z ? bm : sub2(bm, hm)), z ? bp : sub2(bp, hp));
                    *reinterpret_cast<float2*>(s + ip * S::PSTR + o) = np_;
                    *reinterpret_cast<float2*>(s + im * S::PSTR + o) = nm_;
                }
            }
            continue;
        }
        float2 inv = f2(0.0f), pres = f2(0.0f);
        if (SYS == kEuler) {
            inv = make_float2(__frcp_rn(W[0].x), __frcp_rn(W[0].y));
            float2 ke = mul2(W[1], W[1]);
#pragma unroll
            for (int b = 1; b < D; ++b) ke = fma2(W[1 + b], W[1 + b], ke);
            pres = mul2(gm1, sub2(W[1 + D], mul2(mul2(f2(0.5f), ke), inv)));
        }
#pragma unroll
        for (int a = 0; a < D; ++a) {
            float2 Q[M];
            if (SYS == kAdvection) {
                Q[0] = mul2(f2((float)I.adv[a]), W[0]);
            } else {
                const float2 ua = mul2(W[1 + a], inv);
                Q[0] = W[1 + a];
#pragma unroll
                for (int b = 0; b < D; ++b) Q[1 + b] = b == a ? fma2(W[1 + b], ua, pres) : mul2(W[1 + b], ua);
                Q[1 + D] = mul2(add2(W[1 + D], pres), ua);
            }
#pragma unroll
            for (int v = 0; v < M; ++v) {
                const float2 base = div2d2<D>(W[v]);
                const float2 hq = mul2(Q[v], inv2l);
                const int ip = (2 * a) * M + v, im = (2 * a + 1) * M + v;
                const float2 fp = get(ip), fm = get(im);
                float2 np_, nm_;
                if (two) {
                    np_ = fma2(twof, add2(base, hq), make_float2(-fp.x, -fp.y));
                    nm_ = fma2(twof, sub2(base, hq), make_float2(-fm.x, -fm.y));
                } else {
                    np_ = fma2(om, add2(base, hq), mul2(omc, fp));
                    nm_ = fma2(om, sub2(base, hq), mul2(omc, fm));
                }
                *reinterpret_cast<float2*>(s + ip * S::PSTR + o) = np_;
                *reinterpret_cast<float2*>(s + im * S::PSTR + o) = nm_;
            }
        }
    }
}

// Tile rows move as 16-byte chunks through the load/store units, spread over
// all threads: cp.async (global -> shared) for the loads, shared -> register
// -> global for the stores.  (Bulk copies of whole rows go through the
// per-SM copy engine one short row at a time, which caps loads plus stores
// of rows this short well below the HBM rate.)  Chunks are grouped by G
// populations per pass so that each thread's (row, chunk) decode is done once.
template <int D, int P, int SYS, typename T, int B0, int B1, int B2, int NTH, bool STORE>
__device__ __forceinline__ void fixed_copy(const Inst& I, int org0, int org1, int org2, T* s)
{
    using S = Shape<D, P, SYS, T, B0, B1, B2>;
    static_assert(S::ROWLEN % S::VEC == 0 && S::RSTR % S::VEC == 0 && S::PSTR % S::VEC == 0,
                  "rows must be whole 16-byte chunks");
    constexpr int CPR = S::ROWLEN / S::VEC;                 // chunks per row
    constexpr int PER_POP = S::NROWS * CPR;
    constexpr int G = NTH / PER_POP >= 1 ? NTH / PER_POP : 1;
    constexpr int GC = G * PER_POP;                          // chunks of one population group
    constexpr int KR = (GC + NTH - 1) / NTH;
    constexpr int NG = (S::NPOP + G - 1) / G;
    const long long rowy = (long long)I.n[0] * S::NN;       // elements from row y to y + 1
    const long long rowz = (long long)(D > 1 ? I.n[1] : 1) * rowy;
    T* fb = static_cast<T*>(I.f) + (((long long)org2 * (D > 1 ? I.n[1] : 1) + org1) * I.n[0] + org0) * S::NN;
    int soff[KR], pg[KR];
    long long goff[KR];
    bool ok[KR];
#pragma unroll
    for (int k = 0; k < KR; ++k) {
        const int c = threadIdx.x + k * NTH;
        ok[k] = GC % NTH == 0 || c < GC;
        const int cc = ok[k] ? c : 0;
        pg[k] = cc / PER_POP;
        const int rem = cc - pg[k] * PER_POP;
        const int row = rem / CPR, cq = rem - (rem / CPR) * CPR;
        const int ly = row % B1, lz = row / B1;
        soff[k] = pg[k] * S::PSTR + row * S::RSTR + cq * S::VEC;
        goff[k] = (long long)pg[k] * I.nodes + lz * rowz + ly * rowy + cq * S::VEC;
    }
#pragma unroll
    for (int g = 0; g < NG; ++g) {
#pragma unroll
        for (int k = 0; k < KR; ++k) {
            if (!ok[k] || (S::NPOP % G != 0 && g * G + pg[k] >= S::NPOP)) continue;
            T* sp = s + g * G * S::PSTR + soff[k];
            T* gp = fb + (long long)(g * G) * I.nodes + goff[k];
            if (STORE) *reinterpret_cast<uint4*>(gp) = *reinterpret_cast<const uint4*>(sp);
            else cp16_g2s(sp, gp);
        }
    }
    if (!STORE) cp_commit();
}

// The work of one tile once its data is in shared memory: sweep, relax,
// store, write the summaries, and meet at a barrier before the buffer is
// reused.
template <int D, int P, int SYS, typename T, int B0, int B1, int B2, int NTH, bool BATCH>
__device__ __forceinline__ void fixed_compute(const Inst& I, int t, T* s, const T* tin, const T* csm)
{
    const TileXYZ c = tile_xyz(I, t);
    const int org0 = c.bx * B0, org1 = c.by * B1, org2 = c.bz * B2;
    if (I.mode == 0) {
        fixed_pm_all<D, P, SYS, T, B0, B1, B2, NTH, 1, BATCH>(I, org0, org1, org2, c.bx, c.by, c.bz, s, tin, csm);
        __syncthreads();
        if constexpr (std::is_same<T, float>::value && Shape<D, P, SYS, T, B0, B1, B2>::ROWLEN % 2 == 0)
            fixed_relax_pairs<D, P, SYS, B0, B1, B2, NTH>(I, s);
        else
            fixed_relax<D, P, SYS, T, B0, B1, B2, NTH>(I, s);
        __syncthreads();
        fixed_copy<D, P, SYS, T, B0, B1, B2, NTH, true>(I, org0, org1, org2, s);
    }
    fixed_pm_all<D, P, SYS, T, B0, B1, B2, NTH, 2, BATCH>(I, org0, org1, org2, c.bx, c.by, c.bz, s, tin, csm);
    __syncthreads();
}

template <int D, int P, int SYS, typename T, int B0, int B1, int B2, int NTH>
__device__ __forceinline__ void fixed_load(const Inst& I, int t, T* s)
{
    const TileXYZ c = tile_xyz(I, t);
    fixed_copy<D, P, SYS, T, B0, B1, B2, NTH, false>(I, c.bx * B0, c.by * B1, c.bz * B2, s);
}

template <int D, int P, int SYS, typename T, int B0, int B1, int B2, int NTH>
__device__ __forceinline__ void fixed_chain_tile(const Inst& I, int t, T* tin)
{
    const TileXYZ c = tile_xyz(I, t);
    fixed_chain<D, P, SYS, T, B0, B1, B2, NTH>(I, c.bx * B0, c.by * B1, c.bz * B2, c.bx, c.by, c.bz, tin);
}

// Fixed-shape step kernel on a persistent grid (blocks walk tiles
// blockIdx.x + k gridDim.x).  With STG = 1 a tile's look-back inflows are
// folded, then its copies issued and waited for, then it is computed.  With STG = 2 the
// block owns two tile buffers: the next tile's copies are issued before the
// current tile is computed, so loads of one tile overlap the work on the
// previous one.
template <int D, int P, int SYS, typename T, int B0, int B1, int B2, int NTH, int MINB, int STG>
__global__ void __launch_bounds__(NTH, MINB) step_kernel_fixed(const __grid_constant__ Inst I)
{
    using S = Shape<D, P, SYS, T, B0, B1, B2>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T* const s0 = reinterpret_cast<T*>(smem_raw);
    T* const s1 = s0 + (STG == 2 ? S::TILE : 0);
    T* const tin = s0 + STG * S::TILE;       // look-back inflows of the current tile
    const int ntiles = I.nblk[0] * I.nblk[1] * I.nblk[2];
    int t = blockIdx.x;
    if (t >= ntiles) return;
    if (STG == 2) fixed_load<D, P, SYS, T, B0, B1, B2, NTH>(I, t, s0);
    for (int i = 0; t < ntiles; ++i, t += gridDim.x) {
        T* const cur = (i & 1) ? s1 : s0;
        // (one buffer: the look-back first, so that its summary loads do not
        // queue behind the tile's copies; the other resident blocks keep
        // HBM busy meanwhile)
        if (I.mode == 0) fixed_chain_tile<D, P, SYS, T, B0, B1, B2, NTH>(I, t, tin);
        if (STG == 1) fixed_load<D, P, SYS, T, B0, B1, B2, NTH>(I, t, cur);
        const int tn = t + gridDim.x;
        if (STG == 2 && tn < ntiles) {
            fixed_load<D, P, SYS, T, B0, B1, B2, NTH>(I, tn, (i & 1) ? s0 : s1);
            cp_wait_prior();
        } else {
            cp_wait_all();
        }
        __syncthreads();
        fixed_compute<D, P, SYS, T, B0, B1, B2, NTH, false>(I, t, cur, tin, nullptr);
    }
}

// Batched fixed-shape step kernel: the thread blocks walk a work list of
// (instance, tile) pairs over several independent problems of the same
// kernel type, with the same one- or two-buffer schedule.  Launch records
// are read from global memory (read-only for the launch).
template <int D, int P, int SYS, typename T, int B0, int B1, int B2, int NTH, int MINB, int STG>
__global__ void __launch_bounds__(NTH, MINB)
    step_kernel_fixed_batch(const Inst* __restrict__ insts, const int2* __restrict__ work, int nwork)
{
    using S = Shape<D, P, SYS, T, B0, B1, B2>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T* const s0 = reinterpret_cast<T*>(smem_raw);
    T* const s1 = s0 + (STG == 2 ? S::TILE : 0);
    T* const tin = s0 + STG * S::TILE;
    int w = blockIdx.x;
    if (w >= nwork) return;
    int2 wk = work[w];
    if (STG == 2) fixed_load<D, P, SYS, T, B0, B1, B2, NTH>(insts[wk.x], wk.y, s0);
    for (int i = 0; w < nwork; ++i, w += gridDim.x) {
        const Inst& I = insts[wk.x];
        T* const cur = (i & 1) ? s1 : s0;
        if (I.mode == 0) fixed_chain_tile<D, P, SYS, T, B0, B1, B2, NTH>(I, wk.y, tin);
        if (STG == 1) fixed_load<D, P, SYS, T, B0, B1, B2, NTH>(I, wk.y, cur);
        const int wn = w + gridDim.x;
        int2 wkn = wk;
        if (wn < nwork) wkn = work[wn];
        if (STG == 2 && wn < nwork) {
            fixed_load<D, P, SYS, T, B0, B1, B2, NTH>(insts[wkn.x], wkn.y, (i & 1) ? s0 : s1);
            cp_wait_prior();
        } else {
            cp_wait_all();
        }
        __syncthreads();
        fixed_compute<D, P, SYS, T, B0, B1, B2, NTH, true>(I, wk.y, cur, tin, nullptr);
        wk = wkn;
    }
}

}  // namespace kin

namespace kin {

// ---------------------------------------------------------------------------
// One launch per step for a batch of 2D Euler problems of different degrees
// ---------------------------------------------------------------------------

// One tile of a fixed shape with one shared-memory buffer: look-back, load,
// sweep, relaxation, store, summaries (the one-buffer schedule of
// step_kernel_fixed), ending at a barrier so that the buffer can be reused.
template <int D, int P, int SYS, typename T, int B0, int B1, int B2, int NTH>
__device__ __forceinline__ void fixed_tile_1buf(const Inst& I, int t, T* s, T* tin)
{
    if (I.mode == 0) fixed_chain_tile<D, P, SYS, T, B0, B1, B2, NTH>(I, t, tin);
    fixed_load<D, P, SYS, T, B0, B1, B2, NTH>(I, t, s);
    cp_wait_all();
    __syncthreads();
    fixed_compute<D, P, SYS, T, B0, B1, B2, NTH, true>(I, t, s, tin, nullptr);
}

// Shared-memory layout of the mixed kernel: one tile buffer as large as the
// largest of the three shapes (cell blocks X0 x X1 for degree 1, Y0 x Y1 for
// degree 2, Z0 x Z1 for degree 3; FP32), then the look-back inflows.
template <int X0, int X1, int Y0, int Y1, int Z0, int Z1>
struct Mixed2D {
    using S1 = Shape<2, 1, kEuler, float, X0, X1, 1>;
    using S2 = Shape<2, 2, kEuler, float, Y0, Y1, 1>;
    using S3 = Shape<2, 3, kEuler, float, Z0, Z1, 1>;
    static constexpr size_t mx(size_t a, size_t b) { return a > b ? a : b; }
    static constexpr size_t TILE = (mx(S1::SMEM, mx(S2::SMEM, S3::SMEM)) + 15) / 16 * 16;
    static constexpr size_t TIN = mx(S1::TIN_BYTES, mx(S2::TIN_BYTES, S3::TIN_BYTES));
    static constexpr size_t SMEM = TILE + TIN;
};

// Persistent kernel over a work list of (degree << 24 | instance, tile)
// pairs covering every tile of every member: each tile runs the fixed-shape
// body of its degree, so one launch advances problems of degrees 1, 2 and 3
// (of any mesh size) by one step.  The host orders the list with the most
// expensive tiles first, so the launch ends on short tiles.
template <int NTH, int MINB, int X0, int X1, int Y0, int Y1, int Z0, int Z1>
__global__ void __launch_bounds__(NTH, MINB)
    step_kernel_mixed2d(const Inst* __restrict__ insts, const int2* __restrict__ work, int nwork)
{
    using MX = Mixed2D<X0, X1, Y0, Y1, Z0, Z1>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float* const s = reinterpret_cast<float*>(smem_raw);
    float* const tin = reinterpret_cast<float*>(smem_raw + MX::TILE);
    for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
        const int2 wk = work[w];
        const Inst& I = insts[wk.x & 0xffffff];
        const int deg = wk.x >> 24;
        if (deg == 1) fixed_tile_1buf<2, 1, kEuler, float, X0, X1, 1, NTH>(I, wk.y, s, tin);
        else if (deg == 2) fixed_tile_1buf<2, 2, kEuler, float, Y0, Y1, 1, NTH>(I, wk.y, s, tin);
        else fixed_tile_1buf<2, 3, kEuler, float, Z0, Z1, 1, NTH>(I, wk.y, s, tin);
    }
}

}  // namespace kin
