// kin_fixed.cuh -- the fused step kernel for a compile-time cell-block shape.
//
// Same computation as the generic kernel of kin_device.cuh (bulk loads,
// look-back inflow, downwind sweeps, relaxation, block summaries, bulk
// stores), specialised on the block extents B0 x B1 x B2 and the thread count
// NTH so that every loop has a constant trip count and every shared-memory
// offset is an immediate.  Differences in the schedule:
//   * shared memory rows and population slabs are padded (by a multiple of 16
//     bytes, which keeps bulk copies legal) with the padding that minimises
//     bank conflicts of the sweep and relaxation access patterns, chosen at
//     compile time;
//   * the threads are split in two halves, one per velocity sign, so each
//     warp sweeps lines of a single direction with no per-cell selects.
#pragma once

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
    static constexpr int M = SYS == kAdvection ? 1 : D + 2;
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

    static constexpr int RP = best_pad(true);
    static constexpr int PP = best_pad(false);
    static constexpr int RSTR = rstr(RP);
    static constexpr int PSTR = pstr(RP, PP);
    static constexpr int TILE = NPOP * PSTR;                        // elements per tile buffer
    static constexpr size_t SMEM = sizeof(T) * (size_t)TILE;
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

// One half of the threads handles the lines of velocity sign SGN of axis A;
// thread 'hid' of the half owns items hid, hid + HALF, ...  The look-back
// inflows of those items live in the registers tr[] (same item order).
template <int D, int P, int SYS, typename T, int B0, int B1, int B2, int NTH, int A, int SGN, int MODE>
__device__ __forceinline__ void fixed_lines(const Inst& I, int hid, int org0, int org1, int org2, int bidx,
                                            T* s, T* tr)
{
    using S = Shape<D, P, SYS, T, B0, B1, B2>;
    constexpr int NP = S::NP, M = S::M, HALF = NTH / 2;
    constexpr int LP = S::lines(A);
    constexpr int ITEMS = M * LP;                   // items of this sign
    constexpr int KPT = S::kpt(A, HALF);
    constexpr int BA = S::ext(A);
    constexpr int CST = S::cstep(S::RP, A);
    constexpr int NS = S::nstep(A);
    constexpr int DIR = 2 * A + SGN;

    if (MODE == 0) {
        // look-back inflows (before the tile's data has arrived)
#pragma unroll
        for (int k = 0; k < KPT; ++k) {
            const int it = hid + k * HALF;
            if (ITEMS % HALF != 0 && it >= ITEMS) break;
            const int v = it / LP, line = it % LP;
            const int pop = (2 * A + SGN) * M + v;
            tr[k] = chain_inflow<T>(I, A, SGN, bidx, pop, fixed_gline<D, NP, A, B0, B1>(I, line, org0, org1, org2));
        }
    } else if (MODE == 1) {
        T Pm[NP][NP], g[NP];
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            g[i] = coef_of(I, DIR, kOffG + i, T(0));
#pragma unroll
            for (int j = 0; j < NP; ++j) Pm[i][j] = coef_of(I, DIR, i * NP + j, T(0));
        }
#pragma unroll
        for (int k = 0; k < KPT; ++k) {
            const int it = hid + k * HALF;
            if (ITEMS % HALF != 0 && it >= ITEMS) break;
            const int v = it / LP, line = it % LP;
            const int pop = (2 * A + SGN) * M + v;
            const int base = S::line_base(S::RP, S::PP, A, pop, line);
            T t = tr[k];
#pragma unroll
            for (int cc = 0; cc < BA; ++cc) {
                T* p = s + base + (SGN == 0 ? cc : BA - 1 - cc) * CST;
                T u[NP], dlt[NP];
#pragma unroll
                for (int j = 0; j < NP; ++j) u[j] = p[j * NS];
#pragma unroll
                for (int i = 0; i < NP; ++i) {
                    T acc = Pm[i][0] * u[0];
#pragma unroll
                    for (int j = 1; j < NP; ++j) acc = fma(Pm[i][j], u[j], acc);
                    dlt[i] = fma(g[i], t, acc);
                }
                t = SGN == 0 ? u[NP - 1] + dlt[NP - 1] : u[0] + dlt[0];
#pragma unroll
                for (int i = 0; i < NP; ++i) p[i * NS] = fma(T(2), dlt[i], u[i]);
            }
        }
    } else {
        T prow[NP];
#pragma unroll
        for (int j = 0; j < NP; ++j) prow[j] = coef_of(I, DIR, kOffProw + j, T(0));
        const T rho = coef_of(I, DIR, kOffRho, T(0));
#pragma unroll
        for (int k = 0; k < KPT; ++k) {
            const int it = hid + k * HALF;
            if (ITEMS % HALF != 0 && it >= ITEMS) break;
            const int v = it / LP, line = it % LP;
            const int pop = (2 * A + SGN) * M + v;
            const int base = S::line_base(S::RP, S::PP, A, pop, line);
            T t = 0, last = 0;
#pragma unroll
            for (int cc = 0; cc < BA; ++cc) {
                const T* p = s + base + (SGN == 0 ? cc : BA - 1 - cc) * CST;
                T u[NP];
#pragma unroll
                for (int j = 0; j < NP; ++j) u[j] = p[j * NS];
                T acc = prow[0] * u[0];
#pragma unroll
                for (int j = 1; j < NP; ++j) acc = fma(prow[j], u[j], acc);
                t = fma(rho, t, acc);
                last = SGN == 0 ? u[NP - 1] : u[0];
            }
            write_summary<T>(I, A, SGN, bidx, pop, fixed_gline<D, NP, A, B0, B1>(I, line, org0, org1, org2), t,
                             last);
        }
    }
}

// MODE 0: look-back inflows, 1: transport sweeps, 2: block summaries.  Each
// sign half runs its own warps (HALF is a multiple of 32).
template <int D, int P, int SYS, typename T, int B0, int B1, int B2, int NTH, int MODE, int KM>
__device__ __forceinline__ void fixed_lines_all(const Inst& I, int org0, int org1, int org2, int bx, int by,
                                                int bz, T* s, T (&tr)[3][KM])
{
    const int tid = threadIdx.x;
    const int hid = tid < NTH / 2 ? tid : tid - NTH / 2;
    if (tid < NTH / 2) {
        fixed_lines<D, P, SYS, T, B0, B1, B2, NTH, 0, 0, MODE>(I, hid, org0, org1, org2, bx, s, tr[0]);
        if constexpr (D > 1) fixed_lines<D, P, SYS, T, B0, B1, B2, NTH, 1, 0, MODE>(I, hid, org0, org1, org2, by, s, tr[1]);
        if constexpr (D > 2) fixed_lines<D, P, SYS, T, B0, B1, B2, NTH, 2, 0, MODE>(I, hid, org0, org1, org2, bz, s, tr[2]);
    } else {
        fixed_lines<D, P, SYS, T, B0, B1, B2, NTH, 0, 1, MODE>(I, hid, org0, org1, org2, bx, s, tr[0]);
        if constexpr (D > 1) fixed_lines<D, P, SYS, T, B0, B1, B2, NTH, 1, 1, MODE>(I, hid, org0, org1, org2, by, s, tr[1]);
        if constexpr (D > 2) fixed_lines<D, P, SYS, T, B0, B1, B2, NTH, 2, 1, MODE>(I, hid, org0, org1, org2, bz, s, tr[2]);
    }
}

template <int D, int P, int SYS, typename T, int B0, int B1, int B2, int NTH>
__device__ __forceinline__ void fixed_relax(const Inst& I, T* s)
{
    using S = Shape<D, P, SYS, T, B0, B1, B2>;
    constexpr int M = S::M, NV = 2 * D, NPOP = S::NPOP;
    const T omega = T(I.omega);
    const bool two = I.omega == 2.0;
    const T inv2d = T(1.0 / (2.0 * D));
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
                const T base = W[v] * inv2d;
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

template <int D, int P, int SYS, typename T, int B0, int B1, int B2, bool STORE>
__device__ __forceinline__ void fixed_issue_copies(const Inst& I, int org0, int org1, int org2, T* s, uint64_t* bar)
{
    using S = Shape<D, P, SYS, T, B0, B1, B2>;
    constexpr int NCH = S::NPOP * S::NROWS;
    constexpr unsigned BYTES = (unsigned)(S::ROWLEN * sizeof(T));
    T* f = static_cast<T*>(I.f);
    const int lane = threadIdx.x;
    if (!STORE) {
        if (lane == 0) mbar_arrive_expect_tx(bar, (unsigned)NCH * BYTES + (I.debug_stall ? 16u : 0u));
        __syncwarp();
    }
#pragma unroll
    for (int k = 0; k < (NCH + 31) / 32; ++k) {
        const int ch = lane + 32 * k;
        if (NCH % 32 != 0 && ch >= NCH) break;
        const int pop = ch / S::NROWS, row = ch % S::NROWS;
        const int ly = row % B1, lz = row / B1;
        const long long g = (long long)pop * I.nodes
            + (((long long)(org2 + lz) * (D > 1 ? I.n[1] : 1) + (org1 + ly)) * I.n[0] + org0) * S::NN;
        T* sp = s + pop * S::PSTR + row * S::RSTR;
        if (STORE) bulk_s2g(f + g, sp, BYTES);
        else bulk_g2s(sp, f + g, BYTES, bar);
    }
    if (STORE) bulk_commit();
}

// One tile of the fixed-shape step: issue the bulk loads, fold the look-back
// inflows while they fly, wait (bounded), sweep, relax, write the summaries
// and issue the bulk stores.  'i' counts the tiles this thread block has
// processed (mbarrier phase).  Returns false if the bounded wait gave up.
template <int D, int P, int SYS, typename T, int B0, int B1, int B2, int NTH, int KM>
__device__ __forceinline__ bool fixed_tile(const Inst& I, int t, int i, T* s, uint64_t* bar, int* flag,
                                           T (&tr)[3][KM])
{
    const int tid = threadIdx.x;
    const bool warp0 = tid < 32;
    const TileXYZ c = tile_xyz(I, t);
    const int org0 = c.bx * B0, org1 = c.by * B1, org2 = c.bz * B2;
    if (warp0) {
        if (i > 0) {
            bulk_wait_read();   // previous tile's stores have read the buffer
            __syncwarp();
        }
        fixed_issue_copies<D, P, SYS, T, B0, B1, B2, false>(I, org0, org1, org2, s, bar);
    }
    if (I.mode == 0) fixed_lines_all<D, P, SYS, T, B0, B1, B2, NTH, 0, KM>(I, org0, org1, org2, c.bx, c.by, c.bz, s, tr);
    if (tid == 0) *flag = mbar_wait_bounded(bar, i & 1, I.wait_cycles) ? 1 : 0;
    __syncthreads();
    if (*flag == 0) {
        // give up: report, wait (bounded) for the copies still in flight
        if (tid == 0) {
            if (I.err) atomicOr(I.err, kErrLoadTimeout);
            mbar_wait_bounded(bar, i & 1, I.wait_cycles);
        }
        if (warp0) bulk_wait_all();
        return false;
    }
    (void)mbar_try_wait(bar, i & 1);
    if (I.mode == 0) {
        fixed_lines_all<D, P, SYS, T, B0, B1, B2, NTH, 1, KM>(I, org0, org1, org2, c.bx, c.by, c.bz, s, tr);
        __syncthreads();
        fixed_relax<D, P, SYS, T, B0, B1, B2, NTH>(I, s);
        __syncthreads();
    }
    fixed_lines_all<D, P, SYS, T, B0, B1, B2, NTH, 2, KM>(I, org0, org1, org2, c.bx, c.by, c.bz, s, tr);
    if (I.mode == 0) fence_proxy_async_smem();
    __syncthreads();
    if (I.mode == 0 && warp0) fixed_issue_copies<D, P, SYS, T, B0, B1, B2, true>(I, org0, org1, org2, s, bar);
    return true;
}

// Fixed-shape step kernel: one tile per loop iteration, one shared-memory
// stage; the grid is persistent (blocks walk tiles blockIdx.x + k gridDim.x).
template <int D, int P, int SYS, typename T, int B0, int B1, int B2, int NTH, int MINB>
__global__ void __launch_bounds__(NTH, MINB) step_kernel_fixed(const __grid_constant__ Inst I)
{
    using S = Shape<D, P, SYS, T, B0, B1, B2>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ int flag;
    T* s = reinterpret_cast<T*>(smem_raw);
    constexpr int KM = S::kpt_max(NTH / 2);
    T tr[3][KM];      // look-back inflows of this thread's lines
    const int ntiles = I.nblk[0] * I.nblk[1] * I.nblk[2];
    int t = blockIdx.x;
    if (t >= ntiles) return;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    for (int i = 0; t < ntiles; ++i, t += gridDim.x)
        if (!fixed_tile<D, P, SYS, T, B0, B1, B2, NTH, KM>(I, t, i, s, &bar, &flag, tr)) return;
    if (threadIdx.x < 32) bulk_wait_all();
}

// Batched fixed-shape step kernel: the thread blocks walk a work list of
// (instance, tile) pairs over several independent problems of the same
// kernel type; each instance's launch record is copied into shared memory
// when a block moves to a tile of another instance.
template <int D, int P, int SYS, typename T, int B0, int B1, int B2, int NTH, int MINB>
__global__ void __launch_bounds__(NTH, MINB)
    step_kernel_fixed_batch(const Inst* __restrict__ insts, const int2* __restrict__ work, int nwork)
{
    using S = Shape<D, P, SYS, T, B0, B1, B2>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ int flag;
    __shared__ __align__(16) Inst Ish;
    T* s = reinterpret_cast<T*>(smem_raw);
    constexpr int KM = S::kpt_max(NTH / 2);
    T tr[3][KM];
    int w = blockIdx.x;
    if (w >= nwork) return;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    int have = -1;
    for (int i = 0; w < nwork; ++i, w += gridDim.x) {
        const int2 wk = work[w];
        if (wk.x != have) {
            // warp 0 may still read the record while issuing the previous tile's stores
            __syncthreads();
            const int4* src = reinterpret_cast<const int4*>(insts + wk.x);
            int4* dst = reinterpret_cast<int4*>(&Ish);
            for (int k = threadIdx.x; k < (int)(sizeof(Inst) / 16); k += NTH) dst[k] = src[k];
            have = wk.x;
        }
        __syncthreads();
        if (!fixed_tile<D, P, SYS, T, B0, B1, B2, NTH, KM>(Ish, wk.y, i, s, &bar, &flag, tr)) return;
    }
    if (threadIdx.x < 32) bulk_wait_all();
}

}  // namespace kin
