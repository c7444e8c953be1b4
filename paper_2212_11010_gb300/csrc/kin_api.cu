// kin_api.cu -- the C ABI (include/kin.h): argument validation, device
// memory, launch configuration and stream ordering.  Every step of the
// method runs in the kernels of kin_device.cuh / kin_aux.cu.
#include "../../include/kin.h"
#include "kin_aux.h"
#include "kin_device.cuh"

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdarg>
#include <cstdio>
#include <cmath>
#include <climits>
#include <cstring>
#include <string>
#include <vector>

using namespace kin;

struct kin_ctx {
    // problem
    int dim = 1, n[3] = {1, 1, 1}, degree = 1, system = 0, m = 1, nvel = 2, npop = 2, NP = 2, NN = 2;
    double lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1}, h[3] = {1, 1, 1};
    double lambda = 1, gamma = 1.4, adv[3] = {0, 0, 0}, omega = 2, dt = 0, sigma = 0;
    // inflow boundaries: per axis flag, the value across the boundary face
    // each population enters through, and which faces have a state
    int inflow[3] = {0, 0, 0};
    double bnd[kMaxPop] = {};
    double bnd_host[kMaxPop] = {};    // the values in the context precision, staged for the device copy
    void* bnd_dev = nullptr;          // T[npop] on the device, read by the look-back
    bool bnd_set[3][2] = {{false, false}, {false, false}, {false, false}};
    int tiles[3] = {1, 1, 1}, L[3] = {1, 1, 1}, iters = 3, precision = KIN_FP64;
    int B[3] = {1, 1, 1}, nblk[3] = {1, 1, 1}, nb[3] = {1, 1, 1};
    size_t cells = 0, nodes = 0, sig_stride = 0, raw_stride = 0, esize = 8;
    double coef_host[6][kCoefStride] = {};   // FP64 block-inverse records (device-computed)
    // runtime
    cudaStream_t stream = nullptr;
    kin_alloc_fn alloc = nullptr;
    kin_free_fn dealloc = nullptr;
    void* alloc_user = nullptr;
    size_t budget = 0, bytes_held = 0;
    std::vector<std::pair<void*, size_t>> blocks;
    void* f = nullptr;
    void* sig[2] = {nullptr, nullptr};
    void* raw[2] = {nullptr, nullptr};
    int cur = 0;
    double* c64 = nullptr;
    void* coef = nullptr;
    double* gll = nullptr;
    double* Wbuf = nullptr;
    double* partial = nullptr;
    double* result = nullptr;
    int* errword = nullptr;
    double wait_timeout_s = 1.0;
    int debug_flags = 0;
    StepKernel kfn = nullptr;
    int smem = 0, grid = 0, stages = 1, threads = kThreads;
    int want_threads = 0, want_stages = 0;
    bool fixed = false;                    // compile-time block shape kernel in use
    // d + 1 velocity sets
    bool simplex = false;
    int vsgn[4][3] = {};
    double minv[16] = {};
    double* sxc64 = nullptr;
    double* sxwork = nullptr;
    void* sxtr[2][3] = {};
    std::vector<double> sx_hrec;      // FP64 records [velocity][sx_stride], passed in the sweep parameters
    SxPlan sx_plan = {};
    int sx_stride = 0;
    // tetrahedral meshes
    bool tet = false;
    int nsub = 0;
    int tsgn[4][3] = {};
    void* tcoef = nullptr;            // T records [velocity][cell][kTetRec]
    int* torder = nullptr;            // [velocity][cells]
    int* tlstart = nullptr;           // [velocity][nsub + 1]
    int* tbounds = nullptr;           // level boundaries
    int* tfref = nullptr;             // [velocity][position][4] packed inflow face references
    void* titer[2] = {nullptr, nullptr};   // subdomain iterates
    std::vector<double> tvol;         // host: cell volumes, for the mass diagnostic
    bool have_state = false;
    bool sum_stale = false;           // f was replaced without recomputing the interface summaries
    cudaEvent_t after_batch = nullptr;   // recorded on a batch's stream after its last step of this context
    bool wait_batch = false;          // the context's next work must wait for after_batch
    long long steps_done = 0;
    bool poisoned = false;
    std::string err;
};

static thread_local std::string g_create_error = "no error";

static kin_status fail(kin_ctx* c, kin_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) {
        c->err = buf;
        if (st == KIN_ECUDA || st == KIN_ETIMEOUT) c->poisoned = true;
    } else {
        g_create_error = buf;
    }
    return st;
}

#define KIN_CUDA(c, call)                                                              \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess)                                                         \
            return fail((c), KIN_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

static kin_status dev_alloc(kin_ctx* c, size_t bytes, void** out)
{
    *out = nullptr;
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~size_t(255);
    if (c->budget && c->bytes_held + bytes > c->budget)
        return fail(c, KIN_EBUDGET, "device memory budget of %zu bytes exceeded (%zu held, %zu asked)",
                    c->budget, c->bytes_held, bytes);
    void* p = nullptr;
    if (c->alloc) {
        p = c->alloc(bytes, (void*)c->stream, c->alloc_user);
        if (!p) return fail(c, KIN_ENOMEM, "allocator hook returned NULL for %zu bytes", bytes);
    } else {
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(c, KIN_ENOMEM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
        }
    }
    c->blocks.push_back({p, bytes});
    c->bytes_held += bytes;
    *out = p;
    return KIN_OK;
}

static void release_all(kin_ctx* c)
{
    if (c->after_batch) cudaEventDestroy(c->after_batch);
    c->after_batch = nullptr;
    for (auto& b : c->blocks) {
        if (c->dealloc) c->dealloc(b.first, b.second, (void*)c->stream, c->alloc_user);
        else cudaFree(b.first);
    }
    c->blocks.clear();
    c->bytes_held = 0;
}

static StepKernel pick_kernel(int dim, int degree, int system, int prec)
{
    switch (dim) {
    case 1: return step_kernel_d1(degree, system, prec);
    case 2: return step_kernel_d2(degree, system, prec);
    case 3: return step_kernel_d3(degree, system, prec);
    default: return nullptr;
    }
}

static size_t block_smem(const kin_ctx* c, const int B[3])
{
    return (size_t)c->npop * B[0] * B[1] * B[2] * c->NN * c->esize;
}

// Largest divisor of L that is smaller than b (at least 1).
static int next_divisor_below(int L, int b)
{
    for (int d = b - 1; d >= 1; --d)
        if (L % d == 0) return d;
    return 1;
}

// Default cell block: start from the whole subdomain and shrink the longest
// extent (z before y before x on ties, to keep the contiguous x rows long)
// until one tile fits the shared-memory target -- two tiles then fit twice
// per SM -- and the grid has enough tiles to fill 152 SMs twice.
static void choose_block(const kin_ctx* c, int B[3])
{
    // a block shape with a compiled fixed-shape kernel, if one fits the subdomains
    int shapes[4][3];
    const int ns = fixed_shapes(c->dim, c->degree, c->system, c->precision, shapes);
    for (int k = 0; k < ns; ++k) {
        bool fits = true;
        for (int a = 0; a < 3; ++a)
            if (c->L[a] % shapes[k][a]) fits = false;
        if (fits) {
            for (int a = 0; a < 3; ++a) B[a] = shapes[k][a];
            return;
        }
    }
    const size_t target = 48 * 1024;
    for (int a = 0; a < 3; ++a) B[a] = c->L[a];
    auto grid_of = [&](const int* b) {
        long long g = 1;
        for (int a = 0; a < c->dim; ++a) g *= c->n[a] / b[a];
        return g;
    };
    for (int guard = 0; guard < 64; ++guard) {
        bool too_big = block_smem(c, B) > target;
        bool too_few = grid_of(B) < 2 * 152;
        if (!too_big && !too_few) break;
        int best = -1;
        for (int a = c->dim - 1; a >= 0; --a)
            if (B[a] > 1 && (best < 0 || B[a] > B[best])) best = a;
        if (best < 0) break;
        if (!too_big && B[best] <= 4) break;     // keep lines reasonably long
        B[best] = next_divisor_below(c->L[best], B[best]);
    }
}

// Bulk copies need every row of a cell block to start on a 16-byte
// boundary and to span a multiple of 16 bytes.
static bool rows_are_16b_aligned(const kin_ctx* c)
{
    const size_t rowb = (size_t)c->B[0] * c->NN * c->esize;
    const size_t popb = c->nodes * c->esize;
    const size_t lineb = (size_t)c->n[0] * c->NN * c->esize;
    return rowb % 16 == 0 && popb % 16 == 0 && lineb % 16 == 0 && ((uintptr_t)c->f % 16) == 0;
}

static Inst make_inst(const kin_ctx* c, int mode)
{
    Inst I;
    memset(&I, 0, sizeof I);
    I.f = c->f;
    I.sig_in = c->sig[c->cur];
    I.raw_in = c->raw[c->cur];
    I.sig_out = c->sig[c->cur ^ 1];
    I.raw_out = c->raw[c->cur ^ 1];
    I.err = c->errword;
    I.nodes = (long long)c->nodes;
    I.sig_stride = (long long)c->sig_stride;
    I.raw_stride = (long long)c->raw_stride;
    for (int d = 0; d < 6; ++d)
        for (int k = 0; k < kCoefStride; ++k) {
            I.cd[d][k] = c->coef_host[d][k];
            I.cf[d][k] = (float)c->coef_host[d][k];
        }
    I.wait_cycles = (long long)((c->wait_timeout_s > 0 ? c->wait_timeout_s : 1.0) * 2.2e9);
    long long tn = 1;
    for (int a = 1; a < c->dim; ++a) tn *= c->NP;
    const int bcells = c->B[0] * c->B[1] * c->B[2];
    for (int a = 0; a < 3; ++a) {
        I.n[a] = c->n[a];
        I.B[a] = c->B[a];
        I.nblk[a] = c->nblk[a];
        I.nb[a] = c->nb[a];
        I.NS[a] = c->tiles[a];
        I.adv[a] = c->adv[a];
        I.ax[a].lines = make_fastdiv((unsigned)((bcells / c->B[a]) * tn));
        I.ax[a].e1 = make_fastdiv((unsigned)(a == 0 ? c->B[1] : c->B[0]));
        I.ax[a].glines = (long long)(c->cells / c->n[a]) * tn;
    }
    I.fd_nblk0 = make_fastdiv((unsigned)c->nblk[0]);
    I.fd_nblk01 = make_fastdiv((unsigned)(c->nblk[0] * c->nblk[1]));
    for (int a = 0; a < 3; ++a) I.fd_nb[a] = make_fastdiv((unsigned)c->nb[a]);
    I.fd_nrows = make_fastdiv((unsigned)(c->B[1] * c->B[2]));
    I.fd_B1 = make_fastdiv((unsigned)c->B[1]);
    I.fd_rowlen = make_fastdiv((unsigned)(c->B[0] * c->NN));
    I.iters = c->iters;
    I.mode = mode;
    I.tma = rows_are_16b_aligned(c) ? 1 : 0;
    I.stages = c->stages;
    I.debug_stall = (c->debug_flags & KIN_DEBUG_STALL_LOAD) ? 1 : 0;
    I.lambda = c->lambda;
    I.gamma = c->gamma;
    I.omega = c->omega;
    I.mu = c->system == KIN_MAXWELL ? (1.0 - 0.5 * c->sigma * c->dt) / (1.0 + 0.5 * c->sigma * c->dt) : 1.0;
    for (int a = 0; a < 3; ++a) I.inflow[a] = c->inflow[a];
    I.bnd = c->bnd_dev;
    // look-back depth per direction: the fewest upstream blocks d with
    // |rho^B|^d <= tol, tol well below the rounding of the precision
    const double tol = c->esize == 4 ? std::ldexp(1.0, -36) : std::ldexp(1.0, -72);
    for (int d = 0; d < 6; ++d) {
        const double rb = std::fabs(c->coef_host[d][kOffRhoB]);
        int depth = 1 << 30;                                   // no truncation
        if (rb < 1.0) depth = rb == 0.0 ? 1 : std::max(1, (int)std::ceil(std::log(tol) / std::log(rb)));
        I.lbdepth[d] = depth;
    }
    return I;
}

// Status of a device error word value h.
static kin_status errword_status(kin_ctx* c, int h)
{
    if (h & kErrLoadTimeout)
        return fail(c, KIN_ETIMEOUT, "a thread block gave up waiting for its bulk loads (bounded wait ran out)");
    if (h) return fail(c, KIN_ETIMEOUT, "device error word 0x%x", h);
    return KIN_OK;
}

// Read the device error word (after the stream has been synchronised).
static kin_status check_errword(kin_ctx* c)
{
    int h = 0;
    KIN_CUDA(c, cudaMemcpyAsync(&h, c->errword, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    KIN_CUDA(c, cudaStreamSynchronize(c->stream));
    return errword_status(c, h);
}

// Work items of one tile: (population, line) pairs per axis and nodes.
static void tile_work(const kin_ctx* c, long long items[3], long long* nodes)
{
    const long long bcells = (long long)c->B[0] * c->B[1] * c->B[2];
    long long tn = 1;
    for (int a = 1; a < c->dim; ++a) tn *= c->NP;
    for (int a = 0; a < 3; ++a) items[a] = a < c->dim ? 2LL * c->m * (bcells / c->B[a]) * tn : 0;
    *nodes = bcells * c->NN;
}

// Threads per block: the multiple of 32 in [128, 256] that leaves the fewest
// idle thread-slots over the phases of a tile (per-axis line items twice --
// transport and summaries -- and the relaxation nodes); ties go to more threads.
static int choose_threads(const kin_ctx* c)
{
    long long items[3], nodes;
    tile_work(c, items, &nodes);
    int best = kThreads;
    long long best_cost = -1;
    for (int nth = kThreads; nth >= 128; nth -= 32) {
        long long cost = ((nodes + nth - 1) / nth) * nth;
        for (int a = 0; a < c->dim; ++a) cost += 2 * ((items[a] + nth - 1) / nth) * nth;
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best = nth;
        }
    }
    return best;
}

// Launch shape: threads, shared-memory stages (two when rows move by bulk
// copies and two tiles fit), carve-out, resident blocks per SM and the
// persistent grid.  Dynamic shared memory = stages x tile + inflow traces.
static cudaError_t configure_launch(kin_ctx* c)
{
    const size_t tile = block_smem(c, c->B);
    long long items[3], nodes;
    tile_work(c, items, &nodes);
    const size_t tin = ((size_t)(items[0] + items[1] + items[2]) * c->esize + 15) & ~size_t(15);
    const bool tma = rows_are_16b_aligned(c);
    // fixed-shape kernel: same result, compile-time shape (bulk copies, one stage)
    FixedKernel fk{nullptr, nullptr, 0, 0};
    int fstages = 1;
    if (c->dim >= 2)
        fstages = c->want_stages ? c->want_stages
                                 : fixed_default_stages(c->dim, c->degree, c->system, c->precision, c->B);
    if (c->dim == 2) fk = fixed_kernel_d2(c->degree, c->system, c->precision, c->B, fstages);
    if (c->dim == 3) fk = fixed_kernel_d3(c->degree, c->system, c->precision, c->B, fstages);
    // (the bounded-wait test hook lives in the bulk-copy path of the generic kernel)
    // (the fixed kernels index the block summaries with 32-bit offsets)
    const bool small_summaries = (double)c->sig_stride * c->npop < 2147483647.0;
    c->fixed = fk.fn && fk.smem <= 227 * 1024 && tma && small_summaries &&
               (c->want_threads == 0 || c->want_threads == fk.threads) &&
               !(c->debug_flags & KIN_DEBUG_STALL_LOAD);
    if (c->fixed) {
        c->kfn = fk.fn;
        c->threads = fk.threads;
        c->stages = fstages;
        c->smem = (int)fk.smem;
    } else {
        c->kfn = pick_kernel(c->dim, c->degree, c->system, c->precision);
        c->threads = c->want_threads ? c->want_threads : choose_threads(c);
        if (!tma) c->stages = 1;
        else if (c->want_stages) c->stages = c->want_stages;
        else c->stages = 1;
        if (c->stages * tile + tin > 227 * 1024) c->stages = 1;
        c->smem = (int)(c->stages * tile + tin);
    }
    cudaError_t e = cudaSuccess;
    if (c->smem > 48 * 1024)
        e = cudaFuncSetAttribute((const void*)c->kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, c->smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute((const void*)c->kfn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    int dev = 0, nsm = 1, occ = 1;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void*)c->kfn, c->threads, c->smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
    const long long ntiles = (long long)c->nblk[0] * c->nblk[1] * c->nblk[2];
    c->grid = (int)std::min<long long>(ntiles, (long long)occ * nsm);
    return cudaSuccess;
}

// Launch of the fused kernel: mode 0 = one full step (reads the summaries
// of buffer cur, writes those of the new state to cur ^ 1 and flips cur);
// mode 1 = block summaries of the current state only, written straight into
// buffer cur (mode 1 reads no summaries), so cur stays: a state set through
// kin_set_state / kin_set_kinetic keeps a member's batch valid.
static kin_status launch_step_on(kin_ctx* c, int mode, cudaStream_t st)
{
    Inst I = make_inst(c, mode);
    if (mode == 1) {
        I.sig_out = c->sig[c->cur];
        I.raw_out = c->raw[c->cur];
    }
    void* args[] = {&I};
    KIN_CUDA(c, cudaLaunchKernel((const void*)c->kfn, dim3(c->grid), dim3(c->threads), args,
                                 (size_t)c->smem, st));
    if (mode == 0) c->cur ^= 1;
    return KIN_OK;
}

static kin_status launch_step(kin_ctx* c, int mode) { return launch_step_on(c, mode, c->stream); }

static PointArgs point_args(const kin_ctx* c)
{
    PointArgs p;
    memset(&p, 0, sizeof p);
    p.dim = c->dim;
    p.degree = c->degree;
    p.m = c->m;
    p.system = c->system;
    p.nvel = c->nvel;
    p.nodes = (long long)c->nodes;
    p.lambda = c->lambda;
    p.gamma = c->gamma;
    for (int a = 0; a < 3; ++a) {
        p.adv[a] = c->adv[a];
        p.h[a] = c->h[a];
    }
    return p;
}

static kin_status check_usable(const kin_ctx* c)
{
    if (!c) return KIN_EINVAL;
    if (c->poisoned) return KIN_ESTATE;
    return KIN_OK;
}

// A batch step runs a context's work on the batch's stream.  The context's
// own stream (or a stream the caller names for a copy) waits for it only
// when the context is next used, so that a stream several contexts share is
// not held up by a batch step of other contexts.
static cudaError_t order_after_batch(kin_ctx* c, cudaStream_t s)
{
    if (!c->wait_batch) return cudaSuccess;
    const cudaError_t e = cudaStreamWaitEvent(s, c->after_batch, 0);
    if (e == cudaSuccess && s == c->stream) c->wait_batch = false;
    return e;
}

// ---- d + 1 velocity sets: launch arguments and one step ----
static SxArgs sx_args(const kin_ctx* c)
{
    SxArgs S;
    memset(&S, 0, sizeof S);
    S.f = c->f;
    S.nodes = (long long)c->nodes;
    long long tn = 1;
    for (int a = 1; a < c->dim; ++a) tn *= c->NP;
    for (int a = 0; a < 3; ++a) {
        S.n[a] = c->n[a];
        S.L[a] = c->L[a];
        S.NS[a] = c->tiles[a];
        S.glines[a] = a < c->dim ? (long long)(c->cells / c->n[a]) * tn : 0;
        S.adv[a] = c->adv[a];
    }
    for (int k = 0; k < 4; ++k)
        for (int a = 0; a < 3; ++a) S.vsgn[k][a] = c->vsgn[k][a];
    S.dim = c->dim;
    S.degree = c->degree;
    S.nn = c->NN;
    S.m = c->m;
    S.nvel = c->nvel;
    S.npop = c->npop;
    S.system = c->system;
    S.omega = c->omega;
    S.gamma = c->gamma;
    for (int i = 0; i < 16; ++i) S.minv[i] = c->minv[i];
    long long total = 0;
    for (int pop = 0; pop < c->npop; ++pop)
        for (int a = 0; a < c->dim; ++a)
            if (c->vsgn[pop / c->m][a] != 0) total += (long long)c->tiles[a] * S.glines[a];
    S.trace_total = total;
    return S;
}

// One step S(dt) for a d + 1 velocity set: K sweeps, then the relaxation.
// Iterate 1 reads its interface inflow from f^n directly; with K = 1 the
// sweep writes f^{n+1} in place, so a trace pass copies iterate 0 first.
static kin_status sx_step(kin_ctx* c)
{
    SxArgs S = sx_args(c);
    const int prec = c->precision == KIN_FP32;
    if (c->iters == 1) {
        for (int a = 0; a < 3; ++a) S.tr_out[a] = c->sxtr[0][a];
        KIN_CUDA(c, sx_launch_trace0(S, prec, c->stream));
    }
    for (int it = 1; it <= c->iters; ++it) {
        for (int a = 0; a < 3; ++a) {
            S.tr_in[a] = c->sxtr[(it - 1) & 1][a];
            S.tr_out[a] = c->sxtr[it & 1][a];
        }
        S.from_f = it == 1 && c->iters > 1;
        S.final_iter = it == c->iters;
        KIN_CUDA(c, sx_launch_sweep(S, prec, c->sx_hrec.data(), c->sx_stride, c->sx_plan, c->stream));
    }
    KIN_CUDA(c, sx_launch_relax(S, prec, c->stream));
    return KIN_OK;
}

// ---- tetrahedral meshes: launch arguments and one step ----
static TetArgs tet_args(const kin_ctx* c)
{
    TetArgs a;
    memset(&a, 0, sizeof a);
    a.ncells = (int)c->cells;
    a.nvel = c->nvel;
    a.m = c->m;
    a.npop = c->npop;
    a.nsub = c->nsub;
    a.system = c->system;
    a.velset = c->simplex ? 1 : 0;
    a.nodes = (long long)c->nodes;
    a.coef = c->tcoef;
    a.order = c->torder;
    a.lstart = c->tlstart;
    a.bounds = c->tbounds;
    a.fref = c->tfref;
    a.f = c->f;
    a.lambda = c->lambda;
    a.gamma = c->gamma;
    a.omega = c->omega;
    a.mu = c->system == KIN_MAXWELL ? (1.0 - 0.5 * c->sigma * c->dt) / (1.0 + 0.5 * c->sigma * c->dt) : 1.0;
    for (int i = 0; i < 3; ++i) a.adv[i] = c->adv[i];
    for (int k = 0; k < 4; ++k)
        for (int i = 0; i < 3; ++i) a.sgn[k][i] = c->tsgn[k][i];
    return a;
}

// One step S(dt) on a tetrahedral mesh: K sweeps (iterate p in titer[p & 1],
// iterate 0 = f^n), then the Crank-Nicolson extrapolation with the
// relaxation.
static kin_status tet_step(kin_ctx* c)
{
    const TetArgs a = tet_args(c);
    const int prec = c->precision == KIN_FP32;
    for (int p = 1; p <= c->iters; ++p) {
        const void* prev = p == 1 ? c->f : c->titer[(p - 1) & 1];
        KIN_CUDA(c, tet_launch_sweep(a, prev, c->titer[p & 1], prec, c->stream));
    }
    KIN_CUDA(c, tet_launch_relax(a, c->titer[c->iters & 1], prec, c->stream));
    return KIN_OK;
}

extern "C" {

kin_status kin_create(const kin_mesh* mesh, const kin_model* model, int degree, double dt,
                      const kin_opts* opts, kin_ctx** out)
{
    if (!out) return fail(nullptr, KIN_EINVAL, "out is NULL");
    *out = nullptr;
    if (!mesh || !model || !opts) return fail(nullptr, KIN_EINVAL, "mesh, model and opts are required");
    if (mesh->dim < 1 || mesh->dim > 3) return fail(nullptr, KIN_EINVAL, "dim must be 1..3");
    if (degree < 1 || degree > 3) return fail(nullptr, KIN_EINVAL, "degree must be 1..3");
    if (model->system != KIN_ADVECTION && model->system != KIN_EULER && model->system != KIN_MAXWELL)
        return fail(nullptr, KIN_EINVAL, "unknown system %d", model->system);
    if (model->system == KIN_MAXWELL && (mesh->dim != 3 || model->velset != KIN_D3Q6))
        return fail(nullptr, KIN_EINVAL, "Maxwell's equations need dim 3 and the D3Q6 velocity set");
    if (model->system == KIN_MAXWELL && !(model->sigma >= 0.0))
        return fail(nullptr, KIN_EINVAL, "the conductivity sigma must be >= 0");
    const bool simplex = (model->velset == KIN_D2Q3 && mesh->dim == 2) ||
                         (model->velset == KIN_D3Q4 && mesh->dim == 3);
    for (int a = 0; a < 3; ++a) {
        if (mesh->inflow[a] != 0 && mesh->inflow[a] != 1)
            return fail(nullptr, KIN_EINVAL, "inflow[%d] must be 0 or 1", a);
        if (mesh->inflow[a] && (a >= mesh->dim || simplex))
            return fail(nullptr, KIN_EINVAL, "inflow boundaries need an axis < dim and an axis velocity set");
    }
    if (model->velset != mesh->dim && !simplex)
        return fail(nullptr, KIN_EINVAL, "velocity set %d does not match dim %d", model->velset, mesh->dim);
    if (simplex && (degree > (mesh->dim == 3 ? 2 : 3)))
        return fail(nullptr, KIN_EINVAL, "the d+1 velocity sets support degree <= %d in %dD",
                    mesh->dim == 3 ? 2 : 3, mesh->dim);
    if (!(model->lambda > 0) || !(dt > 0))
        return fail(nullptr, KIN_EINVAL, "lambda and dt must be positive");
    if (!(model->omega >= 1.0 && model->omega <= 2.0))
        return fail(nullptr, KIN_EINVAL, "omega must lie in [1, 2]");
    if (model->system == KIN_EULER && !(model->gamma > 1.0))
        return fail(nullptr, KIN_EINVAL, "gamma must exceed 1");
    if (opts->iters < 1) return fail(nullptr, KIN_EINVAL, "iters must be >= 1");
    if (opts->precision != KIN_FP64 && opts->precision != KIN_FP32)
        return fail(nullptr, KIN_EINVAL, "unknown precision %d", opts->precision);
    if ((opts->alloc == nullptr) != (opts->free == nullptr))
        return fail(nullptr, KIN_EINVAL, "alloc and free hooks must be given together");
    if (opts->threads != 0 && (opts->threads < 32 || opts->threads > kThreads || opts->threads % 32))
        return fail(nullptr, KIN_EINVAL, "threads must be 0 or a multiple of 32 in [32, %d]", kThreads);
    if (opts->stages < 0 || opts->stages > 2) return fail(nullptr, KIN_EINVAL, "stages must be 0, 1 or 2");

    kin_ctx* c = new (std::nothrow) kin_ctx();
    if (!c) return fail(nullptr, KIN_ENOMEM, "host allocation failed");
    c->dim = mesh->dim;
    c->degree = degree;
    c->system = model->system;
    c->m = model->system == KIN_MAXWELL ? 6 : (model->system == KIN_EULER ? mesh->dim + 2 : 1);
    c->sigma = model->sigma;
    for (int a = 0; a < 3; ++a) c->inflow[a] = mesh->inflow[a];
    c->simplex = simplex;
    c->nvel = simplex ? mesh->dim + 1 : 2 * mesh->dim;
    c->npop = c->nvel * c->m;
    c->NP = degree + 1;
    c->NN = 1;
    for (int a = 0; a < c->dim; ++a) c->NN *= c->NP;
    c->lambda = model->lambda;
    c->gamma = model->gamma;
    c->omega = model->omega;
    c->dt = dt;
    c->iters = opts->iters;
    c->precision = opts->precision;
    c->esize = opts->precision == KIN_FP32 ? 4 : 8;
    c->stream = (cudaStream_t)opts->stream;
    c->alloc = opts->alloc;
    c->dealloc = opts->free;
    c->alloc_user = opts->alloc_user;
    c->budget = opts->mem_budget;
    c->wait_timeout_s = opts->wait_timeout_s;
    c->debug_flags = opts->debug_flags;
    c->want_threads = opts->threads;
    c->want_stages = opts->stages;
    c->cells = 1;
    for (int a = 0; a < 3; ++a) {
        c->adv[a] = model->adv[a];
        if (a < c->dim) {
            if (mesh->n[a] < 1 || !(mesh->hi[a] > mesh->lo[a])) {
                delete c;
                return fail(nullptr, KIN_EINVAL, "axis %d: need n >= 1 and hi > lo", a);
            }
            if (opts->tiles[a] < 1 || mesh->n[a] % opts->tiles[a]) {
                delete c;
                return fail(nullptr, KIN_EINVAL, "axis %d: tiles %d must divide n %d", a,
                            opts->tiles[a], mesh->n[a]);
            }
            c->n[a] = mesh->n[a];
            c->lo[a] = mesh->lo[a];
            c->hi[a] = mesh->hi[a];
            c->h[a] = (mesh->hi[a] - mesh->lo[a]) / mesh->n[a];
            c->tiles[a] = opts->tiles[a];
            c->L[a] = c->n[a] / c->tiles[a];
        } else {
            if (mesh->n[a] > 1) {
                delete c;
                return fail(nullptr, KIN_EINVAL, "axis %d beyond dim must have n = 1", a);
            }
            c->n[a] = 1;
            c->tiles[a] = 1;
            c->L[a] = 1;
        }
        c->cells *= c->n[a];
    }
    c->nodes = c->cells * c->NN;

    if (c->simplex) {
        // signs of the velocity components (D2Q3: 0, 120, 240 degrees; D3Q4 diagonals)
        static const int s2[3][3] = {{1, 0, 0}, {-1, 1, 0}, {-1, -1, 0}};
        static const int s3[4][3] = {{1, 1, 1}, {1, -1, -1}, {-1, 1, -1}, {-1, -1, 1}};
        for (int k = 0; k < c->nvel; ++k)
            for (int a = 0; a < 3; ++a) c->vsgn[k][a] = c->dim == 2 ? s2[k][a] : s3[k][a];
        size_t tn = 1;
        for (int a = 1; a < c->dim; ++a) tn *= c->NP;
        c->sx_stride = c->NN * c->NN + c->NN + c->dim * (int)tn;
        // sweep lanes: the columns of a subdomain along its stepping axis
        if (c->cells > (size_t)INT_MAX || !sx_sweep_shape(sx_args(c), c->precision == KIN_FP32, &c->sx_plan)) {
            const int lanes = c->dim == 2 ? std::max(c->L[0], c->L[1]) : c->L[0] * c->L[1];
            delete c;
            return fail(nullptr, KIN_EINVAL,
                        "a subdomain has %d columns along its sweep axis: at most 1024, whose sweep state fits "
                        "227 KB of shared memory (and at most 2^31 - 1 cells); use more tiles", lanes);
        }
        for (int a = 0; a < 3; ++a) {
            c->B[a] = c->L[a];
            c->nblk[a] = c->tiles[a];
            c->nb[a] = 1;
        }
        kin_status st;
        void* p;
#define ALLOC(dst, bytes)                                                 \
    do {                                                                  \
        st = dev_alloc(c, (bytes), &p);                                   \
        if (st != KIN_OK) {                                               \
            g_create_error = c->err;                                      \
            release_all(c);                                               \
            delete c;                                                     \
            return st;                                                    \
        }                                                                 \
        dst = (decltype(dst))p;                                           \
    } while (0)
        ALLOC(c->f, c->nodes * c->npop * c->esize);
        for (int i = 0; i < 2; ++i)
            for (int a = 0; a < c->dim; ++a)
                ALLOC(c->sxtr[i][a], (size_t)c->npop * c->tiles[a] * (c->cells / c->n[a]) * tn * c->esize);
        ALLOC(c->sxc64, sizeof(double) * 4 * c->sx_stride);
        ALLOC(c->sxwork, sizeof(double) * 4 * 2 * kSxMaxNN * kSxMaxNN);
        ALLOC(c->c64, sizeof(double) * 6 * kCoefStride);
        ALLOC(c->gll, sizeof(double) * 2 * kMaxNP);
        ALLOC(c->Wbuf, sizeof(double) * c->m * c->nodes);
        ALLOC(c->partial, sizeof(double) * kDiagBlocks * (kMaxVars + 1));
        ALLOC(c->result, sizeof(double) * 16);
        ALLOC(c->errword, sizeof(int) * 4);
#undef ALLOC
        SetupArgs sa;
        memset(&sa, 0, sizeof sa);
        sa.dim = c->dim;
        sa.degree = degree;
        sa.lambda = c->lambda;
        sa.dt = dt;
        for (int a = 0; a < 3; ++a) {
            sa.h[a] = c->h[a];
            sa.B[a] = 1;
        }
        sa.c64 = c->c64;
        sa.gll = c->gll;     // Gauss-Lobatto weights for the mass diagnostic
        SxSetupArgs xa;
        memset(&xa, 0, sizeof xa);
        xa.dim = c->dim;
        xa.degree = degree;
        xa.lambda = c->lambda;
        xa.dt = dt;
        for (int a = 0; a < 3; ++a) xa.h[a] = c->h[a];
        xa.stride = c->sx_stride;
        xa.c64 = c->sxc64;
        xa.minv = c->result;
        xa.work = c->sxwork;
        cudaError_t e = cudaMemsetAsync(c->errword, 0, sizeof(int) * 4, c->stream);
        if (e == cudaSuccess) e = launch_setup(sa, c->stream);
        if (e == cudaSuccess) e = sx_launch_setup(xa, c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(c->minv, c->result, sizeof(double) * 16, cudaMemcpyDeviceToHost, c->stream);
        c->sx_hrec.assign((size_t)c->nvel * c->sx_stride, 0.0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(c->sx_hrec.data(), c->sxc64, sizeof(double) * c->nvel * c->sx_stride,
                                cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e == cudaSuccess) {
            e = sx_sweep_plan(sx_args(c), c->precision == KIN_FP32, &c->sx_plan);
            c->grid = c->sx_plan.split ? c->sx_plan.bpv : c->nvel * c->sx_plan.bpv;
            c->threads = c->sx_plan.threads;
            c->smem = (int)c->sx_plan.smem;
        }
        if (e != cudaSuccess) {
            g_create_error = std::string("setup failed: ") + cudaGetErrorString(e);
            release_all(c);
            delete c;
            return KIN_ECUDA;
        }
        *out = c;
        return KIN_OK;
    }

    // cell block
    bool user_block = opts->block[0] || opts->block[1] || opts->block[2];
    if (user_block) {
        for (int a = 0; a < 3; ++a) {
            int b = a < c->dim ? opts->block[a] : 1;
            if (b < 1 || c->L[a] % b) {
                delete c;
                return fail(nullptr, KIN_EINVAL, "axis %d: block %d must divide the subdomain extent %d",
                            a, b, c->L[a]);
            }
            c->B[a] = b;
        }
    } else {
        choose_block(c, c->B);
    }
    for (int a = 0; a < 3; ++a) {
        c->nblk[a] = c->n[a] / c->B[a];
        c->nb[a] = c->L[a] / c->B[a];
    }
    size_t smem = block_smem(c, c->B);
    if (smem > 227 * 1024) {
        delete c;
        return fail(nullptr, KIN_EINVAL, "cell block needs %zu bytes of shared memory (> 227 KB)", smem);
    }
    c->kfn = pick_kernel(c->dim, degree, c->system, c->precision);
    if (!c->kfn) {
        delete c;
        return fail(nullptr, KIN_EINVAL, "no kernel for dim %d degree %d", mesh->dim, degree);
    }

    // summaries: per population, n[a]/B[a] blocks x (cells / n[a]) x NP^{d-1} lines
    size_t tn = 1;
    for (int a = 1; a < c->dim; ++a) tn *= c->NP;
    size_t stride = 0, rstride = 0;
    for (int a = 0; a < c->dim; ++a) {
        stride = std::max(stride, (size_t)c->nblk[a] * (c->cells / c->n[a]) * tn);
        rstride = std::max(rstride, (size_t)c->tiles[a] * (c->cells / c->n[a]) * tn);
    }
    c->sig_stride = stride;
    c->raw_stride = rstride;

    kin_status st;
    const size_t fbytes = c->nodes * c->npop * c->esize;
    const size_t sbytes = stride * c->npop * c->esize;
    const size_t rbytes = rstride * c->npop * c->esize;
    void* p;
#define ALLOC(dst, bytes)                                                 \
    do {                                                                  \
        st = dev_alloc(c, (bytes), &p);                                   \
        if (st != KIN_OK) {                                               \
            g_create_error = c->err;                                      \
            release_all(c);                                               \
            delete c;                                                     \
            return st;                                                    \
        }                                                                 \
        dst = (decltype(dst))p;                                           \
    } while (0)
    ALLOC(c->f, fbytes);
    for (int i = 0; i < 2; ++i) {
        ALLOC(c->sig[i], sbytes);
        ALLOC(c->raw[i], rbytes);
    }
    ALLOC(c->c64, sizeof(double) * 6 * kCoefStride);
    ALLOC(c->coef, c->esize == 4 ? sizeof(float) * 6 * kCoefStride : 16);
    ALLOC(c->gll, sizeof(double) * 2 * kMaxNP);
    ALLOC(c->Wbuf, sizeof(double) * c->m * c->nodes);
    ALLOC(c->partial, sizeof(double) * kDiagBlocks * (kMaxVars + 1));
    ALLOC(c->result, sizeof(double) * 8);
    ALLOC(c->errword, sizeof(int) * 4);
    if (c->inflow[0] || c->inflow[1] || c->inflow[2]) ALLOC(c->bnd_dev, sizeof(double) * kMaxPop);
#undef ALLOC
    if (c->esize == 8) c->coef = c->c64;

    {
        cudaError_t e = configure_launch(c);
        if (e != cudaSuccess) {
            g_create_error = std::string("launch configuration failed: ") + cudaGetErrorString(e);
            release_all(c);
            delete c;
            return KIN_ECUDA;
        }
    }

    SetupArgs sa;
    memset(&sa, 0, sizeof sa);
    sa.dim = c->dim;
    sa.degree = degree;
    sa.lambda = c->lambda;
    sa.dt = dt;
    for (int a = 0; a < 3; ++a) {
        sa.h[a] = c->h[a];
        sa.B[a] = c->B[a];
    }
    sa.c64 = c->c64;
    sa.c32 = c->esize == 4 ? (float*)c->coef : nullptr;
    sa.gll = c->gll;
    cudaError_t e = cudaMemsetAsync(c->errword, 0, sizeof(int) * 4, c->stream);
    if (e == cudaSuccess) e = launch_setup(sa, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->coef_host, c->c64, sizeof(c->coef_host), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        g_create_error = std::string("setup kernel failed: ") + cudaGetErrorString(e);
        release_all(c);
        delete c;
        return KIN_ECUDA;
    }
    *out = c;
    return KIN_OK;
}

kin_status kin_create_tet(const kin_tetmesh* mesh, const kin_model* model, double dt, const kin_opts* opts,
                          kin_ctx** out)
{
    if (!out) return fail(nullptr, KIN_EINVAL, "out is NULL");
    *out = nullptr;
    if (!mesh || !model || !opts) return fail(nullptr, KIN_EINVAL, "mesh, model and opts must be non-NULL");
    if (mesh->ncells < 1 || !mesh->xyz || !mesh->vid || !mesh->nbr || !mesh->sub)
        return fail(nullptr, KIN_EINVAL, "the mesh needs cells, xyz, vid, nbr and sub");
    if (model->system != KIN_ADVECTION && model->system != KIN_EULER && model->system != KIN_MAXWELL)
        return fail(nullptr, KIN_EINVAL, "unknown system %d", model->system);
    if (model->velset != KIN_D3Q6 && model->velset != KIN_D3Q4)
        return fail(nullptr, KIN_EINVAL, "tetrahedral meshes take the D3Q6 or D3Q4 velocity set");
    if (model->system == KIN_MAXWELL && !(model->sigma >= 0.0))
        return fail(nullptr, KIN_EINVAL, "the conductivity sigma must be >= 0");
    if (!(model->lambda > 0) || !(dt > 0)) return fail(nullptr, KIN_EINVAL, "lambda and dt must be positive");
    if (!(model->omega >= 1.0 && model->omega <= 2.0)) return fail(nullptr, KIN_EINVAL, "omega must lie in [1, 2]");
    if (model->system == KIN_EULER && !(model->gamma > 1.0)) return fail(nullptr, KIN_EINVAL, "gamma must exceed 1");
    if (opts->iters < 1) return fail(nullptr, KIN_EINVAL, "iters must be >= 1");
    if (opts->precision != KIN_FP64 && opts->precision != KIN_FP32)
        return fail(nullptr, KIN_EINVAL, "unknown precision %d", opts->precision);
    if ((opts->alloc == nullptr) != (opts->free == nullptr))
        return fail(nullptr, KIN_EINVAL, "alloc and free hooks must be given together");
    const int n = mesh->ncells;
    // topology: neighbours in range, every face's vertices present in the
    // neighbour (the nodes that meet across the face), subdomains 0..nsub-1
    int nsub = 0;
    std::vector<int> fnodes((size_t)n * 12), iface(n, 0);
    for (int cc = 0; cc < n; ++cc) {
        if (mesh->sub[cc] < 0) return fail(nullptr, KIN_EINVAL, "cell %d: negative subdomain", cc);
        nsub = std::max(nsub, mesh->sub[cc] + 1);
        for (int a = 0; a < 4; ++a) {
            const long long R = mesh->nbr[(size_t)cc * 4 + a];
            if (R < 0 || R >= n || R == cc)
                return fail(nullptr, KIN_EINVAL, "cell %d face %d: neighbour %lld out of range", cc, a, R);
            int jj = 0;
            for (int j = 0; j < 4; ++j) {
                if (j == a) continue;
                int found = -1;
                for (int q = 0; q < 4; ++q)
                    if (mesh->vid[R * 4 + q] == mesh->vid[(size_t)cc * 4 + j]) found = q;
                if (found < 0)
                    return fail(nullptr, KIN_EINVAL, "cell %d face %d: vertex %d not in the neighbour", cc, a, j);
                fnodes[(size_t)cc * 12 + a * 3 + jj++] = (int)(R * 4 + found);
            }
            const bool wrap = mesh->wrap && mesh->wrap[(size_t)cc * 4 + a];
            if (wrap || mesh->sub[R] != mesh->sub[cc]) iface[cc] |= 1 << a;
        }
    }
    if ((long long)n * 4 * 36 > (1LL << 31))
        return fail(nullptr, KIN_EINVAL, "too many cells for 32-bit node indices");

    kin_ctx* c = new (std::nothrow) kin_ctx();
    if (!c) return fail(nullptr, KIN_ENOMEM, "host allocation failed");
    c->tet = true;
    c->dim = 3;
    c->degree = 1;
    c->system = model->system;
    c->m = model->system == KIN_MAXWELL ? 6 : (model->system == KIN_EULER ? 5 : 1);
    c->simplex = model->velset == KIN_D3Q4;
    c->nvel = c->simplex ? 4 : 6;
    c->npop = c->nvel * c->m;
    c->NP = 2;
    c->NN = 4;
    c->sigma = model->sigma;
    c->lambda = model->lambda;
    c->gamma = model->gamma;
    c->omega = model->omega;
    c->dt = dt;
    c->iters = opts->iters;
    c->precision = opts->precision;
    c->esize = opts->precision == KIN_FP32 ? 4 : 8;
    c->stream = (cudaStream_t)opts->stream;
    c->alloc = opts->alloc;
    c->dealloc = opts->free;
    c->alloc_user = opts->alloc_user;
    c->budget = opts->mem_budget;
    for (int a = 0; a < 3; ++a) c->adv[a] = model->adv[a];
    c->cells = (size_t)n;
    c->nodes = (size_t)n * 4;
    c->nsub = nsub;
    static const int s3[4][3] = {{1, 1, 1}, {1, -1, -1}, {-1, 1, -1}, {-1, -1, 1}};
    double vel[6][3] = {};
    for (int k = 0; k < c->nvel; ++k)
        for (int a = 0; a < 3; ++a) {
            if (c->simplex) {
                c->tsgn[k][a] = s3[k][a];
                vel[k][a] = c->lambda * s3[k][a];
            } else {
                vel[k][a] = a == k / 2 ? (k % 2 ? -c->lambda : c->lambda) : 0.0;
            }
        }

    // faces oriented by every velocity (the same FP64 formulas as the setup
    // kernel: N_a = -grad psi_a / |grad psi_a|; |V.N| <= 1e-12 |V| is parallel)
    std::vector<unsigned char> ftype((size_t)c->nvel * n, 0);
    c->tvol.assign(n, 0.0);
    for (int cc = 0; cc < n; ++cc) {
        const double* x = mesh->xyz + (size_t)cc * 12;
        double e[3][3];
        for (int b = 0; b < 3; ++b)
            for (int i = 0; i < 3; ++i) e[b][i] = x[3 * (b + 1) + i] - x[i];
        auto cross = [](const double* a, const double* b, double* r) {
            r[0] = a[1] * b[2] - a[2] * b[1];
            r[1] = a[2] * b[0] - a[0] * b[2];
            r[2] = a[0] * b[1] - a[1] * b[0];
        };
        double g[4][3], c12[3], c20[3], c01[3];
        cross(e[1], e[2], c12);
        cross(e[2], e[0], c20);
        cross(e[0], e[1], c01);
        const double det = e[0][0] * c12[0] + e[0][1] * c12[1] + e[0][2] * c12[2];
        if (!(std::fabs(det) > 0)) {
            delete c;
            return fail(nullptr, KIN_EINVAL, "cell %d is degenerate", cc);
        }
        c->tvol[cc] = std::fabs(det) / 6.0;
        for (int i = 0; i < 3; ++i) {
            g[1][i] = c12[i] / det;
            g[2][i] = c20[i] / det;
            g[3][i] = c01[i] / det;
            g[0][i] = -(g[1][i] + g[2][i] + g[3][i]);
        }
        for (int k = 0; k < c->nvel; ++k) {
            const double vmag = std::sqrt(vel[k][0] * vel[k][0] + vel[k][1] * vel[k][1] + vel[k][2] * vel[k][2]);
            unsigned char t = 0;
            for (int a = 0; a < 4; ++a) {
                const double gl = std::sqrt(g[a][0] * g[a][0] + g[a][1] * g[a][1] + g[a][2] * g[a][2]);
                const double vn = -(vel[k][0] * g[a][0] + vel[k][1] * g[a][1] + vel[k][2] * g[a][2]) / gl;
                if (std::fabs(vn) > 1e-12 * vmag) t |= (unsigned char)((vn < 0 ? 1 : 2) << (2 * a));
            }
            ftype[(size_t)k * n + cc] = t;
        }
    }
    // breadth-first levels of every subdomain's oriented graph, per velocity
    std::vector<int> order((size_t)c->nvel * n), lstart((size_t)c->nvel * (nsub + 1)), bounds;
    {
        std::vector<int> bysub(n), sstart(nsub + 1, 0);
        for (int cc = 0; cc < n; ++cc) sstart[mesh->sub[cc] + 1]++;
        for (int q = 0; q < nsub; ++q) sstart[q + 1] += sstart[q];
        std::vector<int> fill(sstart.begin(), sstart.end() - 1);
        for (int cc = 0; cc < n; ++cc) bysub[fill[mesh->sub[cc]]++] = cc;
        std::vector<int> indeg(n), lev(n);
        for (int k = 0; k < c->nvel; ++k) {
            int* ord = order.data() + (size_t)k * n;
            for (int cc = 0; cc < n; ++cc) {
                indeg[cc] = 0;
                lev[cc] = 0;
                for (int a = 0; a < 4; ++a)
                    if (((ftype[(size_t)k * n + cc] >> (2 * a)) & 3) == 1 && !((iface[cc] >> a) & 1)) indeg[cc]++;
            }
            int pos = 0;
            for (int q = 0; q < nsub; ++q) {
                lstart[(size_t)k * (nsub + 1) + q] = (int)bounds.size();
                const int head0 = pos;
                for (int i = sstart[q]; i < sstart[q + 1]; ++i)
                    if (indeg[bysub[i]] == 0) ord[pos++] = bysub[i];
                int head = head0;
                while (head < pos) {
                    const int cc = ord[head++];
                    for (int a = 0; a < 4; ++a) {
                        if (((ftype[(size_t)k * n + cc] >> (2 * a)) & 3) != 2 || ((iface[cc] >> a) & 1)) continue;
                        const int R = (int)mesh->nbr[(size_t)cc * 4 + a];
                        lev[R] = std::max(lev[R], lev[cc] + 1);
                        if (--indeg[R] == 0) ord[pos++] = R;
                    }
                }
                if (pos - head0 != sstart[q + 1] - sstart[q]) {
                    delete c;
                    return fail(nullptr, KIN_EINVAL, "subdomain %d: the oriented cell graph of velocity %d has a cycle "
                                "(a subdomain wrapping the periodic box needs its wrap faces marked)", q, k);
                }
                // the breadth-first order lists the cells level by level
                std::stable_sort(ord + head0, ord + pos, [&](int x, int y) { return lev[x] < lev[y]; });
                for (int i = head0; i < pos; ++i)
                    if (i == head0 || lev[ord[i]] != lev[ord[i - 1]]) bounds.push_back(i);
            }
            lstart[(size_t)k * (nsub + 1) + nsub] = (int)bounds.size();
            bounds.push_back(pos);
        }
    }
    // inflow faces per (velocity, position in its order), one word each:
    // the neighbour cell R << 7, the neighbour's local index (2 bits) of
    // each of the face's three vertices at bits 5, 3 and 1, and bit 0 set
    // when the face is a subdomain interface; -1 on the faces that are not
    // inflow faces (R < 2^24 by the cell-count check above)
    std::vector<int> fref((size_t)c->nvel * n * 4, -1);
    for (int k = 0; k < c->nvel; ++k)
        for (int q = 0; q < n; ++q) {
            const int cc = order[(size_t)k * n + q];
            for (int a = 0; a < 4; ++a) {
                if (((ftype[(size_t)k * n + cc] >> (2 * a)) & 3) != 1) continue;
                const int R = fnodes[(size_t)cc * 12 + a * 3] / 4;
                int wd = (R << 7) | ((iface[cc] >> a) & 1);
                for (int jj = 0; jj < 3; ++jj) wd |= (fnodes[(size_t)cc * 12 + a * 3 + jj] & 3) << (5 - 2 * jj);
                fref[((size_t)k * n + q) * 4 + a] = wd;
            }
        }

    kin_status st;
    void* p;
#define ALLOC(dst, bytes)                                                 \
    do {                                                                  \
        st = dev_alloc(c, (bytes), &p);                                   \
        if (st != KIN_OK) {                                               \
            g_create_error = c->err;                                      \
            release_all(c);                                               \
            delete c;                                                     \
            return st;                                                    \
        }                                                                 \
        dst = (decltype(dst))p;                                           \
    } while (0)
    ALLOC(c->f, c->nodes * c->npop * c->esize);
    for (int i = 0; i < 2; ++i) ALLOC(c->titer[i], c->nodes * c->npop * c->esize);
    ALLOC(c->tcoef, (size_t)c->nvel * n * kTetRec * c->esize);
    ALLOC(c->torder, sizeof(int) * order.size());
    ALLOC(c->tlstart, sizeof(int) * lstart.size());
    ALLOC(c->tbounds, sizeof(int) * bounds.size());
    ALLOC(c->tfref, sizeof(int) * fref.size());
    ALLOC(c->Wbuf, sizeof(double) * c->m * c->nodes);
    ALLOC(c->errword, sizeof(int) * 4);
    // FP64 setup scratch: vertex coordinates, face types, FP64 records
    double* xyz_d = nullptr;
    unsigned char* ft_d = nullptr;
    double* c64_d = nullptr;
    ALLOC(xyz_d, sizeof(double) * 12 * (size_t)n);
    ALLOC(ft_d, ftype.size());
    ALLOC(c64_d, sizeof(double) * (size_t)c->nvel * n * kTetRec);
    int* rank_d = nullptr;
    ALLOC(rank_d, sizeof(int) * (size_t)c->nvel * n);
#undef ALLOC
    std::vector<int> rank((size_t)c->nvel * n);
    for (int k = 0; k < c->nvel; ++k)
        for (int q = 0; q < n; ++q) rank[(size_t)k * n + order[(size_t)k * n + q]] = q;
    cudaError_t e = cudaMemcpyAsync(c->torder, order.data(), sizeof(int) * order.size(), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->tlstart, lstart.data(), sizeof(int) * lstart.size(), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->tbounds, bounds.data(), sizeof(int) * bounds.size(), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->tfref, fref.data(), sizeof(int) * fref.size(), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(xyz_d, mesh->xyz, sizeof(double) * 12 * (size_t)n, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ft_d, ftype.data(), ftype.size(), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(rank_d, rank.data(), sizeof(int) * rank.size(), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->errword, 0, sizeof(int) * 4, c->stream);
    if (e == cudaSuccess) {
        TetSetupArgs sa;
        memset(&sa, 0, sizeof sa);
        sa.ncells = n;
        sa.nvel = c->nvel;
        sa.xyz = xyz_d;
        for (int k = 0; k < 6; ++k)
            for (int i = 0; i < 3; ++i) sa.vel[k][i] = vel[k][i];
        sa.dt = dt;
        sa.ftype = ft_d;
        sa.rank = rank_d;
        sa.c64 = c64_d;
        sa.c32 = c->esize == 4 ? (float*)c->tcoef : nullptr;
        e = tet_launch_setup(sa, c->stream);
    }
    if (e == cudaSuccess && c->esize == 8)
        e = cudaMemcpyAsync(c->tcoef, c64_d, sizeof(double) * (size_t)c->nvel * n * kTetRec,
                            cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        fail(nullptr, KIN_ECUDA, "tetrahedral set-up failed: %s", cudaGetErrorString(e));
        release_all(c);
        delete c;
        return KIN_ECUDA;
    }
    // the set-up scratch goes back (the last four allocations)
    for (int i = 0; i < 4; ++i) {
        auto b = c->blocks.back();
        if (c->dealloc) c->dealloc(b.first, b.second, (void*)c->stream, c->alloc_user);
        else cudaFree(b.first);
        c->bytes_held -= b.second;
        c->blocks.pop_back();
    }
    c->grid = (int)(c->nsub * c->nvel);
    c->threads = kTetSweepThreads;
    *out = c;
    return KIN_OK;
}

kin_status kin_set_state(kin_ctx* c, const double* W, size_t n_values, int on_device)
{
    kin_status st = check_usable(c);
    if (st) return st;
    KIN_CUDA(c, order_after_batch(c, c->stream));
    if (!W) return fail(c, KIN_EINVAL, "W is NULL");
    if (n_values != (size_t)c->m * c->nodes)
        return fail(c, KIN_EINVAL, "expected %zu values, got %zu", (size_t)c->m * c->nodes, n_values);
    const double* src = W;
    if (!on_device) {
        KIN_CUDA(c, cudaMemcpyAsync(c->Wbuf, W, n_values * sizeof(double), cudaMemcpyHostToDevice,
                                    c->stream));
        src = c->Wbuf;
    }
    if (c->tet) {
        KIN_CUDA(c, tet_launch_init(tet_args(c), src, c->precision == KIN_FP32, c->stream));
    } else if (c->simplex) {
        KIN_CUDA(c, sx_launch_init(sx_args(c), src, c->precision == KIN_FP32, c->stream));
    } else {
        KIN_CUDA(c, launch_init(point_args(c), src, c->f, c->precision == KIN_FP32, c->stream));
        st = launch_step(c, 1);
        if (st) return st;
    }
    c->sum_stale = false;
    c->have_state = true;
    c->steps_done = 0;
    if (!on_device) {
        KIN_CUDA(c, cudaStreamSynchronize(c->stream));
        return check_errword(c);
    }
    return KIN_OK;
}

kin_status kin_set_kinetic(kin_ctx* c, const void* f, size_t n_values, int on_device)
{
    kin_status st = check_usable(c);
    if (st) return st;
    KIN_CUDA(c, order_after_batch(c, c->stream));
    if (!f) return fail(c, KIN_EINVAL, "f is NULL");
    if (n_values != (size_t)c->npop * c->nodes)
        return fail(c, KIN_EINVAL, "expected %zu values, got %zu", (size_t)c->npop * c->nodes, n_values);
    KIN_CUDA(c, cudaMemcpyAsync(c->f, f, n_values * c->esize,
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
    if (!c->simplex && !c->tet) {
        st = launch_step(c, 1);
        if (st) return st;
    }
    c->sum_stale = false;
    c->have_state = true;
    if (!on_device) {
        KIN_CUDA(c, cudaStreamSynchronize(c->stream));
        return check_errword(c);
    }
    return KIN_OK;
}

kin_status kin_set_kinetic_async(kin_ctx* c, const void* f, size_t n_values, void* stream)
{
    kin_status st = check_usable(c);
    if (st) return st;
    KIN_CUDA(c, order_after_batch(c, stream ? (cudaStream_t)stream : c->stream));
    if (!f) return fail(c, KIN_EINVAL, "f is NULL");
    if (n_values != (size_t)c->npop * c->nodes)
        return fail(c, KIN_EINVAL, "expected %zu values, got %zu", (size_t)c->npop * c->nodes, n_values);
    cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
    KIN_CUDA(c, cudaMemcpyAsync(c->f, f, n_values * c->esize, cudaMemcpyHostToDevice, s));
    // the interface summaries of the new f are computed by the next step
    // (kin_step, kin_batch_step) or diagnostic that needs them
    if (!c->simplex && !c->tet) c->sum_stale = true;
    c->have_state = true;
    return KIN_OK;
}

kin_status kin_get_kinetic_async(kin_ctx* c, void* f, size_t n_values, void* stream)
{
    kin_status st = check_usable(c);
    if (st) return st;
    KIN_CUDA(c, order_after_batch(c, stream ? (cudaStream_t)stream : c->stream));
    if (!f) return fail(c, KIN_EINVAL, "f is NULL");
    if (n_values != (size_t)c->npop * c->nodes)
        return fail(c, KIN_EINVAL, "expected %zu values, got %zu", (size_t)c->npop * c->nodes, n_values);
    if (!c->have_state) return fail(c, KIN_ESTATE, "no state has been set");
    cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
    KIN_CUDA(c, cudaMemcpyAsync(f, c->f, n_values * c->esize, cudaMemcpyDeviceToHost, s));
    return KIN_OK;
}

// An inflow face without a boundary state (name of the first one, or null).
static const char* missing_boundary(const kin_ctx* c)
{
    static const char* names[3][2] = {{"x lower", "x upper"}, {"y lower", "y upper"}, {"z lower", "z upper"}};
    for (int a = 0; a < 3; ++a)
        for (int sd = 0; sd < 2; ++sd)
            if (c->inflow[a] && !c->bnd_set[a][sd]) return names[a][sd];
    return nullptr;
}

kin_status kin_set_boundary(kin_ctx* c, int axis, int side, const double* W, size_t m)
{
    kin_status st = check_usable(c);
    if (st) return st;
    KIN_CUDA(c, order_after_batch(c, c->stream));
    if (c->tet) return fail(c, KIN_EINVAL, "tetrahedral meshes are periodic: no boundary faces");
    if (axis < 0 || axis >= c->dim || !c->inflow[axis])
        return fail(c, KIN_EINVAL, "axis %d is not an inflow axis", axis);
    if (side != 0 && side != 1) return fail(c, KIN_EINVAL, "side must be 0 (lower) or 1 (upper)");
    if (!W || m != (size_t)c->m) return fail(c, KIN_EINVAL, "expected %d boundary values", c->m);
    for (int v = 0; v < c->m; ++v)
        if (!std::isfinite(W[v])) return fail(c, KIN_EINVAL, "boundary state is not finite");
    if (c->system == KIN_EULER && !(W[0] > 0.0)) return fail(c, KIN_EINVAL, "boundary density must be > 0");
    double M[kMaxPop];
    axis_maxwellian(point_args(c), W, M);
    // the populations moving along +e_axis enter through the lower face, the
    // ones moving along -e_axis through the upper face
    const int k = 2 * axis + side;
    for (int v = 0; v < c->m; ++v) c->bnd[k * c->m + v] = M[k * c->m + v];
    // the device copy, in the context precision, stream-ordered before the next step
    if (c->esize == 4) {
        float* h = reinterpret_cast<float*>(c->bnd_host);
        for (int p = 0; p < c->npop; ++p) h[p] = (float)c->bnd[p];
    } else {
        for (int p = 0; p < c->npop; ++p) c->bnd_host[p] = c->bnd[p];
    }
    KIN_CUDA(c, cudaMemcpyAsync(c->bnd_dev, c->bnd_host, (size_t)c->npop * c->esize, cudaMemcpyHostToDevice,
                                c->stream));
    c->bnd_set[axis][side] = true;
    return KIN_OK;
}

kin_status kin_step(kin_ctx* c, int nsteps)
{
    kin_status st = check_usable(c);
    if (st) return st;
    KIN_CUDA(c, order_after_batch(c, c->stream));
    if (nsteps < 0) return fail(c, KIN_EINVAL, "nsteps must be >= 0");
    if (!c->have_state) return fail(c, KIN_ESTATE, "no state: call kin_set_state or kin_set_kinetic first");
    if (const char* face = missing_boundary(c))
        return fail(c, KIN_ESTATE, "the %s face of an inflow axis has no boundary state (kin_set_boundary)", face);
    if (nsteps > 0 && c->sum_stale) {
        st = launch_step(c, 1);
        if (st) return st;
        c->sum_stale = false;
    }
    for (int s = 0; s < nsteps; ++s) {
        st = c->tet ? tet_step(c) : (c->simplex ? sx_step(c) : launch_step(c, 0));
        if (st) return st;
        c->steps_done++;
    }
    return KIN_OK;
}

kin_status kin_get_state(kin_ctx* c, double* W, size_t n_values, int on_device)
{
    kin_status st = check_usable(c);
    if (st) return st;
    KIN_CUDA(c, order_after_batch(c, c->stream));
    if (!W) return fail(c, KIN_EINVAL, "W is NULL");
    if (n_values != (size_t)c->m * c->nodes)
        return fail(c, KIN_EINVAL, "expected %zu values, got %zu", (size_t)c->m * c->nodes, n_values);
    if (!c->have_state) return fail(c, KIN_ESTATE, "no state has been set");
    double* dst = on_device ? W : c->Wbuf;
    KIN_CUDA(c, launch_moments(point_args(c), c->f, dst, c->precision == KIN_FP32, c->stream));
    if (!on_device) {
        KIN_CUDA(c, cudaMemcpyAsync(W, c->Wbuf, n_values * sizeof(double), cudaMemcpyDeviceToHost,
                                    c->stream));
        KIN_CUDA(c, cudaStreamSynchronize(c->stream));
        return check_errword(c);
    }
    return KIN_OK;
}

kin_status kin_get_kinetic(kin_ctx* c, void* f, size_t n_values, int on_device)
{
    kin_status st = check_usable(c);
    if (st) return st;
    KIN_CUDA(c, order_after_batch(c, c->stream));
    if (!f) return fail(c, KIN_EINVAL, "f is NULL");
    if (n_values != (size_t)c->npop * c->nodes)
        return fail(c, KIN_EINVAL, "expected %zu values, got %zu", (size_t)c->npop * c->nodes, n_values);
    if (!c->have_state) return fail(c, KIN_ESTATE, "no state has been set");
    KIN_CUDA(c, cudaMemcpyAsync(f, c->f, n_values * c->esize,
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    if (!on_device) {
        KIN_CUDA(c, cudaStreamSynchronize(c->stream));
        return check_errword(c);
    }
    return KIN_OK;
}

kin_status kin_diag(kin_ctx* c, double* mass_per_var, double* next_defect, double* iter_residual)
{
    kin_status st = check_usable(c);
    if (st) return st;
    KIN_CUDA(c, order_after_batch(c, c->stream));
    if (!c->have_state) return fail(c, KIN_ESTATE, "no state has been set");
    if ((next_defect || iter_residual) && (c->inflow[0] || c->inflow[1] || c->inflow[2]))
        return fail(c, KIN_EINVAL, "next_defect and iter_residual are not available with inflow axes");
    if (c->tet) {
        // the exact integral of the P1 moments: sum over cells of |L|/4 times
        // the sum of W over the cell's nodes (FP64 moments, host reduction)
        if (next_defect || iter_residual)
            return fail(c, KIN_EINVAL, "next_defect and iter_residual are not available on tetrahedral meshes");
        if (mass_per_var) {
            KIN_CUDA(c, launch_moments(point_args(c), c->f, c->Wbuf, c->precision == KIN_FP32, c->stream));
            std::vector<double> W((size_t)c->m * c->nodes);
            KIN_CUDA(c, cudaMemcpyAsync(W.data(), c->Wbuf, sizeof(double) * W.size(), cudaMemcpyDeviceToHost,
                                        c->stream));
            KIN_CUDA(c, cudaStreamSynchronize(c->stream));
            for (int v = 0; v < c->m; ++v) {
                double acc = 0.0;
                for (size_t cc = 0; cc < c->cells; ++cc) {
                    const double* w = W.data() + (size_t)v * c->nodes + cc * 4;
                    acc += c->tvol[cc] / 4.0 * (w[0] + w[1] + w[2] + w[3]);
                }
                mass_per_var[v] = acc;
            }
        }
        return KIN_OK;
    }
    double host[8] = {0};
    if (mass_per_var) {
        KIN_CUDA(c, launch_mass(point_args(c), c->f, c->gll, c->partial, c->result,
                                c->precision == KIN_FP32, c->stream));
        KIN_CUDA(c, cudaMemcpyAsync(host, c->result, sizeof(double) * kMaxVars, cudaMemcpyDeviceToHost, c->stream));
        KIN_CUDA(c, cudaStreamSynchronize(c->stream));
        for (int v = 0; v < c->m; ++v) mass_per_var[v] = host[v];
    }
    if ((next_defect || iter_residual) && c->simplex) {
        if (next_defect)
            for (int v = 0; v < c->m; ++v) next_defect[v] = NAN;
        if (iter_residual) *iter_residual = NAN;
    } else if (next_defect || iter_residual) {
        if (c->sum_stale) {
            st = launch_step(c, 1);
            if (st) return st;
            c->sum_stale = false;
        }
        DefectArgs da;
        memset(&da, 0, sizeof da);
        da.dim = c->dim;
        da.degree = c->degree;
        da.m = c->m;
        da.iters = c->iters;
        da.sig_stride = (long long)c->sig_stride;
        da.raw_stride = (long long)c->raw_stride;
        da.dt = c->dt;
        da.lambda = c->lambda;
        long long tn = 1;
        for (int a = 1; a < c->dim; ++a) tn *= c->NP;
        for (int a = 0; a < 3; ++a) {
            da.h[a] = c->h[a];
            da.nb[a] = c->nb[a];
            da.NS[a] = c->tiles[a];
            da.glines[a] = a < c->dim ? (long long)(c->cells / c->n[a]) * tn : 0;
        }
        da.total = 0;
        for (int pop = 0; pop < c->npop; ++pop) {
            int a = (pop / c->m) / 2;
            da.per_pop[pop] = (long long)c->tiles[a] * da.glines[a];
            da.total += da.per_pop[pop];
        }
        KIN_CUDA(c, launch_defect(da, c->sig[c->cur], c->raw[c->cur], c->c64, c->gll, c->partial,
                                  c->result, c->precision == KIN_FP32, c->stream));
        KIN_CUDA(c, cudaMemcpyAsync(host, c->result, sizeof(double) * (kMaxVars + 1), cudaMemcpyDeviceToHost,
                                    c->stream));
        KIN_CUDA(c, cudaStreamSynchronize(c->stream));
        if (next_defect)
            for (int v = 0; v < c->m; ++v) next_defect[v] = host[v];
        if (iter_residual) *iter_residual = host[kMaxVars];
    }
    return check_errword(c);
}

kin_status kin_sync(kin_ctx* c)
{
    kin_status st = check_usable(c);
    if (st) return st;
    KIN_CUDA(c, order_after_batch(c, c->stream));
    KIN_CUDA(c, cudaStreamSynchronize(c->stream));
    return check_errword(c);
}

kin_status kin_query(const kin_ctx* c, kin_info* info)
{
    if (!c || !info) return KIN_EINVAL;
    memset(info, 0, sizeof *info);
    info->dim = c->dim;
    info->degree = c->degree;
    info->m = c->m;
    info->nvel = c->nvel;
    info->npop = c->npop;
    info->nodes_per_cell = c->NN;
    info->cells = c->cells;
    info->nodes = c->nodes;
    info->kinetic_values = (size_t)c->npop * c->nodes;
    info->state_values = (size_t)c->m * c->nodes;
    info->device_bytes = c->bytes_held;
    info->precision = c->precision;
    for (int a = 0; a < 3; ++a) info->block[a] = c->B[a];
    info->smem_bytes = c->smem;
    info->grid = c->grid;
    info->threads = c->threads;
    info->stages = c->stages;
    info->specialised = c->fixed ? 1 : 0;
    info->steps_done = c->steps_done;
    return KIN_OK;
}

kin_status kin_destroy(kin_ctx* c)
{
    if (!c) return KIN_OK;
    if (c->wait_batch) cudaEventSynchronize(c->after_batch);
    cudaStreamSynchronize(c->stream);
    release_all(c);
    delete c;
    return KIN_OK;
}

const char* kin_last_error(const kin_ctx* c)
{
    if (!c) return g_create_error.c_str();
    return c->err.empty() ? "no error" : c->err.c_str();
}

}  // extern "C"


// ---------------------------------------------------------------------------
// batches of independent problems
// ---------------------------------------------------------------------------

struct kin_batch {
    struct Group {
        const void* fn = nullptr;
        int threads = 0, grid = 0;
        size_t smem = 0;
        std::vector<int> members;     // indices into kin_batch::members
        int nwork = 0;
        Inst* insts[2] = {nullptr, nullptr};   // launch records for summary parity 0 / 1
        Inst* prep[2] = {nullptr, nullptr};    // summaries-only records (members whose f was replaced)
        int2* work = nullptr;
    };
    std::vector<kin_ctx*> members;
    std::vector<int> expect_cur;      // members' summary parity at batch parity 0
    std::vector<int> solo;            // members stepped by their own kernel
    std::vector<Group> groups;        // groups[0] is the mixed launch when nmixed > 0
    Group mixed;                      // members of the one-launch mixed-degree kernel
    int nmixed = 0;
    void* arena = nullptr;            // one stream-ordered device allocation: launch records and work lists
    std::vector<cudaEvent_t> ev_member;
    cudaEvent_t ev_done = nullptr;
    bool direct = false;              // enqueue the launches per step instead of replaying graphs
    cudaStream_t stream = nullptr;
    bool own_stream = false;          // created here because the caller passed NULL
    cudaGraphExec_t g2[2] = {nullptr, nullptr};   // two steps starting at parity q
    cudaGraphExec_t g1[2] = {nullptr, nullptr};   // one step at parity q
    int parity = 0;
    std::string err = "no error";
};

static thread_local std::string g_batch_error = "no error";

static kin_status batch_fail(kin_batch* b, kin_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (b) b->err = buf;
    else g_batch_error = buf;
    return st;
}

static void batch_release(kin_batch* b)
{
    for (int q = 0; q < 2; ++q) {
        if (b->g2[q]) cudaGraphExecDestroy(b->g2[q]);
        if (b->g1[q]) cudaGraphExecDestroy(b->g1[q]);
    }
    for (auto e : b->ev_member)
        if (e) cudaEventDestroy(e);
    if (b->ev_done) cudaEventDestroy(b->ev_done);
    // stream-ordered free: no device-wide synchronisation while other
    // streams run (the batch's work on its stream finishes first)
    if (b->arena) cudaFreeAsync(b->arena, b->stream);
    b->arena = nullptr;
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    b->stream = nullptr;
}

// Enqueue launch k of a batch step (a kernel-type group, then the solo
// members) at summary parity q (members' cur = expect_cur ^ q) on stream st.
static cudaError_t batch_launch(kin_batch* b, size_t k, int q, cudaStream_t st, bool prep = false)
{
    if (k < b->groups.size()) {
        auto& g = b->groups[k];
        const Inst* insts = prep ? g.prep[q] : g.insts[q];
        const int2* work = g.work;
        int nwork = g.nwork;
        void* args[] = {(void*)&insts, (void*)&work, (void*)&nwork};
        return cudaLaunchKernel(g.fn, dim3(g.grid), dim3(g.threads), args, g.smem, st);
    }
    const int mi = b->solo[k - b->groups.size()];
    kin_ctx* c = b->members[mi];
    const int saved = c->cur;
    c->cur = b->expect_cur[mi] ^ q;
    Inst I = make_inst(c, prep ? 1 : 0);
    if (prep) {
        I.sig_out = c->sig[c->cur];
        I.raw_out = c->raw[c->cur];
    }
    c->cur = saved;
    void* args[] = {&I};
    return cudaLaunchKernel((const void*)c->kfn, dim3(c->grid), dim3(c->threads), args, (size_t)c->smem, st);
}

// Enqueue nsteps batch steps starting at summary parity q: every launch of
// a step on the batch stream, step after step.  (Running the launches of
// different kernel types on forked streams, so that one type's launch could
// fill another's tail, measured no faster: with persistent grids over
// hundreds of tiles per type the tails are short.)
static cudaError_t batch_enqueue_steps(kin_batch* b, int q, int nsteps)
{
    const size_t nl = b->groups.size() + b->solo.size();
    cudaError_t e = cudaSuccess;
    for (int s = 0; s < nsteps && e == cudaSuccess; ++s)
        for (size_t k = 0; k < nl && e == cudaSuccess; ++k) e = batch_launch(b, k, q ^ (s & 1), b->stream);
    return e;
}

static cudaError_t batch_capture(kin_batch* b, int q, int nsteps, cudaGraphExec_t* out)
{
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaError_t el = batch_enqueue_steps(b, q, nsteps);
    e = cudaStreamEndCapture(b->stream, &graph);
    if (el != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return el;
    }
    if (e != cudaSuccess) return e;
    e = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    return e;
}

extern "C" kin_status kin_batch_create(kin_ctx* const* members, int count, void* stream, kin_batch** out)
{
    return kin_batch_create_ex(members, count, stream, 0, out);
}

extern "C" kin_status kin_batch_create_ex(kin_ctx* const* members, int count, void* stream, int flags,
                                          kin_batch** out)
{
    if (!out) return batch_fail(nullptr, KIN_EINVAL, "out is NULL");
    if (flags & ~(KIN_BATCH_DIRECT | KIN_BATCH_MIXED))
        return batch_fail(nullptr, KIN_EINVAL, "unknown flags 0x%x", flags);
    *out = nullptr;
    if (!members || count < 1) return batch_fail(nullptr, KIN_EINVAL, "need at least one member");
    for (int i = 0; i < count; ++i) {
        if (!members[i]) return batch_fail(nullptr, KIN_EINVAL, "member %d is NULL", i);
        if (members[i]->poisoned) return batch_fail(nullptr, KIN_ESTATE, "member %d is poisoned", i);
        if (!members[i]->have_state) return batch_fail(nullptr, KIN_ESTATE, "member %d has no state", i);
        if (missing_boundary(members[i]))
            return batch_fail(nullptr, KIN_ESTATE, "member %d has an inflow face without a boundary state", i);
        if (members[i]->simplex)
            return batch_fail(nullptr, KIN_EINVAL, "member %d uses a d+1 velocity set (not batched)", i);
        if (members[i]->tet)
            return batch_fail(nullptr, KIN_EINVAL, "member %d has a tetrahedral mesh (not batched)", i);
        for (int j = 0; j < i; ++j)
            if (members[j] == members[i]) return batch_fail(nullptr, KIN_EINVAL, "member %d repeats member %d", i, j);
    }
    kin_batch* b = new (std::nothrow) kin_batch();
    if (!b) return batch_fail(nullptr, KIN_ENOMEM, "host allocation failed");
    b->stream = (cudaStream_t)stream;
    if (!b->stream) {
        // graphs cannot be captured on the legacy default stream
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            delete b;
            return batch_fail(nullptr, KIN_ECUDA, "could not create the batch stream");
        }
        b->own_stream = true;
    }
    b->members.assign(members, members + count);
    for (auto* c : b->members) b->expect_cur.push_back(c->cur);

    // With KIN_BATCH_MIXED, one launch for the 2D Euler FP32 members of
    // degrees 1..3 whose cell block matches a slot of a compiled mixed
    // kernel: of the compiled ones, the kernel that covers the most kinetic
    // DOF of the batch.
    std::vector<char> in_mixed(count, 0);
    MixedKernel mk[8];
    const int nmk = (flags & KIN_BATCH_MIXED) ? mixed_kernels_2d(mk, 8) : 0;
    auto mixable = [&](const kin_ctx* c, const MixedKernel& k) {
        return c->fixed && c->dim == 2 && c->system == KIN_EULER && c->precision == KIN_FP32 &&
               c->stages == 1 && c->degree >= 1 && c->degree <= 3 && c->B[0] == k.block[c->degree - 1][0] &&
               c->B[1] == k.block[c->degree - 1][1];
    };
    int best = -1;
    double best_dof = 0;
    for (int k = 0; k < nmk; ++k) {
        double dof = 0;
        for (int i = 0; i < count; ++i)
            if (mixable(b->members[i], mk[k])) dof += (double)b->members[i]->npop * b->members[i]->nodes;
        if (dof > best_dof) {
            best_dof = dof;
            best = k;
        }
    }
    if (best >= 0) {
        b->mixed.fn = mk[best].fn;
        b->mixed.threads = mk[best].threads;
        b->mixed.smem = mk[best].smem;
        for (int i = 0; i < count; ++i)
            if (mixable(b->members[i], mk[best])) {
                in_mixed[i] = 1;
                b->mixed.members.push_back(i);
            }
    }

    // group the other members that run a fixed-shape kernel by kernel
    for (int i = 0; i < count; ++i) {
        if (in_mixed[i]) continue;
        kin_ctx* c = b->members[i];
        FixedKernel fk{nullptr, nullptr, 0, 0};
        if (c->fixed && c->dim == 2) fk = fixed_kernel_d2(c->degree, c->system, c->precision, c->B, c->stages);
        if (c->fixed && c->dim == 3) fk = fixed_kernel_d3(c->degree, c->system, c->precision, c->B, c->stages);
        if (!fk.batch_fn) {
            b->solo.push_back(i);
            continue;
        }
        kin_batch::Group* g = nullptr;
        for (auto& gg : b->groups)
            if (gg.fn == fk.batch_fn) g = &gg;
        if (!g) {
            b->groups.emplace_back();
            g = &b->groups.back();
            g->fn = fk.batch_fn;
            g->threads = fk.threads;
            g->smem = fk.smem;
        }
        g->members.push_back(i);
    }

    if (!b->mixed.members.empty()) b->groups.insert(b->groups.begin(), b->mixed);
    b->nmixed = (int)b->mixed.members.size();

    cudaError_t e = cudaSuccess;
    int dev = 0, nsm = 1;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    // every group's launch records and work list, staged on the host and
    // copied into one device arena (offsets 256-byte aligned)
    std::vector<unsigned char> stage;
    auto place = [&](const void* src, size_t bytes) {
        const size_t off = (stage.size() + 255) / 256 * 256;
        stage.resize(off + bytes);
        memcpy(stage.data() + off, src, bytes);
        return off;
    };
    struct Offs {
        size_t insts[2], prep[2], work;
    };
    std::vector<Offs> offs(b->groups.size());
    for (size_t gi = 0; gi < b->groups.size(); ++gi) {
        auto& g = b->groups[gi];
        if (e != cudaSuccess) break;
        const bool mixed = gi == 0 && b->nmixed > 0;
        std::vector<Inst> h[2], hp[2];
        std::vector<int2> work;
        for (size_t k = 0; k < g.members.size(); ++k) {
            kin_ctx* c = b->members[g.members[k]];
            const int saved = c->cur;
            for (int q = 0; q < 2; ++q) {
                c->cur = b->expect_cur[g.members[k]] ^ q;
                h[q].push_back(make_inst(c, 0));
                Inst I = make_inst(c, 1);
                I.sig_out = c->sig[c->cur];
                I.raw_out = c->raw[c->cur];
                hp[q].push_back(I);
            }
            c->cur = saved;
            const int ntiles = c->nblk[0] * c->nblk[1] * c->nblk[2];
            // mixed launch: the degree rides in the top byte of the instance index
            const int tag = mixed ? (c->degree << 24) : 0;
            for (int t = 0; t < ntiles; ++t) work.push_back(make_int2(tag | (int)k, t));
        }
        if (mixed) {
            // the most expensive tiles first (per-tile DOF, higher degree
            // first on ties), so that the persistent blocks end on short tiles
            auto cost = [&](const int2& w) {
                const kin_ctx* c = b->members[g.members[w.x & 0xffffff]];
                return (double)c->npop * c->NN * c->B[0] * c->B[1] * c->B[2] * (1.0 + 0.01 * c->degree);
            };
            std::stable_sort(work.begin(), work.end(),
                             [&](const int2& x, const int2& y) { return cost(x) > cost(y); });
        }
        g.nwork = (int)work.size();
        if (g.smem > 48 * 1024)
            e = cudaFuncSetAttribute(g.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(g.fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        int occ = 1;
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, g.fn, g.threads, g.smem);
        g.grid = (int)std::min<long long>(g.nwork, (long long)std::max(occ, 1) * nsm);
        for (int q = 0; q < 2; ++q) {
            offs[gi].insts[q] = place(h[q].data(), sizeof(Inst) * h[q].size());
            offs[gi].prep[q] = place(hp[q].data(), sizeof(Inst) * hp[q].size());
        }
        offs[gi].work = place(work.data(), sizeof(int2) * work.size());
    }
    if (e == cudaSuccess && !stage.empty()) {
        e = cudaMallocAsync(&b->arena, stage.size(), b->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->arena, stage.data(), stage.size(), cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);   // the staging vector goes away
        for (size_t gi = 0; gi < b->groups.size() && e == cudaSuccess; ++gi) {
            auto& g = b->groups[gi];
            unsigned char* base = static_cast<unsigned char*>(b->arena);
            for (int q = 0; q < 2; ++q) {
                g.insts[q] = reinterpret_cast<Inst*>(base + offs[gi].insts[q]);
                g.prep[q] = reinterpret_cast<Inst*>(base + offs[gi].prep[q]);
            }
            g.work = reinterpret_cast<int2*>(base + offs[gi].work);
        }
    }
    b->ev_member.assign(count, nullptr);
    for (int i = 0; i < count && e == cudaSuccess; ++i)
        e = cudaEventCreateWithFlags(&b->ev_member[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_done, cudaEventDisableTiming);
    b->direct = (flags & KIN_BATCH_DIRECT) != 0;
    for (int q = 0; q < 2 && e == cudaSuccess && !b->direct; ++q) {
        e = batch_capture(b, q, 2, &b->g2[q]);
        if (e == cudaSuccess) e = batch_capture(b, q, 1, &b->g1[q]);
    }
    if (e != cudaSuccess) {
        kin_status st = batch_fail(nullptr, e == cudaErrorMemoryAllocation ? KIN_ENOMEM : KIN_ECUDA,
                                   "batch set-up failed: %s", cudaGetErrorString(e));
        cudaGetLastError();
        batch_release(b);
        delete b;
        return st;
    }
    *out = b;
    return KIN_OK;
}

extern "C" kin_status kin_batch_step(kin_batch* b, int nsteps)
{
    if (!b) return KIN_EINVAL;
    if (nsteps < 0) return batch_fail(b, KIN_EINVAL, "nsteps must be >= 0");
    for (size_t i = 0; i < b->members.size(); ++i) {
        kin_ctx* c = b->members[i];
        if (c->poisoned) return batch_fail(b, KIN_ESTATE, "member %zu is poisoned", i);
        if (c->cur != (b->expect_cur[i] ^ b->parity))
            return batch_fail(b, KIN_ESTATE, "member %zu was stepped outside the batch", i);
        if (missing_boundary(c))
            return batch_fail(b, KIN_ESTATE, "member %zu has an inflow face without a boundary state", i);
    }
    if (nsteps == 0) return KIN_OK;
    // order the step after each member's earlier work: the work queued on
    // its stream (once per distinct stream) and, when its last step was a
    // batch step on another stream, that step
    cudaError_t e = cudaSuccess;
    std::vector<cudaStream_t> seen;
    for (size_t i = 0; i < b->members.size() && e == cudaSuccess; ++i) {
        kin_ctx* c = b->members[i];
        if (c->wait_batch) e = cudaStreamWaitEvent(b->stream, c->after_batch, 0);
        if (e != cudaSuccess || std::find(seen.begin(), seen.end(), c->stream) != seen.end()) continue;
        seen.push_back(c->stream);
        e = cudaEventRecord(b->ev_member[i], c->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->ev_member[i], 0);
    }
    // members whose f was replaced by kin_set_kinetic_async: one summaries
    // pass over every member, one launch per kernel type, before the step
    bool stale = false;
    for (auto* c : b->members) stale = stale || c->sum_stale;
    if (stale) {
        const size_t nl = b->groups.size() + b->solo.size();
        for (size_t k = 0; k < nl && e == cudaSuccess; ++k) e = batch_launch(b, k, b->parity, b->stream, true);
        if (e == cudaSuccess)
            for (auto* c : b->members) c->sum_stale = false;
    }
    if (b->direct) {
        if (e == cudaSuccess) e = batch_enqueue_steps(b, b->parity, nsteps);
        if (nsteps & 1) b->parity ^= 1;
    } else {
        int left = nsteps;
        while (e == cudaSuccess && left >= 2) {
            e = cudaGraphLaunch(b->g2[b->parity], b->stream);
            left -= 2;
        }
        if (e == cudaSuccess && left == 1) {
            e = cudaGraphLaunch(b->g1[b->parity], b->stream);
            b->parity ^= 1;
        }
    }
    if (e == cudaSuccess) e = cudaEventRecord(b->ev_done, b->stream);
    // each member's later work waits for this step when the member is next used
    for (size_t i = 0; i < b->members.size() && e == cudaSuccess; ++i) {
        kin_ctx* c = b->members[i];
        if (!c->after_batch) e = cudaEventCreateWithFlags(&c->after_batch, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(c->after_batch, b->stream);
        if (e == cudaSuccess) c->wait_batch = true;
    }
    if (e != cudaSuccess) return batch_fail(b, KIN_ECUDA, "batch step failed: %s", cudaGetErrorString(e));
    for (auto* c : b->members) {
        if (nsteps & 1) c->cur ^= 1;
        c->steps_done += nsteps;
    }
    return KIN_OK;
}

extern "C" kin_status kin_batch_sync(kin_batch* b)
{
    if (!b) return KIN_EINVAL;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return batch_fail(b, KIN_ECUDA, "batch sync failed: %s", cudaGetErrorString(e));
    // the error words are read on the batch's stream: a member's own stream
    // may be shared with, and busy on behalf of, contexts outside the batch
    std::vector<int> h(b->members.size(), 0);
    for (size_t i = 0; i < b->members.size() && e == cudaSuccess; ++i)
        e = cudaMemcpyAsync(&h[i], b->members[i]->errword, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return batch_fail(b, KIN_ECUDA, "batch sync failed: %s", cudaGetErrorString(e));
    for (size_t i = 0; i < b->members.size(); ++i) {
        kin_status st = errword_status(b->members[i], h[i]);
        if (st) return batch_fail(b, st, "member %zu: %s", i, b->members[i]->err.c_str());
    }
    return KIN_OK;
}

extern "C" kin_status kin_batch_destroy(kin_batch* b)
{
    if (!b) return KIN_OK;
    cudaStreamSynchronize(b->stream);
    batch_release(b);
    delete b;
    return KIN_OK;
}

extern "C" kin_status kin_batch_info(const kin_batch* b, int* launches_per_step, int* mixed_members)
{
    if (!b) return KIN_EINVAL;
    if (launches_per_step) *launches_per_step = (int)(b->groups.size() + b->solo.size());
    if (mixed_members) *mixed_members = b->nmixed;
    return KIN_OK;
}

extern "C" const char* kin_batch_last_error(const kin_batch* b)
{
    return b ? b->err.c_str() : g_batch_error.c_str();
}

// ---------------------------------------------------------------------------
// kin_step_noalloc: the step kernels with their scratch in a static device
// array, for callers that cannot allocate device memory.
//
// Some callers cannot let a library call cudaMalloc: host applications whose
// own memory pool reserves the device's memory up front (a library
// allocation would fail or fragment that pool), and code paths that run on a
// fixed memory plan where an allocation failure at run time is not
// acceptable.  This entry point takes the caller's kinetic state and keeps
// everything else it needs -- the FP64/FP32 block-inverse coefficients, the
// Gauss-Lobatto rule and the two ping-pong copies of the block summaries --
// in g_noalloc_scratch below.
//
// The array is a file-scope __device__ object, so every GPU that loads this
// library holds kNoallocScratchBytes of it until the process exits.  Host
// code may not use its name as an address: the address is taken once per
// device, with that device current, by cudaGetSymbolAddress.
// ---------------------------------------------------------------------------

#include <mutex>

namespace {

constexpr size_t kNoallocScratchBytes = size_t(16) << 20;   // 16 MiB per device
constexpr int kNoallocMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_addr[kNoallocMaxDevices] = {};

void noalloc_msg(char* buf, size_t len, const char* fmt, ...)
{
    if (!buf || !len) return;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, len, fmt, ap);
    va_end(ap);
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

extern "C" kin_status kin_step_noalloc(const kin_mesh* mesh, const kin_model* model, int degree,
                                       double dt, const kin_opts* opts, void* f, int nsteps,
                                       char* errbuf, size_t errlen)
{
    if (errbuf && errlen) errbuf[0] = '\0';
    if (!mesh || !model || !opts || !f) {
        noalloc_msg(errbuf, errlen, "mesh, model, opts and f are required");
        return KIN_EINVAL;
    }
    if (nsteps < 0) {
        noalloc_msg(errbuf, errlen, "nsteps must be >= 0");
        return KIN_EINVAL;
    }
    if (mesh->dim < 1 || mesh->dim > 3 || degree < 1 || degree > 3 ||
        (model->system != KIN_ADVECTION && model->system != KIN_EULER && model->system != KIN_MAXWELL) ||
        (model->system == KIN_MAXWELL && (mesh->dim != 3 || !(model->sigma >= 0.0))) || model->velset != mesh->dim ||
        mesh->inflow[0] || mesh->inflow[1] || mesh->inflow[2] ||
        !(model->lambda > 0) || !(dt > 0) || !(model->omega >= 1.0 && model->omega <= 2.0) ||
        (model->system == KIN_EULER && !(model->gamma > 1.0)) || opts->iters < 1 ||
        (opts->precision != KIN_FP64 && opts->precision != KIN_FP32)) {
        noalloc_msg(errbuf, errlen, "invalid mesh, model, degree, dt or opts (same rules as kin_create)");
        return KIN_EINVAL;
    }

    // The same problem set-up as kin_create, on the stack: the buffers point
    // into the static scratch instead of allocations.
    kin_ctx c;
    c.dim = mesh->dim;
    c.degree = degree;
    c.system = model->system;
    c.m = model->system == KIN_MAXWELL ? 6 : (model->system == KIN_EULER ? mesh->dim + 2 : 1);
    c.sigma = model->sigma;
    c.nvel = 2 * mesh->dim;
    c.npop = c.nvel * c.m;
    c.NP = degree + 1;
    c.NN = 1;
    for (int a = 0; a < c.dim; ++a) c.NN *= c.NP;
    c.lambda = model->lambda;
    c.gamma = model->gamma;
    c.omega = model->omega;
    c.dt = dt;
    c.iters = opts->iters;
    c.precision = opts->precision;
    c.esize = opts->precision == KIN_FP32 ? 4 : 8;
    c.stream = (cudaStream_t)opts->stream;
    if (opts->threads != 0 && (opts->threads < 32 || opts->threads > kThreads || opts->threads % 32)) {
        noalloc_msg(errbuf, errlen, "threads must be 0 or a multiple of 32 in [32, %d]", kThreads);
        return KIN_EINVAL;
    }
    if (opts->stages < 0 || opts->stages > 2) {
        noalloc_msg(errbuf, errlen, "stages must be 0, 1 or 2");
        return KIN_EINVAL;
    }
    c.want_threads = opts->threads;
    c.want_stages = opts->stages;
    c.wait_timeout_s = opts->wait_timeout_s;     // the bound on device waits, as in kin_create
    c.cells = 1;
    for (int a = 0; a < 3; ++a) {
        c.adv[a] = model->adv[a];
        if (a < c.dim) {
            if (mesh->n[a] < 1 || !(mesh->hi[a] > mesh->lo[a]) || opts->tiles[a] < 1 ||
                mesh->n[a] % opts->tiles[a]) {
                noalloc_msg(errbuf, errlen, "axis %d: need n >= 1, hi > lo and tiles dividing n", a);
                return KIN_EINVAL;
            }
            c.n[a] = mesh->n[a];
            c.lo[a] = mesh->lo[a];
            c.hi[a] = mesh->hi[a];
            c.h[a] = (mesh->hi[a] - mesh->lo[a]) / mesh->n[a];
            c.tiles[a] = opts->tiles[a];
            c.L[a] = c.n[a] / c.tiles[a];
        } else {
            if (mesh->n[a] > 1) {
                noalloc_msg(errbuf, errlen, "axis %d beyond dim must have n = 1", a);
                return KIN_EINVAL;
            }
            c.n[a] = 1;
            c.tiles[a] = 1;
            c.L[a] = 1;
        }
        c.cells *= c.n[a];
    }
    c.nodes = c.cells * c.NN;
    if (opts->block[0] || opts->block[1] || opts->block[2]) {
        for (int a = 0; a < 3; ++a) {
            int b = a < c.dim ? opts->block[a] : 1;
            if (b < 1 || c.L[a] % b) {
                noalloc_msg(errbuf, errlen, "axis %d: block %d must divide the subdomain extent %d", a, b, c.L[a]);
                return KIN_EINVAL;
            }
            c.B[a] = b;
        }
    } else {
        choose_block(&c, c.B);
    }
    for (int a = 0; a < 3; ++a) {
        c.nblk[a] = c.n[a] / c.B[a];
        c.nb[a] = c.L[a] / c.B[a];
    }
    const size_t smem = block_smem(&c, c.B);
    if (smem > 227 * 1024) {
        noalloc_msg(errbuf, errlen, "cell block needs %zu bytes of shared memory (> 227 KB)", smem);
        return KIN_EINVAL;
    }
    c.kfn = pick_kernel(c.dim, degree, c.system, c.precision);
    size_t tn = 1;
    for (int a = 1; a < c.dim; ++a) tn *= c.NP;
    size_t stride = 0, rstride = 0;
    for (int a = 0; a < c.dim; ++a) {
        stride = std::max(stride, (size_t)c.nblk[a] * (c.cells / c.n[a]) * tn);
        rstride = std::max(rstride, (size_t)c.tiles[a] * (c.cells / c.n[a]) * tn);
    }
    c.sig_stride = stride;
    c.raw_stride = rstride;

    // scratch layout: c64 | c32 | gll | error word | sig0 | raw0 | sig1 | raw1
    const size_t off_c64 = 0;
    const size_t off_c32 = align256(off_c64 + sizeof(double) * 6 * kCoefStride);
    const size_t off_gll = align256(off_c32 + sizeof(float) * 6 * kCoefStride);
    const size_t off_err = align256(off_gll + sizeof(double) * 2 * kMaxNP);
    const size_t off_sum = align256(off_err + sizeof(int) * 4);
    const size_t sbytes = align256(stride * c.npop * c.esize);
    const size_t rbytes = align256(rstride * c.npop * c.esize);
    const size_t need = off_sum + 2 * sbytes + 2 * rbytes;
    if (need > kNoallocScratchBytes) {
        noalloc_msg(errbuf, errlen,
                    "problem needs %zu bytes of scratch; kin_step_noalloc is limited to %zu bytes "
                    "(use kin_create for larger problems)", need, kNoallocScratchBytes);
        return KIN_EINVAL;
    }

    // per-device address of the static scratch (first call on each device)
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kNoallocMaxDevices) {
        noalloc_msg(errbuf, errlen, "cudaGetDevice failed or device ordinal out of range");
        return KIN_ECUDA;
    }
    unsigned char* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_addr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                noalloc_msg(errbuf, errlen, "cudaGetSymbolAddress(g_noalloc_scratch) failed: %s",
                            cudaGetErrorString(e));
                return KIN_ECUDA;
            }
            g_noalloc_addr[dev] = p;
        }
        base = static_cast<unsigned char*>(g_noalloc_addr[dev]);
    }
    c.f = f;
    c.c64 = reinterpret_cast<double*>(base + off_c64);
    c.coef = c.esize == 4 ? (void*)(base + off_c32) : (void*)c.c64;
    c.gll = reinterpret_cast<double*>(base + off_gll);
    c.errword = reinterpret_cast<int*>(base + off_err);
    c.sig[0] = base + off_sum;
    c.raw[0] = base + off_sum + sbytes;
    c.sig[1] = base + off_sum + sbytes + rbytes;
    c.raw[1] = base + off_sum + 2 * sbytes + rbytes;
    c.cur = 0;

    e = configure_launch(&c);
    if (e != cudaSuccess) {
        noalloc_msg(errbuf, errlen, "launch configuration failed: %s", cudaGetErrorString(e));
        return KIN_ECUDA;
    }
    SetupArgs sa;
    memset(&sa, 0, sizeof sa);
    sa.dim = c.dim;
    sa.degree = degree;
    sa.lambda = c.lambda;
    sa.dt = dt;
    for (int a = 0; a < 3; ++a) {
        sa.h[a] = c.h[a];
        sa.B[a] = c.B[a];
    }
    sa.c64 = c.c64;
    sa.c32 = c.esize == 4 ? (float*)c.coef : nullptr;
    sa.gll = c.gll;
    // the error word must start at zero; everything else is written before it is read
    e = cudaMemsetAsync(c.errword, 0, sizeof(int) * 4, c.stream);
    if (e == cudaSuccess) e = launch_setup(sa, c.stream);
    // the block-inverse records travel in the launch parameters
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c.coef_host, c.c64, sizeof(c.coef_host), cudaMemcpyDeviceToHost, c.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    // summaries of the caller's state, then nsteps full steps (every scratch
    // region is written before it is read, so nothing needs clearing)
    for (int s = 0; e == cudaSuccess && s <= nsteps; ++s) {
        Inst I = make_inst(&c, s == 0 ? 1 : 0);
        void* args[] = {&I};
        e = cudaLaunchKernel((const void*)c.kfn, dim3(c.grid), dim3(c.threads), args, (size_t)c.smem,
                             c.stream);
        c.cur ^= 1;
    }
    if (e != cudaSuccess) {
        noalloc_msg(errbuf, errlen, "kernel launch failed: %s", cudaGetErrorString(e));
        return KIN_ECUDA;
    }
    int word = 0;
    e = cudaMemcpyAsync(&word, c.errword, sizeof(int), cudaMemcpyDeviceToHost, c.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    if (e != cudaSuccess) {
        noalloc_msg(errbuf, errlen, "step failed: %s", cudaGetErrorString(e));
        return KIN_ECUDA;
    }
    if (word) {
        noalloc_msg(errbuf, errlen, "a bounded device wait ran out (error word 0x%x)", word);
        return KIN_ETIMEOUT;
    }
    return KIN_OK;
}
