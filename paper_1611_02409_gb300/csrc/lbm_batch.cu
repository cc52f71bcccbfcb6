// Batched independent instances (include/lbm.h, lbm_batch_*): one persistent launch per
// time step walks a device work list of chunks over every active instance; walls, the
// buffer flip, per-instance FP64 residuals and the work-list compaction are small
// kernels; a window of `check_every` steps is captured once into a CUDA graph and
// replayed.  The per-cell arithmetic is the single-instance code (collide_store and
// wall_column), so a batched instance reproduces lbm_step bit for bit.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "dispatch.cuh"

#include <nvtx3/nvToolsExt.h>

namespace lbm {
namespace batch {

constexpr int LAT = LAT_D2Q37;
constexpr int ST = ST_FP32;
constexpr int Q = Lattice<LAT>::Q;
using KP = KParams<LAT>;
constexpr int kThreads = 128;
// Work items a block takes in a row (at most) before moving on by the grid's stride:
// consecutive items mostly share an instance (its parameters stay staged), while the
// resident blocks together sweep one band of the work list at a time (DRAM locality).
// Measured with 128-cell items: 16 against 2, 4, 8, 32 and one contiguous range per block
// (a 4096^2 instance 9.07 GLUPS against 8.63 contiguous; 64 x 512^2 and 256 uneven squares
// 9.96-9.98).
constexpr int kGroup = 16;

struct Inst {
    long long buf[2];   // float offsets of the two population buffers in the arena
    long long snap;     // float offset of the residual snapshot (2 nx ny floats)
    int ncomp;          // fluid cells updated per step (nx * ny_comp)
    int cur, active, walls, have_snap, steps;
    double residual;
    WallParams wp;
};

// One chunk of `CPT` x 128 consecutive fluid cells (row-major over the computed rows) of
// one instance per work item; each block takes kGroup consecutive items at a time (mostly
// of one instance, whose launch parameters are staged in shared memory whenever the item's
// instance changes), then moves on by the grid's stride.  REF: some instance of the batch has
// a reference state (the step with the reference's shifts, zero for the others).
template <int CPT, bool REF>
__global__ void __launch_bounds__(kThreads, 4) k_bstep(const Inst *__restrict__ inst, const KP *__restrict__ kps,
                                                       const int2 *__restrict__ work, const int *__restrict__ nwork,
                                                       float *__restrict__ arena)
{
    __shared__ __align__(16) long long skp_raw[(sizeof(KP) + 7) / 8];
    const KP &kp = *reinterpret_cast<const KP *>(skp_raw);
    const int nw = nwork[0];
    // kGroup items at a time where the list gives every block several groups, fewer on
    // short lists (each block still gets about four groups)
    const int grp = max(1, min(kGroup, nw / (4 * (int)gridDim.x)));
    int cached = -1;
    for (int w = blockIdx.x * grp; w < nw; w += (w % grp == grp - 1) ? ((int)gridDim.x - 1) * grp + 1 : 1) {
        const int2 it = work[w];
        if (it.x != cached) {
            __syncthreads();
            const long long *srcp = reinterpret_cast<const long long *>(kps + it.x);
            for (int k = threadIdx.x; k < (int)((sizeof(KP) + 7) / 8); k += kThreads) skp_raw[k] = srcp[k];
            __syncthreads();
            cached = it.x;
        }
        const Inst &d = inst[it.x];
        const int cur = d.cur, walls = d.walls, ncomp = d.ncomp;
        const float *src = arena + d.buf[cur];
        float *dst = arena + d.buf[cur ^ 1];
        const int nx = kp.nx, ny = kp.ny, gh = kp.gh, plane = (int)kp.plane;
        const int sx = nx < 4, sy = ny < 4;
#pragma unroll 1
        for (int c = 0; c < CPT; ++c) {
            const int cell = it.y * (kThreads * CPT) + c * kThreads + threadIdx.x;
            if (cell >= ncomp) break;
            const int x = cell % nx;
            const int y = kp.y0 + cell / nx;
            // the plane stride is opaque per cell, so the 2Q products I * plane are formed
            // where they are used instead of being hoisted out of the loop into registers
            int pl = plane;
            asm volatile("" : "+r"(pl));
            // source rows (as element offsets) and columns of the 7 stencil displacements
            // -3..3; an instance's 2Q planes span < 2^31 elements
            int rowo[7], col[7];
            static_for<0, 7>([&](auto KK) {
                constexpr int C = decltype(KK)::value - 3;
                const int ys = walls ? y - C + gh : wrap_sub<C>(y, ny, sy);
                rowo[KK] = ys * nx;
                col[KK] = wrap_sub<C>(x, nx, sx);
            });
            float s[Q], t[Q];
            static_for<0, Q>([&](auto II) {
                constexpr int I = decltype(II)::value;
                constexpr int cx = cv<LAT, I, 0>(), cy = cv<LAT, I, 1>();
                const int idx = rowo[cy + 3] + col[cx + 3];
                s[I] = __ldg(src + (I * pl + idx));
                t[I] = __ldg(src + ((Q + I) * pl + idx));
            });
            const int o = (y + gh) * nx + x;
            collide_store<LAT, ST, REF>(kp, ArrayPop{s, t}, dst, o, StrideOff<4>{pl});
        }
    }
}

// Walls of every active channel on its freshly written buffer, then the buffer flip and
// step count of every active instance: one block per instance, which touches only its
// own buffer and record, so walls and flip need no ordering across blocks.
__global__ void k_bwalls_flip(Inst *__restrict__ inst, const KP *__restrict__ kps, float *arena)
{
    Inst &d = inst[blockIdx.x];
    if (!d.active) return;
    if (d.walls) {
        const KP &kp = kps[blockIdx.x];
        float *buf = arena + d.buf[d.cur ^ 1];
        for (int j = threadIdx.x; j < 2 * kp.nx; j += blockDim.x)
            wall_column<LAT, ST>(buf, kp, d.wp, j % kp.nx, j / kp.nx);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        d.cur ^= 1;
        d.steps += 1;
    }
}

// Residual max_{X in u_x, T} ||X - X_prev|| / (m ||X||) of every active instance, FP64
// sums in a fixed order (deterministic).  Stage 1: block (i, k) sums chunk k (kResChunk
// cells) of instance i into partials[i][k] and refreshes the snapshot of its cells;
// stage 2: one thread per instance adds its chunks' partials in order and decides;
// below `tol` the instance becomes inactive.
constexpr int kResThreads = 256;
constexpr int kResChunk = 16 * kResThreads;

__global__ void __launch_bounds__(kResThreads) k_bresid_part(const Inst *__restrict__ inst, const KP *__restrict__ kps,
                                                             float *arena, int maxchunks, double *partials)
{
    const Inst &d = inst[blockIdx.x];
    if (!d.active) return;
    const KP &kp = kps[blockIdx.x];
    const int n = kp.nx * kp.ny;
    const int f0 = blockIdx.y * kResChunk;
    if (f0 >= n) return;
    const int f1 = min(n, f0 + kResChunk);
    const float *buf = arena + d.buf[d.cur];
    float *snap = arena + d.snap;
    const int have = d.have_snap;
    double a[4] = {0, 0, 0, 0};
    for (int f = f0 + threadIdx.x; f < f1; f += kResThreads) {
        const int x = f % kp.nx, y = f / kp.nx;
        float s[Q], t[Q];
        load_cell<LAT, ST>(buf, kp, (long long)(y + kp.gh) * kp.nx + x, s, t);
        RawMoments<2> mo;
        raw_moments<LAT>(kp, ArrayPop{s, t}, mo);
        CellState<2> c;
        cell_state<LAT>(kp, mo, c);
        const float ux = c.u[0], th = c.th_eq;
        if (have) {
            const double du = (double)ux - snap[f], dT = (double)th - snap[n + f];
            a[0] += du * du;
            a[2] += dT * dT;
        }
        a[1] += (double)ux * ux;
        a[3] += (1.0 + th) * (1.0 + th);
        snap[f] = ux;
        snap[n + f] = th;
    }
    __shared__ double sh[kResThreads / 32][4];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const double x = warp_sum(a[v]);
        if (lane == 0) sh[wid][v] = x;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double t = 0.0;
        for (int w = 0; w < kResThreads / 32; ++w) t += sh[w][threadIdx.x];
        partials[((long long)blockIdx.x * maxchunks + blockIdx.y) * 4 + threadIdx.x] = t;
    }
}

__global__ void k_bresid_final(Inst *inst, const KP *__restrict__ kps, int n_inst, int maxchunks,
                               const double *__restrict__ partials, int m, double tol)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_inst) return;
    Inst &d = inst[i];
    if (!d.active) return;
    const int n = kps[i].nx * kps[i].ny;
    const int nch = (n + kResChunk - 1) / kResChunk;
    double t[4] = {0, 0, 0, 0};
    for (int k = 0; k < nch; ++k)
        for (int v = 0; v < 4; ++v) t[v] += partials[((long long)i * maxchunks + k) * 4 + v];
    // a non-finite field makes its sums NaN (the comparisons below would read those as
    // zero): report NaN and stop the instance
    const bool bad = isnan(t[0]) || isnan(t[1]) || isnan(t[2]) || isnan(t[3]);
    if (bad) {
        d.residual = NAN;
        d.active = 0;
    } else if (d.have_snap) {
        const double ru = t[1] > 0 ? sqrt(t[0] / t[1]) : (t[0] > 0 ? INFINITY : 0.0);
        const double rT = t[3] > 0 ? sqrt(t[2] / t[3]) : 0.0;
        d.residual = fmax(ru, rT) / m;
        if (d.residual < tol) d.active = 0;  // converged
    } else {
        d.residual = INFINITY;
        d.have_snap = 1;
    }
}

// Work list: offsets of every active instance's chunks, then the items themselves.
__global__ void k_bwork_offsets(const Inst *inst, int n, int tile, int *off, int *nwork)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int acc = 0, act = 0;
        for (int i = 0; i < n; ++i) {
            off[i] = acc;
            if (inst[i].active) {
                acc += (inst[i].ncomp + tile - 1) / tile;
                act++;
            }
        }
        nwork[0] = acc;
        nwork[1] = act;
    }
}

__global__ void k_bwork_fill(const Inst *inst, int tile, const int *off, int2 *work)
{
    const int i = blockIdx.x;
    if (!inst[i].active) return;
    const int nc = (inst[i].ncomp + tile - 1) / tile;
    for (int j = threadIdx.x; j < nc; j += blockDim.x) work[off[i] + j] = make_int2(i, j);
}

__global__ void k_bcount(const Inst *inst, int n, int *nwork)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int act = 0;
        for (int i = 0; i < n; ++i) act += inst[i].active;
        nwork[1] = act;
    }
}

} // namespace batch
} // namespace lbm

using namespace lbm;
using namespace lbm::batch;

struct lbm_batch {
    int n = 0;
    std::vector<Ctx> ctx;
    std::vector<Inst> inst0;       // host image at creation
    Inst *d_inst = nullptr;
    KP *d_kp = nullptr;
    float *d_arena = nullptr;
    size_t arena_elems = 0;
    int2 *d_work = nullptr;
    int *d_off = nullptr;
    double *d_rpart = nullptr;      // residual partial sums [instance][chunk][4]
    int maxchunks = 1;
    int *d_nwork = nullptr;
    int *h_nwork = nullptr;         // pinned
    cudaStream_t stream = nullptr;
    cudaGraphExec_t exec = nullptr;
    int g_tile = 0, g_window = 0;
    double g_tol = 0.0;
    int tile = 128;                 // cells per work item
    bool ref = false;               // some instance has a reference state
    int num_sms = 0;
    std::string err;
};

namespace {

int bfail(lbm_batch *b, int code, const std::string &m)
{
    if (b) b->err = m;
    return set_global_error(code, m.c_str());
}

#define LBM_BCK(b, call)                                                                                       \
    do {                                                                                                       \
        cudaError_t e_ = (call);                                                                               \
        if (e_ != cudaSuccess) return bfail(b, LBM_ERR_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
    } while (0)

using StepFn = void (*)(const Inst *, const KP *, const int2 *, const int *, float *);

StepFn step_kernel(int tile, bool ref)
{
    if (ref) return tile == 512 ? k_bstep<4, true> : tile == 256 ? k_bstep<2, true> : k_bstep<1, true>;
    return tile == 512 ? k_bstep<4, false> : tile == 256 ? k_bstep<2, false> : k_bstep<1, false>;
}

int step_grid(int tile, bool ref, int num_sms)
{
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, step_kernel(tile, ref), kThreads, 0);
    return (nb > 0 ? nb : 1) * num_sms;
}

void launch_window(lbm_batch *b, int window, double tol, int tile)
{
    const int n = b->n;
    // persistent grid: the resident blocks of every SM, but no more than the work items
    // of all instances (the work list only shrinks as instances converge)
    long long items = 0;
    for (const Inst &in : b->inst0) items += (in.ncomp + tile - 1) / tile;
    const int grid = (int)std::max(1LL, std::min((long long)step_grid(tile, b->ref, b->num_sms), items));
    const StepFn kstep = step_kernel(tile, b->ref);
    k_bwork_offsets<<<1, 32, 0, b->stream>>>(b->d_inst, n, tile, b->d_off, b->d_nwork);
    k_bwork_fill<<<n, 128, 0, b->stream>>>(b->d_inst, tile, b->d_off, b->d_work);
    for (int s = 0; s < window; ++s) {
        kstep<<<grid, kThreads, 0, b->stream>>>(b->d_inst, b->d_kp, b->d_work, b->d_nwork, b->d_arena);
        k_bwalls_flip<<<n, 64, 0, b->stream>>>(b->d_inst, b->d_kp, b->d_arena);
    }
    k_bresid_part<<<dim3(n, b->maxchunks), kResThreads, 0, b->stream>>>(b->d_inst, b->d_kp, b->d_arena,
                                                                         b->maxchunks, b->d_rpart);
    k_bresid_final<<<(n + 127) / 128, 128, 0, b->stream>>>(b->d_inst, b->d_kp, n, b->maxchunks, b->d_rpart, window,
                                                           tol);
    k_bcount<<<1, 32, 0, b->stream>>>(b->d_inst, n, b->d_nwork);
}

int ensure_graph(lbm_batch *b, int window, double tol, int tile)
{
    if (b->exec && b->g_window == window && b->g_tol == tol && b->g_tile == tile) return LBM_OK;
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    cudaGraph_t g;
    LBM_BCK(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    launch_window(b, window, tol, tile);
    LBM_BCK(b, cudaStreamEndCapture(b->stream, &g));
    cudaError_t e = cudaGraphInstantiate(&b->exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return bfail(b, LBM_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    b->g_window = window;
    b->g_tol = tol;
    b->g_tile = tile;
    return LBM_OK;
}

int reset_state(lbm_batch *b)
{
    LBM_BCK(b, cudaMemsetAsync(b->d_arena, 0, b->arena_elems * sizeof(float), b->stream));
    LBM_BCK(b, cudaMemcpyAsync(b->d_inst, b->inst0.data(), sizeof(Inst) * b->n, cudaMemcpyHostToDevice, b->stream));
    LBM_BCK(b, cudaStreamSynchronize(b->stream));
    return LBM_OK;
}

} // namespace

extern "C" {

int lbm_batch_create(int n, const lbm_params *params, lbm_batch **out)
{
    if (!out || !params || n < 1) return set_global_error(LBM_ERR_ARG, "need n >= 1 parameter sets");
    *out = nullptr;
    lbm_batch *b = new lbm_batch();
    b->n = n;
    b->ctx.resize(n);
    b->inst0.resize(n);
    std::vector<KP> kps(n);
    size_t off = 0;
    auto align = [](size_t v) { return (v + 63) & ~(size_t)63; };
    size_t max_items = 0;
    for (int i = 0; i < n; ++i) {
        const lbm_params &p = params[i];
        if (p.lattice != LBM_D2Q37 || p.storage != LBM_FP32 || p.bc_x != LBM_PERIODIC) {
            delete b;
            return set_global_error(LBM_ERR_ARG, "batched instances are D2Q37, FP32 storage, periodic in x");
        }
        int D, Qd;
        double r;
        int rc = make_ctx(p, b->ctx[i], &D, &Qd, &r);
        if (rc != LBM_OK && rc != LBM_WARN_PR_RANGE) {
            delete b;
            return rc;
        }
        Ctx &c = b->ctx[i];
        // the step kernel forms an instance's element offsets (p * plane + cell, p < 2 Q) in
        // 32-bit integers
        if ((long long)2 * Q * c.plane >= (1LL << 31)) {
            delete b;
            return set_global_error(LBM_ERR_ARG, "a batched instance's 2 Q planes must hold fewer than 2^31 values");
        }
        kps[i] = make_kparams<LAT>(c);
        b->ref = b->ref || has_reference(c);
        Inst &in = b->inst0[i];
        memset(&in, 0, sizeof(in));
        const size_t pop = (size_t)2 * Q * c.plane;
        in.buf[0] = (long long)off;
        off = align(off + pop);
        in.buf[1] = (long long)off;
        off = align(off + pop);
        in.snap = (long long)off;
        off = align(off + (size_t)2 * c.nx * c.ny);
        in.ncomp = c.nx * (c.walls ? c.ny - 2 : c.ny);
        in.walls = c.walls;
        in.active = 1;
        in.residual = std::numeric_limits<double>::infinity();
        for (int bb = 0; bb < 2; ++bb) {
            for (int d = 0; d < 3; ++d) in.wp.vw[bb][d] = (float)(c.wall_u[bb][d] / c.r);
            in.wp.thw[bb] = (float)(c.wall_T[bb] - 1.0);
        }
        max_items += (in.ncomp + kThreads - 1) / kThreads;
        b->maxchunks = std::max(b->maxchunks, (c.nx * c.ny + kResChunk - 1) / kResChunk);
    }
    b->arena_elems = off;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_arena, b->arena_elems * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_inst, sizeof(Inst) * n);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_kp, sizeof(KP) * n);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_work, sizeof(int2) * (max_items + 1));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_off, sizeof(int) * n);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_rpart, sizeof(double) * 4 * n * (size_t)b->maxchunks);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_nwork, sizeof(int) * 2);
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_nwork, sizeof(int) * 2);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_kp, kps.data(), sizeof(KP) * n, cudaMemcpyHostToDevice, b->stream);
    if (e != cudaSuccess) {
        int code = set_global_error(LBM_ERR_NOMEM, (std::string("batch allocation: ") + cudaGetErrorString(e)).c_str());
        lbm_batch_destroy(b);
        return code;
    }
    int rc = reset_state(b);
    if (rc) {
        lbm_batch_destroy(b);
        return rc;
    }
    *out = b;
    return LBM_OK;
}

int lbm_batch_destroy(lbm_batch *b)
{
    if (!b) return LBM_OK;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    cudaFree(b->d_arena);
    cudaFree(b->d_inst);
    cudaFree(b->d_kp);
    cudaFree(b->d_work);
    cudaFree(b->d_off);
    cudaFree(b->d_rpart);
    cudaFree(b->d_nwork);
    if (b->h_nwork) cudaFreeHost(b->h_nwork);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
    return LBM_OK;
}

int lbm_batch_init_fields(lbm_batch *b, int i, const double *rho, const double *u, const double *T, int mem)
{
    return lbm_batch_init_fields_neq(b, i, rho, u, T, nullptr, nullptr, mem);
}

int lbm_batch_init_fields_neq(lbm_batch *b, int i, const double *rho, const double *u, const double *T,
                              const double *Pi, const double *q, int mem)
{
    if (!b || i < 0 || i >= b->n || !rho || !u || !T) return bfail(b, LBM_ERR_ARG, "bad instance or null field");
    const Ctx &c = b->ctx[i];
    const size_t n = (size_t)c.nx * c.ny;
    Inst in;
    LBM_BCK(b, cudaMemcpyAsync(&in, b->d_inst + i, sizeof(Inst), cudaMemcpyDeviceToHost, b->stream));
    LBM_BCK(b, cudaStreamSynchronize(b->stream));
    const double *dr = rho, *du = u, *dT = T, *dP = Pi, *dq = q;
    double *stage = nullptr;
    if (mem == LBM_MEM_HOST) {
        LBM_BCK(b, cudaMalloc(&stage, sizeof(double) * n * 9));
        LBM_BCK(b, cudaMemcpyAsync(stage, rho, sizeof(double) * n, cudaMemcpyHostToDevice, b->stream));
        LBM_BCK(b, cudaMemcpyAsync(stage + n, u, sizeof(double) * n * 2, cudaMemcpyHostToDevice, b->stream));
        LBM_BCK(b, cudaMemcpyAsync(stage + 3 * n, T, sizeof(double) * n, cudaMemcpyHostToDevice, b->stream));
        dr = stage;
        du = stage + n;
        dT = stage + 3 * n;
        dP = dq = nullptr;
        if (Pi) {
            LBM_BCK(b, cudaMemcpyAsync(stage + 4 * n, Pi, sizeof(double) * n * 3, cudaMemcpyHostToDevice, b->stream));
            dP = stage + 4 * n;
        }
        if (q) {
            LBM_BCK(b, cudaMemcpyAsync(stage + 7 * n, q, sizeof(double) * n * 2, cudaMemcpyHostToDevice, b->stream));
            dq = stage + 7 * n;
        }
    }
    Launch<LAT, ST>::init_neq(c, b->d_arena + in.buf[in.cur], dr, du, dT, dP, dq, b->stream);
    // wall and ghost rows from the initial fluid rows, as lbm_init_fields does
    if (c.walls) Launch<LAT, ST>::walls(c, b->d_arena + in.buf[in.cur], b->stream);
    in.active = 1;
    in.steps = 0;
    in.have_snap = 0;
    in.residual = std::numeric_limits<double>::infinity();
    LBM_BCK(b, cudaMemcpyAsync(b->d_inst + i, &in, sizeof(Inst), cudaMemcpyHostToDevice, b->stream));
    LBM_BCK(b, cudaStreamSynchronize(b->stream));
    if (stage) cudaFree(stage);
    LBM_BCK(b, cudaGetLastError());
    return LBM_OK;
}

static int batch_run(lbm_batch *b, int max_steps, double tol, int check_every, int *steps_taken)
{
    // a window of check_every steps is captured as one CUDA graph (two nodes per step)
    if (!b || max_steps < 0 || check_every < 1 || check_every > 100000)
        return bfail(b, LBM_ERR_ARG, "need max_steps >= 0 and 1 <= check_every <= 100000");
    int rc = ensure_graph(b, check_every, tol, b->tile);
    if (rc) return rc;
    int done = 0;
    while (done < max_steps) {
        LBM_BCK(b, cudaGraphLaunch(b->exec, b->stream));
        done += check_every;
        LBM_BCK(b, cudaMemcpyAsync(b->h_nwork, b->d_nwork, sizeof(int) * 2, cudaMemcpyDeviceToHost, b->stream));
        LBM_BCK(b, cudaStreamSynchronize(b->stream));
        if (b->h_nwork[1] == 0) break;
    }
    if (steps_taken) *steps_taken = done;
    return LBM_OK;
}

int lbm_batch_run(lbm_batch *b, int max_steps, double tol, int check_every, int *steps_taken)
{
    nvtxRangePushA("lbm_batch_run");  // NVTX range over the whole run (profilers)
    const int rc = batch_run(b, max_steps, tol, check_every, steps_taken);
    nvtxRangePop();
    return rc;
}

int lbm_batch_status(lbm_batch *b, int *steps, double *residual, int *active)
{
    if (!b) return LBM_ERR_ARG;
    std::vector<Inst> h(b->n);
    LBM_BCK(b, cudaMemcpyAsync(h.data(), b->d_inst, sizeof(Inst) * b->n, cudaMemcpyDeviceToHost, b->stream));
    LBM_BCK(b, cudaStreamSynchronize(b->stream));
    for (int i = 0; i < b->n; ++i) {
        if (steps) steps[i] = h[i].steps;
        if (residual) residual[i] = h[i].residual;
        if (active) active[i] = h[i].active;
    }
    return LBM_OK;
}

int lbm_batch_activate(lbm_batch *b, int i)
{
    if (!b || i >= b->n) return bfail(b, LBM_ERR_ARG, "bad instance");
    std::vector<Inst> h(b->n);
    LBM_BCK(b, cudaMemcpyAsync(h.data(), b->d_inst, sizeof(Inst) * b->n, cudaMemcpyDeviceToHost, b->stream));
    LBM_BCK(b, cudaStreamSynchronize(b->stream));
    for (int k = 0; k < b->n; ++k) {
        if ((i >= 0 && k != i) || std::isnan(h[k].residual)) continue;
        h[k].active = 1;
        h[k].have_snap = 0;
        h[k].residual = std::numeric_limits<double>::infinity();
    }
    LBM_BCK(b, cudaMemcpyAsync(b->d_inst, h.data(), sizeof(Inst) * b->n, cudaMemcpyHostToDevice, b->stream));
    LBM_BCK(b, cudaStreamSynchronize(b->stream));
    return LBM_OK;
}

int lbm_batch_moments(lbm_batch *b, int i, double *rho, double *u, double *T, double *Pi, double *q, int mem)
{
    if (!b || i < 0 || i >= b->n) return bfail(b, LBM_ERR_ARG, "bad instance");
    const Ctx &c = b->ctx[i];
    Inst in;
    LBM_BCK(b, cudaMemcpyAsync(&in, b->d_inst + i, sizeof(Inst), cudaMemcpyDeviceToHost, b->stream));
    LBM_BCK(b, cudaStreamSynchronize(b->stream));
    const size_t n = (size_t)c.nx * c.ny;
    const float *buf = b->d_arena + in.buf[in.cur];
    if (mem == LBM_MEM_HOST) {
        double *stage = nullptr;
        LBM_BCK(b, cudaMalloc(&stage, sizeof(double) * n * 9));
        double *sr = stage, *su = stage + n, *sT = stage + 3 * n, *sP = stage + 4 * n, *sq = stage + 7 * n;
        Launch<LAT, ST>::moments(c, buf, sr, su, sT, sP, sq, b->stream);
        if (rho) LBM_BCK(b, cudaMemcpyAsync(rho, sr, sizeof(double) * n, cudaMemcpyDeviceToHost, b->stream));
        if (u) LBM_BCK(b, cudaMemcpyAsync(u, su, sizeof(double) * n * 2, cudaMemcpyDeviceToHost, b->stream));
        if (T) LBM_BCK(b, cudaMemcpyAsync(T, sT, sizeof(double) * n, cudaMemcpyDeviceToHost, b->stream));
        if (Pi) LBM_BCK(b, cudaMemcpyAsync(Pi, sP, sizeof(double) * n * 3, cudaMemcpyDeviceToHost, b->stream));
        if (q) LBM_BCK(b, cudaMemcpyAsync(q, sq, sizeof(double) * n * 2, cudaMemcpyDeviceToHost, b->stream));
        LBM_BCK(b, cudaStreamSynchronize(b->stream));
        cudaFree(stage);
    } else {
        Launch<LAT, ST>::moments(c, buf, rho, u, T, Pi, q, b->stream);
        LBM_BCK(b, cudaStreamSynchronize(b->stream));
    }
    LBM_BCK(b, cudaGetLastError());
    return LBM_OK;
}

int lbm_batch_autotune(lbm_batch *b, int steps, int *chosen)
{
    if (!b || steps < 1 || steps > 100000) return bfail(b, LBM_ERR_ARG, "need 1 <= steps <= 100000");
    cudaEvent_t e0, e1;
    LBM_BCK(b, cudaEventCreate(&e0));
    LBM_BCK(b, cudaEventCreate(&e1));
    const int tiles[3] = {128, 256, 512};
    float best = -1.f;
    int best_tile = 128;
    for (int k = 0; k < 3; ++k) {
        int rc = reset_state(b);
        if (rc) return rc;
        rc = ensure_graph(b, steps, -1.0, tiles[k]);  // tol < 0: nothing converges
        if (rc) return rc;
        LBM_BCK(b, cudaGraphLaunch(b->exec, b->stream));  // warm-up replay
        LBM_BCK(b, cudaEventRecord(e0, b->stream));
        LBM_BCK(b, cudaGraphLaunch(b->exec, b->stream));
        LBM_BCK(b, cudaEventRecord(e1, b->stream));
        LBM_BCK(b, cudaEventSynchronize(e1));
        float ms = 0.f;
        LBM_BCK(b, cudaEventElapsedTime(&ms, e0, e1));
        if (best < 0 || ms < best) {
            best = ms;
            best_tile = tiles[k];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->tile = best_tile;
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    int rc = reset_state(b);
    if (rc) return rc;
    if (chosen) *chosen = best_tile;
    return LBM_OK;
}

} // extern "C"
