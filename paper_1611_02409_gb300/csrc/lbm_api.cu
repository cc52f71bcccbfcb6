// C ABI of the library (declared in include/lbm.h): handle lifetime, parameter mapping,
// buffers, and the host side of every entry point.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "kernels.cuh"

#include <nvtx3/nvToolsExt.h>

namespace {
// NVTX range over one entry point (visible in profilers; no cost without one attached)
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};
} // namespace
#include "ops.h"

struct lbm_handle {
    lbm_params p;
    int D, Q;
    double r;
    int c[128][3];
    double w[128];
    double Nf, omega, nuG, tau_s, tau_q;
    lbm::Ctx ctx;
    lbm::Ops ops;
    cudaStream_t stream;
    size_t elem;           // bytes per stored population
    size_t buf_elems;      // elements per population buffer (2 Q planes)
    void *buf[2];
    int cur;
    long long steps;
    // scratch
    double *d_partials;
    int diag_blocks;
    double *d_out;
    double *h_out;         // pinned
    void *d_snap;          // u_x and T - 1 of the previous diagnostics call (storage's arithmetic type)
    int have_snap;
    long long snap_step;
    int *d_err;            // [0] error word of the kernels' bounded waits, [1] fault injection
    double *d_stage;       // device staging for host-memory field I/O
    size_t stage_bytes;
    std::string err;
};

// The measured-fastest variant for the configuration (GB300, 4096^2 / 256^3 workloads):
// paired cells for 16-bit storage on the 2-D lattice (even rows), the two-pass kernel for
// the 3-D lattice and D2Q77 (their 206 and 154 values per cell do not fit the register
// file), else direct.
static int default_kernel(const lbm_handle *h)
{
    if (h->ops.paired_ok(h->ctx)) return LBM_KERNEL_PAIRED;
    if (h->D == 3 || h->p.lattice == LBM_D2Q77 || h->p.storage == LBM_FP64) return LBM_KERNEL_TWOPASS;
    return LBM_KERNEL_DIRECT;
}


namespace {

thread_local std::string g_create_err;

int set_err(lbm_handle *h, int code, const std::string &msg)
{
    if (h) h->err = msg;
    else g_create_err = msg;
    return code;
}

int cuda_fail(lbm_handle *h, cudaError_t e, const char *what)
{
    return set_err(h, LBM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define LBM_CK(h, call)                                                                                        \
    do {                                                                                                       \
        cudaError_t e_ = (call);                                                                               \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, #call);                                                 \
    } while (0)

long long ncell(const lbm_handle *h) { return (long long)h->p.nx * h->p.ny * h->p.nz; }

int ensure_stage(lbm_handle *h, size_t bytes)
{
    if (h->stage_bytes >= bytes) return LBM_OK;
    if (h->d_stage) cudaFree(h->d_stage);
    h->d_stage = nullptr;
    h->stage_bytes = 0;
    cudaError_t e = cudaMalloc(&h->d_stage, bytes);
    if (e != cudaSuccess) return set_err(h, LBM_ERR_NOMEM, std::string("staging allocation: ") + cudaGetErrorString(e));
    h->stage_bytes = bytes;
    return LBM_OK;
}

} // namespace

namespace lbm {
__global__ void __launch_bounds__(kDiagThreads) k_diag_final(const double *__restrict__ partials, int nblk,
                                                              double *out)
{
    double acc[kDiagNV];
#pragma unroll
    for (int v = 0; v < kDiagNV; ++v) acc[v] = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x)
#pragma unroll
        for (int v = 0; v < kDiagNV; ++v) acc[v] += partials[(long long)b * kDiagNV + v];
    block_sums(acc, out);
}

void launch_diag_final(const double *partials, int nblk, double *out, cudaStream_t st)
{
    k_diag_final<<<1, kDiagThreads, 0, st>>>(partials, nblk, out);
}

int set_global_error(int code, const char *msg) { return set_err(nullptr, code, msg); }
} // namespace lbm

extern "C" {

const char *lbm_last_error(const lbm_handle *h) { return h ? h->err.c_str() : g_create_err.c_str(); }

struct Mapped {
    int D;
    double Nf, omega, nuG, tau_s, tau_q;
    bool warn;
};

// Validation and parameter mapping shared by lbm_create and lbm_map_params.
static int map_params(const lbm_params &p, Mapped &m)
{
    if (p.lattice == LBM_D2Q37 || p.lattice == LBM_D2Q33 || p.lattice == LBM_D2Q77) m.D = 2;
    else if (p.lattice == LBM_D3Q103) m.D = 3;
    else return set_err(nullptr, LBM_ERR_ARG, "unknown lattice");
    const int D = m.D;
    if (p.nx < 1 || p.ny < 1 || (D == 3 && p.nz < 1)) return set_err(nullptr, LBM_ERR_ARG, "grid sizes must be >= 1");
    if ((long long)p.nx * p.ny * (D == 3 ? p.nz : 1) > (1LL << 31) - 1)
        return set_err(nullptr, LBM_ERR_ARG, "grid too large");
    // the kernels launch one block row per stored row (gridDim.y, walls add four ghost
    // rows) and one block layer per plane (gridDim.z), each at most 65535
    if (p.ny + (p.bc_y == LBM_WALLS ? 4 : 0) > 65535 || (D == 3 && p.nz > 65535))
        return set_err(nullptr, LBM_ERR_ARG, "ny (plus 4 ghost rows with walls) and nz must not exceed 65535");
    if (p.bc_y != LBM_PERIODIC && p.bc_y != LBM_WALLS) return set_err(nullptr, LBM_ERR_ARG, "bad bc_y");
    if (p.bc_y == LBM_WALLS && (p.lattice == LBM_D2Q33 || p.lattice == LBM_D2Q77 || p.ny < 5))
        return set_err(nullptr, LBM_ERR_ARG, "walls need D2Q37 or D3Q103 and ny >= 5");
    if (p.bc_x != LBM_PERIODIC && p.bc_x != LBM_OPEN) return set_err(nullptr, LBM_ERR_ARG, "bad bc_x");
    if (p.bc_x == LBM_OPEN && D != 2) return set_err(nullptr, LBM_ERR_ARG, "open x ends need D = 2");
    if (p.storage < LBM_FP32 || p.storage > LBM_FP64) return set_err(nullptr, LBM_ERR_ARG, "bad storage");
    if (p.storage == LBM_FP64 && p.lattice != LBM_D2Q37 && p.lattice != LBM_D3Q103)
        return set_err(nullptr, LBM_ERR_ARG, "FP64 storage is built for D2Q37 and D3Q103");
    if (p.pr_mode != LBM_PR_SHIFTED && p.pr_mode != LBM_PR_LITERAL) return set_err(nullptr, LBM_ERR_ARG, "bad pr_mode");
    if (!(p.Pr > 0) || !(p.tau > 0.5) || !(p.kappa > 0) || !(p.kappa <= 1))
        return set_err(nullptr, LBM_ERR_ARG, "need Pr > 0, tau > 1/2, 0 < kappa <= 1");
    // Eq. Gamma: N_f = 2/(gamma - 1) - D
    double Nf = p.gamma > 0 ? 2.0 / (p.gamma - 1.0) - D : p.N_f;
    if (p.gamma > 0 && !(p.gamma > 1.0)) return set_err(nullptr, LBM_ERR_ARG, "gamma must exceed 1");
    if (Nf < -1e-12 || !std::isfinite(Nf)) return set_err(nullptr, LBM_ERR_ARG, "N_f < 0 (gamma above (D+2)/D)");
    if (Nf < 0) Nf = 0;
    if (p.kappa == 1.0 && std::fabs(p.Pr - 1.0) > 1e-12)
        return set_err(nullptr, LBM_ERR_ARG, "kappa = 1 leaves no freedom for Pr != 1");
    if (p.bc_y == LBM_WALLS && !(p.wall_T[0] > 0 && p.wall_T[1] > 0))
        return set_err(nullptr, LBM_ERR_ARG, "wall temperatures must be > 0");
    if (!(p.rho0 == 0 || (p.rho0 > 0 && std::isfinite(p.rho0))) || !(p.T0 == 0 || (p.T0 > 0 && std::isfinite(p.T0))))
        return set_err(nullptr, LBM_ERR_ARG, "reference state: rho0 and T0 must be > 0 (or 0 for 1)");
    if (p.pr_mode == LBM_PR_LITERAL) {
        m.omega = p.Pr / p.tau;             // rate Pr/tau_f (Eq. DiscreteReductionG)
        m.tau_s = p.tau;
        m.tau_q = p.tau / p.Pr;
        m.nuG = p.kappa < 1 ? (1.0 - 1.0 / p.Pr) / (1.0 - p.kappa) : 0.0; // 1 - nu + kappa nu = 1/Pr
    } else {
        m.tau_s = p.tau;
        m.tau_q = 0.5 + (p.tau - 0.5) / p.Pr; // viscosity / conductivity ratio = Pr
        m.omega = 1.0 / m.tau_q;
        m.nuG = p.kappa < 1 ? (1.0 - m.tau_q / m.tau_s) / (1.0 - p.kappa) : 0.0;
    }
    if (!(m.omega > 0 && m.omega < 2)) return set_err(nullptr, LBM_ERR_ARG, "relaxation rate outside (0, 2)");
    m.Nf = Nf;
    m.warn = m.nuG < -0.5;
    return LBM_OK;
}

} // extern "C"

namespace lbm {
// Validates p and fills c (host fields only: geometry, coefficients, lattice weights)
// as lbm_create does; D and Q receive the lattice dimensions.  Returns an LBM status.
int make_ctx(const lbm_params &pin, Ctx &c, int *D_out, int *Q_out, double *r_out)
{
    lbm_params p = pin;
    Mapped mp;
    int rc = map_params(p, mp);
    if (rc) return rc;
    if (mp.D == 2) p.nz = 1;
    int cc[128][3];
    double w[128], r;
    const int Q = derive_lattice(p.lattice, cc, w, &r);
    if (Q < 0) return set_err(nullptr, LBM_ERR_ARG, "lattice derivation failed");
    memset(&c, 0, sizeof(c));
    c.storage = p.storage;
    c.walls = p.bc_y == LBM_WALLS;
    c.open_x = p.bc_x == LBM_OPEN;
    c.nx = p.nx;
    c.ny = p.ny;
    c.nz = p.nz;
    c.gh = c.walls ? 2 : 0;
    c.nys = p.ny + 2 * c.gh;
    c.plane = (long long)p.nx * c.nys * p.nz;
    c.omega = mp.omega;
    c.kappa = p.kappa;
    c.a_tr = (1.0 - p.kappa) * (1.0 - mp.nuG);
    c.a_sig = (1.0 - p.kappa) * mp.nuG;
    c.Nf = mp.Nf;
    c.r = r;
    for (int i = 0; i < Q; ++i) c.w[i] = w[i];
    for (int b = 0; b < 2; ++b) {
        for (int d = 0; d < 3; ++d) c.wall_u[b][d] = p.wall_u[b][d];
        c.wall_T[b] = p.wall_T[b];
    }
    c.rho0 = p.rho0 == 0 ? 1.0 : p.rho0;
    c.T0 = p.T0 == 0 ? 1.0 : p.T0;
    c.kernel = 1;
    if (D_out) *D_out = mp.D;
    if (Q_out) *Q_out = Q;
    if (r_out) *r_out = r;
    return mp.warn ? LBM_WARN_PR_RANGE : LBM_OK;
}
} // namespace lbm

extern "C" {

int lbm_map_params(const lbm_params *p, double *out)
{
    if (!p || !out) return set_err(nullptr, LBM_ERR_ARG, "null argument");
    Mapped m;
    int rc = map_params(*p, m);
    if (rc) return rc;
    out[0] = m.Nf;
    out[1] = m.omega;
    out[2] = m.nuG;
    out[3] = m.tau_s;
    out[4] = m.tau_q;
    out[5] = p->kappa;
    return m.warn ? LBM_WARN_PR_RANGE : LBM_OK;
}

int lbm_lattice_table(int lattice, int *D, int *Q, double *r, int *c, double *w)
{
    int cc[128][3];
    double ww[128], rr;
    int q = lbm::derive_lattice(lattice, cc, ww, &rr);
    if (q < 0) return set_err(nullptr, LBM_ERR_ARG, "unknown lattice");
    if (D) *D = lattice == LBM_D3Q103 ? 3 : 2;
    if (Q) *Q = q;
    if (r) *r = rr;
    for (int i = 0; i < q; ++i) {
        if (c)
            for (int d = 0; d < 3; ++d) c[3 * i + d] = cc[i][d];
        if (w) w[i] = ww[i];
    }
    return LBM_OK;
}

int lbm_lattice_unit_scale(int lattice, double *r)
{
    if (!r) return set_err(nullptr, LBM_ERR_ARG, "null r");
    return lbm_lattice_table(lattice, nullptr, nullptr, r, nullptr, nullptr);
}

int lbm_create(const lbm_params *pin, void *stream, lbm_handle **out)
{
    NvtxRange nvtx_("lbm_create");
    g_create_err.clear();
    if (!pin || !out) return set_err(nullptr, LBM_ERR_ARG, "null argument");
    *out = nullptr;
    lbm_params p = *pin;
    Mapped mp;
    int rc = map_params(p, mp);
    if (rc) return rc;
    const int D = mp.D;
    if (D == 2) p.nz = 1;
    const double Nf = mp.Nf, omega = mp.omega, nuG = mp.nuG, tau_s = mp.tau_s, tau_q = mp.tau_q;
    lbm_handle *h = new lbm_handle();
    h->p = p;
    h->D = D;
    h->Q = lbm::derive_lattice(p.lattice, h->c, h->w, &h->r);
    if (h->Q < 0) {
        delete h;
        return set_err(nullptr, LBM_ERR_ARG, "lattice derivation failed");
    }
    h->Nf = Nf;
    h->omega = omega;
    h->nuG = nuG;
    h->tau_s = tau_s;
    h->tau_q = tau_q;
    h->stream = (cudaStream_t)stream;
    lbm::Ctx &c = h->ctx;
    memset(&c, 0, sizeof(c));
    c.storage = p.storage;
    c.walls = p.bc_y == LBM_WALLS;
    c.open_x = p.bc_x == LBM_OPEN;
    c.nx = p.nx;
    c.ny = p.ny;
    c.nz = p.nz;
    c.gh = c.walls ? 2 : 0;
    c.nys = p.ny + 2 * c.gh;
    c.plane = (long long)p.nx * c.nys * p.nz;
    c.omega = omega;
    c.kappa = p.kappa;
    c.a_tr = (1.0 - p.kappa) * (1.0 - nuG);
    c.a_sig = (1.0 - p.kappa) * nuG;
    c.Nf = Nf;
    c.r = h->r;
    for (int i = 0; i < h->Q; ++i) c.w[i] = h->w[i];
    for (int b = 0; b < 2; ++b) {
        for (int d = 0; d < 3; ++d) c.wall_u[b][d] = p.wall_u[b][d];
        c.wall_T[b] = p.wall_T[b];
    }
    c.rho0 = p.rho0 == 0 ? 1.0 : p.rho0;
    c.T0 = p.T0 == 0 ? 1.0 : p.T0;
    h->ops = lbm::ops_for(p.lattice, p.storage);
    h->elem = (size_t)lbm::storage_bytes(p.storage);
    h->buf_elems = (size_t)2 * h->Q * (size_t)c.plane;
    for (int k = 0; k < 2; ++k) {
        cudaError_t e = cudaMalloc(&h->buf[k], h->buf_elems * h->elem);
        if (e != cudaSuccess) {
            int code = set_err(nullptr, LBM_ERR_NOMEM, std::string("population buffer: ") + cudaGetErrorString(e));
            if (k) cudaFree(h->buf[0]);
            delete h;
            return code;
        }
    }
    const long long n = ncell(h);
    h->diag_blocks = (int)std::min<long long>((n + lbm::kDiagThreads - 1) / lbm::kDiagThreads, 1216);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&h->ctx.num_sms, cudaDevAttrMultiProcessorCount, dev);
    h->ctx.kernel = default_kernel(h);
    cudaError_t e = cudaMalloc(&h->d_partials, sizeof(double) * lbm::kDiagNV * (h->diag_blocks + 1));
    if (e == cudaSuccess) e = cudaMalloc(&h->d_err, 2 * sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_err, 0, 2 * sizeof(int), h->stream);
    if (e == cudaSuccess) h->ctx.d_err = h->d_err;
    if (e == cudaSuccess) e = cudaMallocHost(&h->h_out, sizeof(double) * lbm::kDiagNV);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->buf[0], 0, h->buf_elems * h->elem, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->buf[1], 0, h->buf_elems * h->elem, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        int code = set_err(nullptr, LBM_ERR_CUDA, std::string("create: ") + cudaGetErrorString(e));
        lbm_destroy(h);
        return code;
    }
    h->d_out = h->d_partials + (size_t)lbm::kDiagNV * h->diag_blocks;
    *out = h;
    if (nuG < -0.5) {
        h->err = "Gaussian parameter nu < -1/2 (outside the paper's Pr range)";
        return LBM_WARN_PR_RANGE;
    }
    return LBM_OK;
}

int lbm_destroy(lbm_handle *h)
{
    if (!h) return LBM_OK;
    cudaStreamSynchronize(h->stream);
    for (int k = 0; k < 2; ++k)
        if (h->buf[k]) cudaFree(h->buf[k]);
    if (h->d_partials) cudaFree(h->d_partials);
    if (h->d_err) cudaFree(h->d_err);
    if (h->h_out) cudaFreeHost(h->h_out);
    if (h->d_snap) cudaFree(h->d_snap);
    if (h->d_stage) cudaFree(h->d_stage);
    delete h;
    return LBM_OK;
}

int lbm_lattice_info(const lbm_handle *h, int *D, int *Q, double *r, int *c, double *w)
{
    if (!h) return LBM_ERR_ARG;
    if (D) *D = h->D;
    if (Q) *Q = h->Q;
    if (r) *r = h->r;
    for (int i = 0; i < h->Q; ++i) {
        if (c)
            for (int d = 0; d < 3; ++d) c[3 * i + d] = h->c[i][d];
        if (w) w[i] = h->w[i];
    }
    return LBM_OK;
}

int lbm_coefficients(const lbm_handle *h, double *out)
{
    if (!h || !out) return LBM_ERR_ARG;
    out[0] = h->Nf;
    out[1] = h->omega;
    out[2] = h->nuG;
    out[3] = h->tau_s;
    out[4] = h->tau_q;
    out[5] = h->p.kappa;
    return LBM_OK;
}

int lbm_init_fields(lbm_handle *h, const double *rho, const double *u, const double *T, int mem)
{
    if (!h || !rho || !u || !T) return set_err(h, LBM_ERR_ARG, "null field");
    const long long n = ncell(h);
    const double *dr = rho, *du = u, *dT = T;
    if (mem == LBM_MEM_HOST) {
        int rc = ensure_stage(h, sizeof(double) * n * (h->D + 2));
        if (rc) return rc;
        double *s = h->d_stage;
        LBM_CK(h, cudaMemcpyAsync(s, rho, sizeof(double) * n, cudaMemcpyHostToDevice, h->stream));
        LBM_CK(h, cudaMemcpyAsync(s + n, u, sizeof(double) * n * h->D, cudaMemcpyHostToDevice, h->stream));
        LBM_CK(h, cudaMemcpyAsync(s + n * (1 + h->D), T, sizeof(double) * n, cudaMemcpyHostToDevice, h->stream));
        dr = s;
        du = s + n;
        dT = s + n * (1 + h->D);
    } else if (mem != LBM_MEM_DEVICE) {
        return set_err(h, LBM_ERR_ARG, "bad mem");
    }
    h->ops.init(h->ctx, h->buf[h->cur], dr, du, dT, h->stream);
    // the wall and ghost rows from the initial fluid rows, as after every step: the first
    // streaming then exchanges mass with the walls in balance (reading R6)
    if (h->ctx.walls) h->ops.walls(h->ctx, h->buf[h->cur], h->stream);
    LBM_CK(h, cudaGetLastError());
    h->steps = 0;
    h->have_snap = 0;
    return LBM_OK;
}

int lbm_init_fields_neq(lbm_handle *h, const double *rho, const double *u, const double *T, const double *Pi,
                        const double *q, int mem)
{
    NvtxRange nvtx_("lbm_init_fields_neq");
    if (!h || !rho || !u || !T) return set_err(h, LBM_ERR_ARG, "null field");
    const long long n = ncell(h);
    const int D = h->D, np = D * (D + 1) / 2;
    const double *dr = rho, *du = u, *dT = T, *dP = Pi, *dq = q;
    if (mem == LBM_MEM_HOST) {
        int rc = ensure_stage(h, sizeof(double) * n * (2 + D + np + D));
        if (rc) return rc;
        double *s = h->d_stage;
        LBM_CK(h, cudaMemcpyAsync(s, rho, sizeof(double) * n, cudaMemcpyHostToDevice, h->stream));
        LBM_CK(h, cudaMemcpyAsync(s + n, u, sizeof(double) * n * D, cudaMemcpyHostToDevice, h->stream));
        LBM_CK(h, cudaMemcpyAsync(s + n * (1 + D), T, sizeof(double) * n, cudaMemcpyHostToDevice, h->stream));
        dr = s;
        du = s + n;
        dT = s + n * (1 + D);
        dP = dq = nullptr;
        if (Pi) {
            LBM_CK(h, cudaMemcpyAsync(s + n * (2 + D), Pi, sizeof(double) * n * np, cudaMemcpyHostToDevice, h->stream));
            dP = s + n * (2 + D);
        }
        if (q) {
            LBM_CK(h, cudaMemcpyAsync(s + n * (2 + D + np), q, sizeof(double) * n * D, cudaMemcpyHostToDevice,
                                      h->stream));
            dq = s + n * (2 + D + np);
        }
    } else if (mem != LBM_MEM_DEVICE) {
        return set_err(h, LBM_ERR_ARG, "bad mem");
    }
    h->ops.init_neq(h->ctx, h->buf[h->cur], dr, du, dT, dP, dq, h->stream);
    if (h->ctx.walls) h->ops.walls(h->ctx, h->buf[h->cur], h->stream);
    LBM_CK(h, cudaGetLastError());
    h->steps = 0;
    h->have_snap = 0;
    return LBM_OK;
}

} // extern "C"

namespace {
// FP32 fields widened to the FP64 the initialisation takes.
__global__ void k_widen(const float *__restrict__ s, double *__restrict__ d, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        d[i] = (double)s[i];
}
} // namespace

extern "C" {

int lbm_init_fields_typed(lbm_handle *h, const void *rho, const void *u, const void *T, const void *Pi,
                          const void *q, int dtype, int mem)
{
    if (!h || !rho || !u || !T) return set_err(h, LBM_ERR_ARG, "null field");
    if (dtype == LBM_DTYPE_F64)
        return lbm_init_fields_neq(h, (const double *)rho, (const double *)u, (const double *)T, (const double *)Pi,
                                   (const double *)q, mem);
    if (dtype != LBM_DTYPE_F32) return set_err(h, LBM_ERR_ARG, "bad dtype");
    if (mem != LBM_MEM_HOST && mem != LBM_MEM_DEVICE) return set_err(h, LBM_ERR_ARG, "bad mem");
    const long long n = ncell(h);
    const int D = h->D, np = D * (D + 1) / 2;
    const void *in[5] = {rho, u, T, Pi, q};
    const long long cnt[5] = {n, D * n, n, np * n, D * n};
    long long off[5], total = 0;
    for (int k = 0; k < 5; ++k) {
        off[k] = total;
        if (in[k]) total += cnt[k];
    }
    const double *out[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    if (mem == LBM_MEM_HOST) {
        std::vector<double> wide((size_t)total);
        for (int k = 0; k < 5; ++k) {
            if (!in[k]) continue;
            const float *s = static_cast<const float *>(in[k]);
            for (long long i = 0; i < cnt[k]; ++i) wide[(size_t)(off[k] + i)] = (double)s[i];
            out[k] = wide.data() + off[k];
        }
        // pageable host memory: the staged copies have left `wide` when the call returns
        return lbm_init_fields_neq(h, out[0], out[1], out[2], out[3], out[4], LBM_MEM_HOST);
    }
    int rc = ensure_stage(h, sizeof(double) * (size_t)total);
    if (rc) return rc;
    for (int k = 0; k < 5; ++k) {
        if (!in[k]) continue;
        double *d = h->d_stage + off[k];
        const int blocks = (int)std::min<long long>((cnt[k] + 255) / 256, 4096);
        k_widen<<<blocks, 256, 0, h->stream>>>(static_cast<const float *>(in[k]), d, cnt[k]);
        out[k] = d;
    }
    LBM_CK(h, cudaGetLastError());
    return lbm_init_fields_neq(h, out[0], out[1], out[2], out[3], out[4], LBM_MEM_DEVICE);
}

int lbm_step(lbm_handle *h, int nsteps)
{
    NvtxRange nvtx_("lbm_step");
    if (!h || nsteps < 0) return set_err(h, LBM_ERR_ARG, "bad nsteps");
    for (int k = 0; k < nsteps; ++k) {
        void *src = h->buf[h->cur], *dst = h->buf[h->cur ^ 1];
        h->ops.step(h->ctx, src, dst, h->stream);
        if (h->ctx.walls) h->ops.walls(h->ctx, dst, h->stream);
        h->cur ^= 1;
    }
    h->steps += nsteps;
    LBM_CK(h, cudaGetLastError());
    return LBM_OK;
}

// Reads the device error word after a synchronisation; clears it.
static int check_device_error(lbm_handle *h)
{
    int v = 0;
    LBM_CK(h, cudaMemcpy(&v, h->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (v) {
        LBM_CK(h, cudaMemset(h->d_err, 0, sizeof(int)));
        return set_err(h, LBM_ERR_TIMEOUT, "a device-side wait gave up; results of the affected steps are invalid");
    }
    return LBM_OK;
}

int lbm_moments(lbm_handle *h, double *rho, double *u, double *T, double *Pi, double *q, int mem)
{
    NvtxRange nvtx_("lbm_moments");
    if (!h) return LBM_ERR_ARG;
    const long long n = ncell(h);
    const int D = h->D, np = D * (D + 1) / 2;
    if (mem == LBM_MEM_HOST) {
        int rc = ensure_stage(h, sizeof(double) * n * (1 + D + 1 + np + D));
        if (rc) return rc;
        double *s = h->d_stage;
        double *sr = s, *su = s + n, *sT = s + n * (1 + D), *sP = s + n * (2 + D), *sq = s + n * (2 + D + np);
        h->ops.moments(h->ctx, h->buf[h->cur], rho ? sr : nullptr, u ? su : nullptr, T ? sT : nullptr,
                       Pi ? sP : nullptr, q ? sq : nullptr, h->stream);
        LBM_CK(h, cudaGetLastError());
        if (rho) LBM_CK(h, cudaMemcpyAsync(rho, sr, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream));
        if (u) LBM_CK(h, cudaMemcpyAsync(u, su, sizeof(double) * n * D, cudaMemcpyDeviceToHost, h->stream));
        if (T) LBM_CK(h, cudaMemcpyAsync(T, sT, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream));
        if (Pi) LBM_CK(h, cudaMemcpyAsync(Pi, sP, sizeof(double) * n * np, cudaMemcpyDeviceToHost, h->stream));
        if (q) LBM_CK(h, cudaMemcpyAsync(q, sq, sizeof(double) * n * D, cudaMemcpyDeviceToHost, h->stream));
    } else if (mem == LBM_MEM_DEVICE) {
        h->ops.moments(h->ctx, h->buf[h->cur], rho, u, T, Pi, q, h->stream);
        LBM_CK(h, cudaGetLastError());
    } else {
        return set_err(h, LBM_ERR_ARG, "bad mem");
    }
    LBM_CK(h, cudaStreamSynchronize(h->stream));
    return check_device_error(h);
}

int lbm_diagnostics(lbm_handle *h, double *out)
{
    NvtxRange nvtx_("lbm_diagnostics");
    if (!h || !out) return set_err(h, LBM_ERR_ARG, "null argument");
    const long long n = ncell(h);
    const size_t snap_elem = h->p.storage == LBM_FP64 ? sizeof(double) : sizeof(float);
    if (!h->d_snap) LBM_CK(h, cudaMalloc(&h->d_snap, snap_elem * 2 * n));
    h->ops.diag(h->ctx, h->buf[h->cur], h->d_snap, h->have_snap, h->d_partials, h->diag_blocks, h->stream);
    lbm::launch_diag_final(h->d_partials, h->diag_blocks, h->d_out, h->stream);
    LBM_CK(h, cudaGetLastError());
    LBM_CK(h, cudaMemcpyAsync(h->h_out, h->d_out, sizeof(double) * lbm::kDiagNV, cudaMemcpyDeviceToHost, h->stream));
    LBM_CK(h, cudaStreamSynchronize(h->stream));
    {
        int rc = check_device_error(h);
        if (rc) return rc;
    }
    const double *a = h->h_out;
    out[0] = (double)n + a[0];
    out[1] = a[1];
    out[2] = a[2];
    out[3] = h->D == 3 ? a[3] : 0.0;
    out[4] = (double)n * 0.5 * (h->D + h->Nf) + a[4];
    const long long m = h->steps - h->snap_step;
    out[5] = 0.0;
    if (h->have_snap && m > 0) {
        double ru = a[6] > 0 ? std::sqrt(a[5] / a[6]) : 0.0;
        double rT = a[8] > 0 ? std::sqrt(a[7] / a[8]) : 0.0;
        out[5] = std::max(ru, rT) / (double)m;
    }
    out[6] = a[9];
    out[7] = (double)h->steps;
    h->have_snap = 1;
    h->snap_step = h->steps;
    if (a[9] > 0) return set_err(h, LBM_ERR_UNSTABLE, "non-finite or non-positive density / temperature");
    return LBM_OK;
}

int lbm_debug_inject_stall(lbm_handle *h, int on)
{
    if (!h) return LBM_ERR_ARG;
    const int v = on ? 1 : 0;
    LBM_CK(h, cudaMemcpyAsync(h->d_err + 1, &v, sizeof(int), cudaMemcpyHostToDevice, h->stream));
    LBM_CK(h, cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

int lbm_set_kernel(lbm_handle *h, int variant)
{
    if (!h) return LBM_ERR_ARG;
    if (variant == LBM_KERNEL_AUTO) variant = default_kernel(h);
    if (variant == LBM_KERNEL_STAGED && !h->ops.staged_ok(h->ctx))
        return set_err(h, LBM_ERR_ARG, "staged kernel needs D = 2 and nx a multiple of 128");
    if (variant == LBM_KERNEL_PAIRED && !h->ops.paired_ok(h->ctx))
        return set_err(h, LBM_ERR_ARG, "paired kernel needs D = 2, 16-bit storage and nx even");
    if (variant < LBM_KERNEL_DIRECT || variant > LBM_KERNEL_TWOPASS) return set_err(h, LBM_ERR_ARG, "bad variant");
    if (h->p.storage == LBM_FP64 && variant != LBM_KERNEL_TWOPASS)
        return set_err(h, LBM_ERR_ARG, "FP64 storage runs on the two-pass kernel only");
    h->ctx.kernel = variant;
    return LBM_OK;
}

int lbm_autotune(lbm_handle *h, int steps, int *chosen)
{
    if (!h || steps < 1) return set_err(h, LBM_ERR_ARG, "bad arguments");
    cudaEvent_t e0, e1;
    LBM_CK(h, cudaEventCreate(&e0));
    LBM_CK(h, cudaEventCreate(&e1));
    float best = -1.f;
    int best_v = LBM_KERNEL_DIRECT;
    for (int v = LBM_KERNEL_DIRECT; v <= LBM_KERNEL_TWOPASS; ++v) {
        if (v == LBM_KERNEL_STAGED && !h->ops.staged_ok(h->ctx)) continue;
        if (v == LBM_KERNEL_PAIRED && !h->ops.paired_ok(h->ctx)) continue;
        if (h->p.storage == LBM_FP64 && v != LBM_KERNEL_TWOPASS) continue;
        h->ctx.kernel = v;
        int rc = lbm_step(h, 2);
        if (rc) return rc;
        LBM_CK(h, cudaEventRecord(e0, h->stream));
        rc = lbm_step(h, steps);
        if (rc) return rc;
        LBM_CK(h, cudaEventRecord(e1, h->stream));
        LBM_CK(h, cudaEventSynchronize(e1));
        float ms = 0.f;
        LBM_CK(h, cudaEventElapsedTime(&ms, e0, e1));
        if (best < 0 || ms < best) {
            best = ms;
            best_v = v;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    {
        int rc = check_device_error(h);
        if (rc) return rc;
    }
    h->ctx.kernel = best_v;
    LBM_CK(h, cudaMemsetAsync(h->buf[0], 0, h->buf_elems * h->elem, h->stream));
    LBM_CK(h, cudaMemsetAsync(h->buf[1], 0, h->buf_elems * h->elem, h->stream));
    LBM_CK(h, cudaStreamSynchronize(h->stream));
    h->steps = 0;
    h->have_snap = 0;
    if (chosen) *chosen = best_v;
    return LBM_OK;
}

int lbm_get_populations(lbm_handle *h, double *g, double *hh, int mem)
{
    if (!h) return LBM_ERR_ARG;
    const size_t bytes = sizeof(double) * (size_t)h->Q * (size_t)ncell(h);
    if (mem == LBM_MEM_HOST) {
        int rc = ensure_stage(h, 2 * bytes);
        if (rc) return rc;
        double *sg = h->d_stage, *sh = h->d_stage + bytes / sizeof(double);
        h->ops.get_pops(h->ctx, h->buf[h->cur], sg, sh, h->stream);
        LBM_CK(h, cudaGetLastError());
        if (g) LBM_CK(h, cudaMemcpyAsync(g, sg, bytes, cudaMemcpyDeviceToHost, h->stream));
        if (hh) LBM_CK(h, cudaMemcpyAsync(hh, sh, bytes, cudaMemcpyDeviceToHost, h->stream));
    } else {
        h->ops.get_pops(h->ctx, h->buf[h->cur], g, hh, h->stream);
        LBM_CK(h, cudaGetLastError());
    }
    LBM_CK(h, cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

int lbm_set_populations(lbm_handle *h, const double *g, const double *hh, int mem)
{
    if (!h || !g || !hh) return set_err(h, LBM_ERR_ARG, "null argument");
    const size_t bytes = sizeof(double) * (size_t)h->Q * (size_t)ncell(h);
    const double *dg = g, *dh = hh;
    if (mem == LBM_MEM_HOST) {
        int rc = ensure_stage(h, 2 * bytes);
        if (rc) return rc;
        double *sg = h->d_stage, *sh = h->d_stage + bytes / sizeof(double);
        LBM_CK(h, cudaMemcpyAsync(sg, g, bytes, cudaMemcpyHostToDevice, h->stream));
        LBM_CK(h, cudaMemcpyAsync(sh, hh, bytes, cudaMemcpyHostToDevice, h->stream));
        dg = sg;
        dh = sh;
    }
    h->ops.set_pops(h->ctx, h->buf[h->cur], dg, dh, h->stream);
    // ghost rows are a function of the domain rows: rebuild them
    if (h->ctx.walls) h->ops.walls(h->ctx, h->buf[h->cur], h->stream);
    LBM_CK(h, cudaGetLastError());
    LBM_CK(h, cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

} // extern "C"
