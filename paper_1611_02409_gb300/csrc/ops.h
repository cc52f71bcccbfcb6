// Plain host-side interface between the C-ABI layer and the per-lattice kernel units.
#pragma once
#include <cuda_runtime.h>

namespace lbm {

struct Ctx {
    int storage, walls;
    int nx, ny, nz, nys, gh;
    long long plane;       // stored cells per population plane
    double omega, kappa, a_tr, a_sig, Nf, r;
    double w[128];
    double wall_u[2][3], wall_T[2];
    int *d_err;            // device error word (bounded waits that gave up set it)
    int open_x;            // open (zero-gradient) x ends
    int num_sms;
    int kernel;            // LBM_KERNEL_*: 1 direct, 2 staged, 3 paired, 4 two-pass
    double rho0, T0;       // reference state of the stored deviations
};

// Bytes of one stored population in storage form LBM_FP32 (0), LBM_FP16 (1), LBM_BF16 (2)
// or LBM_FP64 (3).
inline int storage_bytes(int storage) { return storage == 0 ? 4 : storage == 3 ? 8 : 2; }

struct Ops {
    void (*init)(const Ctx &, void *dst, const double *rho, const double *u, const double *T, cudaStream_t);
    void (*init_neq)(const Ctx &, void *dst, const double *rho, const double *u, const double *T, const double *Pi,
                     const double *q, cudaStream_t);
    void (*step)(const Ctx &, const void *src, void *dst, cudaStream_t);
    void (*walls)(const Ctx &, void *buf, cudaStream_t);
    void (*moments)(const Ctx &, const void *buf, double *rho, double *u, double *T, double *Pi, double *q,
                    cudaStream_t);
    void (*diag)(const Ctx &, const void *buf, void *snap, int have_snap, double *partials, int nblk,
                 cudaStream_t);   // snap: 2 n values of the storage's arithmetic type
    void (*get_pops)(const Ctx &, const void *buf, double *g, double *h, cudaStream_t);
    void (*set_pops)(const Ctx &, void *buf, const double *g, const double *h, cudaStream_t);
    bool (*staged_ok)(const Ctx &);
    bool (*paired_ok)(const Ctx &);
};

Ops ops_d2q37_fp32();
Ops ops_d2q37_fp16();
Ops ops_d2q37_bf16();
Ops ops_d3q103_fp32();
Ops ops_d3q103_fp16();
Ops ops_d3q103_bf16();
Ops ops_d2q33_fp32();
Ops ops_d2q33_fp16();
Ops ops_d2q33_bf16();
Ops ops_d2q77_fp32();
Ops ops_d2q77_fp16();
Ops ops_d2q77_bf16();
Ops ops_d2q37_fp64();
Ops ops_d3q103_fp64();

// The launch table of a lattice (LBM_D2Q37 = 1, LBM_D3Q103 = 2, LBM_D2Q33 = 3, LBM_D2Q77 = 4)
// and storage form (FP64 storage: D2Q37 and D3Q103 only, checked by the caller).
inline Ops ops_for(int lattice, int storage)
{
    if (storage == 3) return lattice == 2 ? ops_d3q103_fp64() : ops_d2q37_fp64();
    if (lattice == 1) return storage == 1 ? ops_d2q37_fp16() : storage == 2 ? ops_d2q37_bf16() : ops_d2q37_fp32();
    if (lattice == 3) return storage == 1 ? ops_d2q33_fp16() : storage == 2 ? ops_d2q33_bf16() : ops_d2q33_fp32();
    if (lattice == 4) return storage == 1 ? ops_d2q77_fp16() : storage == 2 ? ops_d2q77_bf16() : ops_d2q77_fp32();
    return storage == 1 ? ops_d3q103_fp16() : storage == 2 ? ops_d3q103_bf16() : ops_d3q103_fp32();
}
void launch_diag_final(const double *partials, int nblk, double *out, cudaStream_t st);

}  // namespace lbm
struct lbm_params;
namespace lbm {
// Validation + mapping + lattice as lbm_create does it (lbm_api.cu).
int make_ctx(const lbm_params &p, Ctx &c, int *D, int *Q, double *r);

// Sets the handle-free error text (lbm_last_error(NULL)) and returns `code`.
int set_global_error(int code, const char *msg);

// FP64 lattice derivation (lattice_host.cu): fills c (Q x 3), w (Q) and r; returns Q or -1.
int derive_lattice(int lattice, int (*c)[3], double *w, double *r);

} // namespace lbm
