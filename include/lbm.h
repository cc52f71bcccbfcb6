/*
 * lbm.h — C ABI of the GB300 (sm_103a) polyatomic ES-BGK lattice Boltzmann library.
 *
 * The scheme is that of Hu, Zhang, Du, Jin, Kong, "A lattice Boltzmann scheme with
 * arbitrary Prandtl number and specific heat ratio based on the polyatomic ES-BGK model"
 * (arXiv 1611.02409).  Each step pull-streams the mass populations g_i and the energy
 * populations h_i, takes their moments, builds the ES-BGK Gaussian from the general
 * Hermite-coefficient formula truncated at fourth order, relaxes both sets toward it and
 * applies the walls (Sec. V, Eqs. DiscreteReductionG and DiscreteReductionH).
 *
 * Conventions shared by every entry point
 *   - Return value: LBM_OK (0) or an LBM_ERR_* code; LBM_WARN_PR_RANGE (> 0 but not an
 *     error) from lbm_create.  The text of the last error is lbm_last_error(handle).
 *   - Units are the paper's dimensionless ones (Sec. V, "dimensionless variables"):
 *     theta_0 = R_g T_0 = 1, so the sound speed of the isothermal gas is sqrt(T); the
 *     lattice maps xi_i = r c_i with integer c_i, so one lattice spacing per time step is
 *     r (lbm_lattice_info).  Lattice kinematic viscosity: (T/r^2)(tau - 1/2).
 *   - Fields are SoA, [component][z][y][x] row-major, x fastest, over the Nx x Ny (x Nz)
 *     domain, in double precision.  Pointers are device pointers unless the call's
 *     `mem` argument is LBM_MEM_HOST; the caller owns them.
 *   - The library owns the population buffers (allocated in lbm_create, freed in
 *     lbm_destroy).  All device work is queued on the stream given to lbm_create;
 *     lbm_step returns before the GPU finishes.  Device-side failures surface at the
 *     next synchronising call (lbm_moments, lbm_diagnostics).
 *   - A handle is not thread-safe.
 */
#ifndef LBM_H
#define LBM_H

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define LBM_OK 0
#define LBM_ERR_ARG 1        /* invalid argument or inadmissible parameters        */
#define LBM_ERR_CUDA 2       /* a CUDA call failed (text in lbm_last_error)         */
#define LBM_ERR_UNSTABLE 3   /* non-finite or non-positive density / temperature    */
#define LBM_ERR_NOMEM 4      /* device allocation failed                            */
#define LBM_ERR_TIMEOUT 5    /* a bounded device-side wait gave up (the step's data
                                are not valid); the context stays usable             */
#define LBM_WARN_PR_RANGE 100 /* Gaussian parameter nu < -1/2: outside the paper's
                                2/3 <= Pr bound for its literal mapping (Sec. III)  */

/* lattices: Sec. VI Table D2Q37; D3Q103 is this library's 3-D degree-9 lattice
 * (shells 000,100,111,200,210,220,222,300,311,333 at the D2Q37 scale r) */
#define LBM_D2Q37 1
#define LBM_D3Q103 2
/* Shim's D2Q33 (Sec. VI B, Table D2Q33: shells (0,0) (1,0) (1,1) (2,0) (2,2) (3,0) (2,1)
 * (4,4), reach 4; the shock-tube lattice): its own scale r (the root of its degree-9
 * moment system, printed as 0.819381 sqrt(2)); no walls; direct and two-pass kernels. */
#define LBM_D2Q33 3
/* D2Q77, this library's degree-13 lattice for the sixth-order (Burnett) expansion of
 * Sec. IV (a^(5), a^(6)), which the paper names but prints no lattice for: shells (0,0)
 * (1,0) (1,1) (2,0) (2,1) (2,2) (3,0) (3,1) (3,2) (3,3) (4,0) (4,1) (4,4) (5,0) (5,3),
 * reach 5, its own scale r = 0.97000849874 (the root of its degree-13 moment system); the
 * equilibrium is expanded to order 6.  Periodic or open x ends, no walls; two-pass
 * (default) and direct kernels. */
#define LBM_D2Q77 4

/* parameter mapping (Sec. III Eq. Pr, Sec. V Eq. DiscreteReductionG):
 *   LBM_PR_SHIFTED: tau_s = tau, tau_q = (tau - 1/2)/Pr + 1/2, omega = 1/tau_q and the
 *                   Gaussian's nu from 1 - nu + kappa nu = tau_q/tau_s, so the lattice
 *                   viscosity / conductivity ratio is the set Pr;
 *   LBM_PR_LITERAL: omega = Pr/tau and 1 - nu + kappa nu = 1/Pr as printed. */
#define LBM_PR_SHIFTED 0
#define LBM_PR_LITERAL 1

/* population storage: every precision holds (g_i - w_i)/w_i and (h_i - w_i N_f/2)/w_i,
 * the deviations from the rest state rho = T = 1, u = 0 scaled by the weight.  FP32, FP16
 * and BF16 storage compute in FP32 (FP16 / BF16 round to nearest even when stored).
 * LBM_FP64 stores and computes in FP64 (D2Q37 and D3Q103, two-pass kernel only, twice the
 * bytes of FP32): for steady states that must match an FP64 reference more closely than
 * the FP32 iteration allows, whose fixed points wander by a few 1e-6 of u with the path
 * taken to them.  No paper counterpart: the paper states no precision. */
#define LBM_FP32 0
#define LBM_FP16 1
#define LBM_BF16 2
#define LBM_FP64 3

/* y boundaries */
#define LBM_PERIODIC 0
#define LBM_WALLS 1 /* hybrid kinetic (KBC) + non-equilibrium extrapolation walls (Sec. VI A) */
/* x boundaries (bc_x): periodic, or open ends (Sec. VI B, the shock tube) read as zero
 * gradient: a population that would stream in from beyond x = 0 or x = nx - 1 is the
 * boundary cell's own of that velocity */
#define LBM_OPEN 2

/* stream-collide kernel variants (lbm_set_kernel / lbm_autotune) */
#define LBM_KERNEL_AUTO 0    /* the library's default for the configuration: PAIRED
                                where admissible, TWOPASS on D3Q103, D2Q77 and with
                                FP64 storage, else DIRECT                              */
#define LBM_KERNEL_DIRECT 1  /* one cell per thread, populations gathered from HBM     */
#define LBM_KERNEL_STAGED 2  /* persistent tiles staged in shared memory by bulk
                                asynchronous copies (D2Q37, periodic x, nx a multiple
                                of the tile width: 128 cells)                          */
#define LBM_KERNEL_PAIRED 3  /* two neighbouring cells per thread in packed FP32 pairs
                                (D2Q37, FP16 or BF16 storage, periodic x, nx even)     */
#define LBM_KERNEL_TWOPASS 4 /* one cell per thread, populations read twice (moments,
                                then relaxation) instead of held in registers (16-bit
                                storage on D3Q103: kept packed between the passes);
                                every lattice, the only form for FP64 storage          */

/* memory space of field pointers */
#define LBM_MEM_DEVICE 0
#define LBM_MEM_HOST 1

typedef struct lbm_params {
    int lattice;          /* LBM_D2Q37, LBM_D2Q33, LBM_D2Q77 (D = 2) or LBM_D3Q103 (D = 3)   */
    double Pr;            /* target Prandtl number, > 0 (Eq. Pr)                          */
    double gamma;         /* if > 0: N_f = 2/(gamma - 1) - D (Eq. Gamma); else N_f is used */
    double N_f;           /* additional degrees of freedom, >= 0, real                     */
    double kappa;         /* ES-BGK kappa in (0, 1]; kappa = 1 forces Pr = 1               */
    double tau;           /* tau_f = tau / dt in lattice steps, > 1/2                      */
    int pr_mode;          /* LBM_PR_SHIFTED or LBM_PR_LITERAL                              */
    int storage;          /* LBM_FP32, LBM_FP16, LBM_BF16 or LBM_FP64                      */
    int nx, ny, nz;       /* grid; nz = 1 for D = 2; nx, ny >= 1 (walls: ny >= 5);
                             ny (+ 4 with walls) and nz at most 65535                        */
    int bc_y;             /* LBM_PERIODIC or LBM_WALLS (D2Q37, D3Q103; walls are the planes
                             y = 0 and y = ny - 1, z periodic)                            */
    double wall_u[2][3];  /* bottom (y = 0) / top (y = ny-1) wall velocity (tangential x)   */
    double wall_T[2];     /* bottom / top wall temperature, > 0                            */
    int bc_x;             /* LBM_PERIODIC (default, 0) or LBM_OPEN (D = 2)                 */
    double rho0, T0;      /* reference state of the stored populations, > 0 (0 reads as 1):
                             the library stores each population less the rest equilibrium
                             at (rho0, u = 0, T0), scaled by its weight.  Only the rounding
                             of the stored values depends on it (16-bit storage keeps its
                             relative precision on flows whose mean state is far from
                             rho = T = 1); the scheme, its lattice (Gauss-Hermite at unit
                             temperature, Sec. III) and every input and output are the same */
} lbm_params;

typedef struct lbm_handle lbm_handle;

/* Validates *p, maps the parameters, derives the lattice in FP64, allocates the two
 * population buffers on the current device and binds `stream` (a cudaStream_t, may be
 * NULL for the legacy default stream).  On success *out receives the handle and the
 * populations are those of rho = 1, u = 0, T = 1.  Returns LBM_OK, LBM_WARN_PR_RANGE
 * (handle valid), LBM_ERR_ARG, LBM_ERR_NOMEM or LBM_ERR_CUDA (no handle). */
int lbm_create(const lbm_params *p, void *stream, lbm_handle **out);

/* Frees the handle and its device buffers (synchronises its stream first). */
int lbm_destroy(lbm_handle *h);

/* Text of the last error on this handle ("" if none); a static string for h == NULL
 * describing the last lbm_create failure. */
const char *lbm_last_error(const lbm_handle *h);

/* Lattice of a handle: D, Q, scale r, integer velocities c[Q][3] and weights w[Q]
 * (host arrays of at least Q entries, each may be NULL), in the library's own order. */
int lbm_lattice_info(const lbm_handle *h, int *D, int *Q, double *r, int *c, double *w);

/* Mapped coefficients: out[0..5] = N_f, omega, nu (Gaussian), tau_s, tau_q, kappa. */
int lbm_coefficients(const lbm_handle *h, double *out);

/* Handle-free host helpers (no device work): the lattice as lbm_create derives it
 * (weights re-solved in FP64 from the degree-9 moment conditions, Sec. VI A), and the
 * mapping of a parameter set to out[0..5] as in lbm_coefficients.  lbm_map_params
 * returns LBM_ERR_ARG for an inadmissible set and LBM_WARN_PR_RANGE as lbm_create does. */
int lbm_lattice_table(int lattice, int *D, int *Q, double *r, int *c, double *w);

/* The lattice's scale r (xi_i = r c_i; one lattice spacing per time step is r in the
 * paper's units, Sec. V "dimensionless variables": dx = r dt), as lbm_lattice_table
 * derives it.  Host only; LBM_ERR_ARG for an unknown lattice or r == NULL. */
int lbm_lattice_unit_scale(int lattice, double *r);
int lbm_map_params(const lbm_params *p, double *out);

/* Sets every domain population to the discrete equilibrium of the fields with
 * Lambda = T delta: g_i = G_i(rho, u, T delta), h_i = (N_f/2) T G_i.  rho[n], u[D][n],
 * T[n] with n = Nx Ny Nz.  With walls, the wall procedure then rebuilds the wall and ghost
 * rows from the first fluid rows, as after every step, so the fluid rows keep exactly
 * their initial mass from the first step on (the wall rows' reported fields are then the
 * wall procedure's, not the input's).  `mem` = LBM_MEM_DEVICE or LBM_MEM_HOST (host arrays
 * are staged through a device copy on the handle's stream).  Resets the step counter. */
int lbm_init_fields(lbm_handle *h, const double *rho, const double *u, const double *T, int mem);

/* lbm_init_fields plus a non-equilibrium part (warm start from predicted profiles;
 * no paper counterpart): Pi[D(D+1)/2][n] (rho sigma as lbm_moments reports it, may be
 * NULL) contributes its traceless part of Pi - rho T delta through the second Hermite
 * term of g (reproducing Pi; mass, momentum and energy unchanged); q[D][n] (may be NULL)
 * a heat flux, (D+2)/(D+2+N_f) of it through the third Hermite term of g and the rest
 * through the first of h. */
int lbm_init_fields_neq(lbm_handle *h, const double *rho, const double *u, const double *T, const double *Pi,
                        const double *q, int mem);

/* lbm_init_fields_neq with fields of either precision: dtype LBM_DTYPE_F64 (double
 * arrays, exactly lbm_init_fields_neq) or LBM_DTYPE_F32 (float arrays, widened to FP64
 * first: on the host for LBM_MEM_HOST, by a kernel on the handle's stream into the
 * handle's staging buffer for LBM_MEM_DEVICE).  Pi and q may be NULL (equilibrium only, as
 * lbm_init_fields).  No paper counterpart: a convenience of the interface.  LBM_ERR_ARG for
 * a null field, an unknown dtype or mem; LBM_ERR_NOMEM if the staging buffer cannot grow. */
#define LBM_DTYPE_F64 0
#define LBM_DTYPE_F32 1
int lbm_init_fields_typed(lbm_handle *h, const void *rho, const void *u, const void *T, const void *Pi,
                          const void *q, int dtype, int mem);

/* Queues nsteps fused pull-stream + collide steps (+ the wall kernel when bc_y is
 * LBM_WALLS) on the handle's stream.  nsteps >= 0. */
int lbm_step(lbm_handle *h, int nsteps);

/* Macroscopic fields of the stored (post-collision) populations, per domain cell:
 * rho[n]; u[D][n]; T[n] = T_eq; Pi[D(D+1)/2][n] = rho sigma (xx, xy, (xz), yy, (yz), (zz));
 * q[D][n] = sum_i g_i |xi_i - u|^2 (xi_i - u)/2 + h_i (xi_i - u).  Any pointer may be
 * NULL.  Synchronises the handle's stream. */
int lbm_moments(lbm_handle *h, double *rho, double *u, double *T, double *Pi, double *q, int mem);

/* FP64 global diagnostics over the domain (deterministic reduction):
 * out[0] mass sum rho; out[1..3] momentum sum rho u; out[4] total energy
 * sum rho E = sum_i (xi_i^2 g_i / 2 + h_i); out[5] residual
 * max_{X in {u_x, T}} ||X - X_prev||_2 / (m ||X||_2) against the fields of the previous
 * lbm_diagnostics call m steps earlier (0 on the first call); out[6] number of cells with
 * a non-finite value, rho <= 0 or T <= 0; out[7] steps taken since lbm_init_fields.
 * Synchronises; returns LBM_ERR_UNSTABLE when out[6] > 0. */
int lbm_diagnostics(lbm_handle *h, double *out);

/* Selects the stream-collide kernel variant; LBM_ERR_ARG if the variant does not
 * support this handle's configuration.  No paper counterpart: an implementation choice. */
int lbm_set_kernel(lbm_handle *h, int variant);

/* Times every admissible variant over `steps` steps (after 2 warm-up steps) on the
 * handle's stream, selects the fastest and writes it to *chosen (may be NULL).  Resets
 * the populations to the rest state (call before lbm_init_fields) and the step counter. */
int lbm_autotune(lbm_handle *h, int steps, int *chosen);

/* Fault injection for failure-detection tests (no paper counterpart).  on != 0: the
 * staged kernel (LBM_KERNEL_STAGED) announces each tile's bytes but issues no copy, so its
 * bounded waits run out (after ~2^22 SM cycles instead of ~2^31); the steps leave their
 * output undefined and the next synchronising call (lbm_diagnostics, lbm_moments) returns
 * LBM_ERR_TIMEOUT.  Nothing faults and the context stays usable; on = 0 restores normal
 * operation (re-initialise the fields).  Other kernels ignore it.  Synchronises. */
int lbm_debug_inject_stall(lbm_handle *h, int on);

/* Host-side audit of the stream-collide kernels' addressing (tests only; no device work,
 * no paper counterpart).  For the configuration *p and kernel variant (LBM_KERNEL_DIRECT,
 * LBM_KERNEL_STAGED, LBM_KERNEL_PAIRED, LBM_KERNEL_TWOPASS or LBM_AUDIT_BATCH), forms
 * every element index the variant gathers from and stores to (and, with walls, those of
 * the wall kernel), for every computed cell, with the kernels' own index helpers and
 * the launch's wrap threshold, and counts the accesses outside the 2 Q planes of a
 * population buffer (and the 32-bit accesses of the paired kernel off a 4-byte boundary,
 * the staged kernel's bulk copies off a 16-byte boundary).
 * wrap_threshold > 0 replaces the launch's threshold (extents below it take the modulo
 * wrap) so a test can show that a wrong one is caught; 0 keeps the launch's.  Returns the
 * count (0: every access in bounds), or minus an LBM status for invalid parameters or a
 * variant the configuration does not admit. */
long long lbm_debug_index_audit(const lbm_params *p, int variant, int wrap_threshold);
/* The reference state's shifts as the kernels use them (tests only; no device work): for
 * the configuration *p (its rho0, T0), dg[i] and dh[i] receive the shift of velocity i's
 * stored g and h deviations (host arrays of Q doubles, the library's velocity order; the
 * rest equilibrium at (rho0, T0) over the weight, less rho = T = 1, Sec. IV), and
 * share[0..4] the reference's share of the moment sums sum_i w_i dg_i, sum_i w_i dh_i and
 * sum_i w_i dg_i c_ia^2 (a = x, y, z; each as its hi + lo pair summed).  Returns Q, or
 * minus an LBM status for invalid parameters. */
int lbm_debug_reference_state(const lbm_params *p, double *dg, double *dh, double *share);
/* variant value for lbm_debug_index_audit: the batched step's addressing for one instance
 * (D2Q37, FP32, periodic x; also checks that its 32-bit offsets do not overflow) */
#define LBM_AUDIT_BATCH 5

/* Conservation totals of caller-owned FP64 device fields, allocating nothing (the paper
 * has no counterpart: this serves callers that cannot call cudaMalloc, for instance code
 * whose device memory was all reserved up front by a host framework, or a time-critical
 * loop that must not risk the device synchronisation an allocation can bring).
 *   rho[n], u[D][n], T[n]: device arrays in the field layout above (e.g. lbm_moments
 *     output); out: device array of 6 doubles receiving sum rho, sum rho u_x, _y, _z
 *     (0 for D = 2), sum rho (u^2/2 + (D + N_f) T / 2) and the number of cells with a
 *     non-finite value, rho <= 0 or T <= 0.  N_f as lbm_coefficients reports it.
 *   Work is queued on `stream` (a cudaStream_t, NULL = legacy default stream); the call
 *   does not synchronise.  Limit: n <= 33,554,432 cells, else LBM_ERR_ARG.
 * The block partial sums live in one fixed 96 KiB __device__ array inside the library,
 * held on every GPU that loads it until the process exits.  Each call made outside a
 * stream capture looks that array's address up (cudaGetSymbolAddress) with the device
 * current; a call inside a capture reuses the address of the last call on that device,
 * so make a first call on each device before any stream capture.  Every call shares the
 * array and its last contents; each call overwrites the rows it reads, so nothing needs
 * clearing, but calls that overlap on the GPU (other streams, other threads) race on it.
 * Errors: LBM_ERR_ARG, LBM_ERR_CUDA; text in lbm_last_error(NULL). */
int lbm_field_totals_static(int D, double N_f, long long n, const double *rho, const double *u, const double *T,
                            double *out, void *stream);

/* Checkpoint / resume: copies the domain populations (not ghost rows) as FP64 absolute
 * values g[Q][n], h[Q][n] (host or device per `mem`) out of / into the handle.  The
 * reference state's shift is added / removed in FP64, so the values do not depend on it
 * beyond the rounding of the storage form. */
int lbm_get_populations(lbm_handle *h, double *g, double *hh, int mem);
int lbm_set_populations(lbm_handle *h, const double *g, const double *hh, int mem);

/* ---------------------------------------------------------------------------------
 * Batched instances (no paper counterpart: a throughput layer).  Many independent 2-D
 * D2Q37 FP32 instances (each with its own grid, boundaries, Pr, gamma, kappa, tau and
 * walls) advance together: every time step is one persistent launch walking a device
 * work list of 128-cell chunks over all active instances, followed by the wall, flip,
 * residual and work-list kernels, all replayed from a CUDA graph.  An instance stops
 * when its residual (as in lbm_diagnostics out[5]) falls below the tolerance at a
 * check; the work list then drops it.  The batch owns its device memory and a stream.
 * --------------------------------------------------------------------------------- */
typedef struct lbm_batch lbm_batch;

/* n >= 1 parameter sets (lattice LBM_D2Q37, storage LBM_FP32, periodic x for every one;
 * each instance's 2 Q population planes below 2^31 values, i.e. at most 29,020,049 cells
 * per plane, nx (ny + 4) with walls and nx ny without: LBM_ERR_ARG otherwise, checked
 * before any device work); every instance starts at the rest state.  Returns LBM_OK or an
 * error (text in lbm_last_error(NULL)). */
int lbm_batch_create(int n, const lbm_params *params, lbm_batch **out);
int lbm_batch_destroy(lbm_batch *b);

/* Equilibrium initial state of instance i from its fields (layout and `mem` as in
 * lbm_init_fields); marks it active and resets its step count and residual. */
int lbm_batch_init_fields(lbm_batch *b, int i, const double *rho, const double *u, const double *T, int mem);
/* ... with the non-equilibrium part of lbm_init_fields_neq. */
int lbm_batch_init_fields_neq(lbm_batch *b, int i, const double *rho, const double *u, const double *T,
                              const double *Pi, const double *q, int mem);

/* Advances every active instance until all have converged (residual < tol at a check,
 * checks every `check_every` steps, 1 <= check_every <= 100000: one window is captured as
 * a CUDA graph) or `max_steps` steps have been taken by the batch, in whole windows (the
 * last may run past max_steps by up to check_every - 1 steps).  An instance whose fields
 * turn non-finite stops at its next check with residual NaN (lbm_batch_status); the
 * others carry on.  Synchronises.  *steps_taken (may be NULL) receives the number of
 * batch steps run. */
int lbm_batch_run(lbm_batch *b, int max_steps, double tol, int check_every, int *steps_taken);

/* Per-instance status (host arrays of n entries, any may be NULL): steps taken, last
 * residual (infinity before the second check), active flag (0 once converged). */
int lbm_batch_status(lbm_batch *b, int *steps, double *residual, int *active);

/* Re-activates instance i (every instance when i < 0) without touching its populations
 * or step count, so a finished batch can continue to a tighter tolerance; its next
 * residual check takes a fresh snapshot.  An instance whose residual is NaN (a diverged
 * run, deactivated at its check) stays inactive.  Synchronises the batch's stream. */
int lbm_batch_activate(lbm_batch *b, int i);

/* Fields of instance i (as lbm_moments). */
int lbm_batch_moments(lbm_batch *b, int i, double *rho, double *u, double *T, double *Pi, double *q, int mem);

/* Times the step kernel's tile sizes (128, 256 or 512 cells per work item) over
 * `steps` steps (1 <= steps <= 100000, one captured window) on the current state and
 * keeps the fastest; *chosen receives the tile.  Resets every instance to the rest state
 * (call before lbm_batch_init_fields). */
int lbm_batch_autotune(lbm_batch *b, int steps, int *chosen);

/* ---------------------------------------------------------------------------------
 * Surrogate network (no paper counterpart: the learned warm start).  A multilayer
 * perceptron sizes[0] -> sizes[1] -> ... -> sizes[nlayers] with GELU on every hidden
 * layer and a linear output, trained on the mean squared error with Adam.  Products run
 * on the tensor cores in bfloat16 with FP32 accumulation (lbm_mlp_set_gemm); weights are
 * kept in FP32.
 * Parameters are packed per layer as W (sizes[l] x sizes[l+1], row-major) then b.
 * All device work is queued on `stream`; calls that return host data synchronise.
 * --------------------------------------------------------------------------------- */
typedef struct lbm_mlp lbm_mlp;

int lbm_mlp_create(int nlayers, const int *sizes, int max_batch, void *stream, lbm_mlp **out);
int lbm_mlp_destroy(lbm_mlp *h);
long long lbm_mlp_num_params(const lbm_mlp *h);
/* Host FP32 parameters in (resets the Adam state) / out; grads (may be NULL) receives the
 * gradients of the last lbm_mlp_backward in the same packing. */
int lbm_mlp_set_params(lbm_mlp *h, const float *params);
int lbm_mlp_get_params(lbm_mlp *h, float *params, float *grads);
/* x: device [batch][sizes[0]] FP32; y (device, may be NULL): [batch][sizes[nlayers]]. */
int lbm_mlp_forward(lbm_mlp *h, int batch, const float *x, float *y);
/* Gradients of mean((y - target)^2) for the last forward; target: device FP32 like y;
 * *loss (may be NULL, synchronises) receives the loss. */
int lbm_mlp_backward(lbm_mlp *h, const float *target, double *loss);
/* One Adam step (Kingma & Ba, bias-corrected) with the last gradients. */
int lbm_mlp_adam(lbm_mlp *h, float lr, float b1, float b2, float eps);

/* Matrix-product form of the handle's products.  LBM_MLP_GEMM_TCGEN05 (the default):
 * 128 x 64 output tiles as tcgen05 MMAs with operands staged in shared memory and the
 * accumulator in tensor memory; LBM_MLP_GEMM_MMA_SYNC: warp-level mma.sync m16n8k16.
 * Both take BF16 operands and accumulate in FP32.  A tcgen05 product whose completion
 * wait times out (about a second) leaves its output unwritten and makes the next
 * synchronising call (lbm_mlp_backward with a loss, lbm_mlp_get_params) return
 * LBM_ERR_TIMEOUT. */
#define LBM_MLP_GEMM_TCGEN05 0
#define LBM_MLP_GEMM_MMA_SYNC 1
int lbm_mlp_set_gemm(lbm_mlp *h, int kind);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
