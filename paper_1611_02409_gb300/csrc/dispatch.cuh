// Host-side launch wrappers of the kernels for one lattice (included by one .cu per
// lattice, which instantiates them and exports an Ops table to the C-ABI layer).
#pragma once
#include <algorithm>
#include <cmath>

#include "tma_kernel.cuh"
#include "ops.h"

namespace lbm {

// The reference state's per-shell shifts and their share of the raw moments (KParams::ref_*).
// phi, the rest equilibrium at temperature T0 relative to the weight, is the truncated
// Hermite series of a Maxwellian at rest (Sec. IV) summed in closed form: with u = 0 and
// Lambda = T0 delta only the isotropic terms of even order 2n remain, and
// a^(2n).H^(2n)(xi)/(2n)! = (1 - T0)^n L_n^(D/2-1)(xi^2/2) (generalised Laguerre
// polynomials), so phi = sum_{n <= N/2} (1 - T0)^n L_n^(D/2-1)(r^2 |c|^2 / 2).
template <int LAT, class S> void set_reference(const Ctx &c, KParams<LAT, S> &kp)
{
    constexpr int D = Lattice<LAT>::D, Q = Lattice<LAT>::Q, NSH = Lattice<LAT>::NSHELL;
    const double alpha = 0.5 * D - 1.0;
    for (int i = 0; i < Q; ++i) {
        const int sh = Lattice<LAT>::T.shell[i];
        const int *cv = Lattice<LAT>::T.c[i];
        const double x = 0.5 * c.r * c.r * (cv[0] * cv[0] + cv[1] * cv[1] + cv[2] * cv[2]);
        double Lm = 0.0, L = 1.0, phi = 1.0, pw = 1.0;   // L_{n-1}, L_n, partial sum, (1 - T0)^n
        for (int nn = 1; nn <= Lattice<LAT>::ORDER / 2; ++nn) {
            const double Ln = nn == 1 ? 1.0 + alpha - x : ((2 * nn - 1 + alpha - x) * L - (nn - 1 + alpha) * Lm) / nn;
            Lm = L;
            L = Ln;
            pw *= 1.0 - c.T0;
            phi += pw * L;
        }
        kp.ref_g[sh] = (S)(c.rho0 * phi - 1.0);
        kp.ref_h[sh] = (S)(0.5 * c.Nf * (c.rho0 * c.T0 * phi - 1.0));
    }
    for (int sh = 0; sh < NSH; ++sh) {
        kp.ref_wg[sh] = (S)((double)kp.omega * (double)kp.ref_g[sh]);
        kp.ref_wh[sh] = (S)((double)kp.omega * (double)kp.ref_h[sh]);
    }
    double tot[5] = {0, 0, 0, 0, 0};
    for (int i = 0; i < Q; ++i) {
        const int sh = Lattice<LAT>::T.shell[i];
        const double dg = (double)kp.ref_g[sh], dh = (double)kp.ref_h[sh];
        tot[0] += c.w[i] * dg;
        tot[1] += c.w[i] * dh;
        for (int a = 0; a < D; ++a) tot[2 + a] += c.w[i] * dg * Lattice<LAT>::T.c[i][a] * Lattice<LAT>::T.c[i][a];
    }
    for (int k = 0; k < 5; ++k) {
        kp.ref_hi[k] = (S)tot[k];
        kp.ref_lo[k] = (S)(tot[k] - (double)kp.ref_hi[k]);
    }
}

template <int LAT, class S = float> KParams<LAT, S> make_kparams(const Ctx &c)
{
    KParams<LAT, S> kp;
    kp.nx = c.nx;
    kp.ny = c.ny;
    kp.nz = c.nz;
    kp.nys = c.nys;
    kp.gh = c.gh;
    kp.y0 = c.walls ? 1 : 0;
    kp.open_x = c.open_x;
    kp.ny_comp = c.walls ? c.ny - 2 : c.ny;
    kp.plane = c.plane;
    kp.omega = (S)c.omega;
    kp.kappa = (S)c.kappa;
    kp.a_tr = (S)c.a_tr;
    kp.a_sig = (S)c.a_sig;
    kp.Nf = (S)c.Nf;
    kp.halfNf = (S)(0.5 * c.Nf);
    kp.r = (S)c.r;
    kp.r_d = c.r;
    const double R2 = c.r * c.r;
    kp.R2_hi = (S)R2;
    kp.R2_lo = (S)(R2 - (double)kp.R2_hi);
    for (int i = 0; i < KParams<LAT, S>::Q; ++i) {
        kp.w[i] = (S)c.w[i];
        const int sh = Lattice<LAT>::T.shell[i];
        kp.wsh_hi[sh] = (S)c.w[i];
        kp.wsh_lo[sh] = (S)(c.w[i] - (double)kp.wsh_hi[sh]);
        for (int d = 0; d < 3; ++d) kp.cvel[i][d] = (signed char)Lattice<LAT>::T.c[i][d];
    }
    set_reference<LAT, S>(c, kp);
    kp.r_lo = (S)(c.r - (double)kp.r);
    for (int K = 0; K < Monos<Lattice<LAT>::D>::K; ++K) {
        const int m = Monos<Lattice<LAT>::D>::M.deg[K];
        double f = 1.0;
        for (int d = 0; d < Lattice<LAT>::D; ++d)
            for (int k = 2; k <= Monos<Lattice<LAT>::D>::M.e[K][d]; ++k) f *= k;
        const double C = std::pow(c.r, m) / f;
        kp.cm_hi[K] = (S)C;
        kp.cm_lo[K] = (S)(C - (double)kp.cm_hi[K]);
    }
    const long long elem = storage_bytes(c.storage);
    for (int p = 0; p < 2 * KParams<LAT, S>::Q; ++p) {
        const int i = p % KParams<LAT, S>::Q;
        const long long cx = Lattice<LAT>::T.c[i][0], cy = Lattice<LAT>::T.c[i][1], cz = Lattice<LAT>::T.c[i][2];
        kp.soff[p] = (long long)p * c.plane * elem;
        kp.goff[p] = ((long long)p * c.plane - cz * (long long)c.nys * c.nx - cy * c.nx - cx) * elem;
    }
    return kp;
}

// A reference state other than rho = T = 1: the step kernels with its shifts.
inline bool has_reference(const Ctx &c) { return c.rho0 != 1.0 || c.T0 != 1.0; }

template <int LAT, int ST> struct Launch {
    using T = typename Storage<ST>::T;
    using R = typename Storage<ST>::R;
    static constexpr int kTx = 128;
    static KParamsOf<LAT, ST> kparams(const Ctx &c) { return make_kparams<LAT, R>(c); }

    static dim3 rows_grid(const Ctx &c, int rows, int tx) { return dim3((c.nx + tx - 1) / tx, rows, c.nz); }

    static void init(const Ctx &c, void *dst, const double *rho, const double *u, const double *T_, cudaStream_t st)
    {
        k_init<LAT, ST><<<rows_grid(c, c.nys, 64), 64, 0, st>>>((T *)dst, kparams(c), rho, u, T_, nullptr, nullptr);
    }
    static void init_neq(const Ctx &c, void *dst, const double *rho, const double *u, const double *T_,
                         const double *Pi, const double *q, cudaStream_t st)
    {
        k_init<LAT, ST><<<rows_grid(c, c.nys, 64), 64, 0, st>>>((T *)dst, kparams(c), rho, u, T_, Pi, q);
    }
    // shared-memory-staged path: 2-D, nx a multiple of the tile width
    static bool staged_ok(const Ctx &c)
    {
        return LAT == LAT_D2Q37 && ST != ST_FP64 && !c.open_x && c.nx % TileGeom<ST>::TW == 0 && c.d_err != nullptr;
    }
    static bool tma_ok(const Ctx &c) { return c.kernel == 2 && staged_ok(c); }
    // two cells per thread: 2-D, 16-bit storage, even rows
    static bool paired_ok(const Ctx &c)
    {
        return LAT == LAT_D2Q37 && !c.open_x && (ST == ST_FP16 || ST == ST_BF16) && c.nx % 2 == 0;
    }
    template <bool W> static void step_tma(const Ctx &c, const KParams<LAT> &kp, const void *src, void *dst,
                                           cudaStream_t st)
    {
        constexpr size_t smem = tma_smem_bytes<LAT, ST>();
        static int blocks_per_sm = -1;
        if (blocks_per_sm < 0) {
            cudaFuncSetAttribute(k_stream_collide_tma<LAT, ST, W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
            int nb = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_stream_collide_tma<LAT, ST, W>, 128, smem);
            blocks_per_sm = nb > 0 ? nb : 1;
        }
        const int ntiles = (c.nx / TileGeom<ST>::TW) * kp.ny_comp * c.nz;
        const int grid = std::min(ntiles, blocks_per_sm * c.num_sms);
        k_stream_collide_tma<LAT, ST, W><<<grid, 128, smem, st>>>((const T *)src, (T *)dst, kp, ntiles, c.d_err);
    }
    static void step(const Ctx &c, const void *src, void *dst, cudaStream_t st)
    {
        const KParamsOf<LAT, ST> kp = kparams(c);
        if constexpr (LAT == LAT_D2Q37 && ST != ST_FP64) {
            if (tma_ok(c)) {
                if (c.walls) step_tma<true>(c, kp, src, dst, st);
                else step_tma<false>(c, kp, src, dst, st);
                return;
            }
        }
        if constexpr (LAT == LAT_D2Q37 && (ST == ST_FP16 || ST == ST_BF16)) {
            if (c.kernel == 3 && paired_ok(c)) {
                const dim3 grid((c.nx / 2 + kTx - 1) / kTx, kp.ny_comp, 1);
                const int sy = c.ny < 4;
                // the reference state's shifts only where the handle has one
                const bool ref = has_reference(c);
                auto *k = c.walls ? (ref ? k_stream_collide_pair_ref<LAT, ST, true> : k_stream_collide_pair<LAT, ST, true>)
                                  : (ref ? k_stream_collide_pair_ref<LAT, ST, false> : k_stream_collide_pair<LAT, ST, false>);
                k<<<grid, kTx, 0, st>>>((const T *)src, (T *)dst, kp, sy);
                return;
            }
        }
        const dim3 grid = rows_grid(c, kp.ny_comp, kTx);
        constexpr int kWrap = wrap_threshold<LAT>();
        const int sx = c.nx < kWrap, sy = c.ny < kWrap, sz = c.nz < kWrap;
        // walls on D2Q37 and D3Q103 (reach 3); the create call rejects them for D2Q33 and D2Q77
        constexpr bool W2 = LAT == LAT_D2Q37 || LAT == LAT_D3Q103;
        // D3Q103 with packed 16-bit storage takes the reference form even at rho0 = T0 = 1
        // (zero shifts, the same results): it compiles to 40 B of spills against 196 B and
        // runs 10 % faster at 256^3
        const bool ref = has_reference(c) || twopass_pack<LAT, ST>();
        // FP64 storage: two-pass only (148 / 412 doubles per cell do not fit the registers)
        if (c.kernel == 4 || ST == ST_FP64) {
            auto *k = W2 && c.walls ? (ref ? k_stream_collide_2p<LAT, ST, W2, true> : k_stream_collide_2p<LAT, ST, W2, false>)
                                    : (ref ? k_stream_collide_2p<LAT, ST, false, true> : k_stream_collide_2p<LAT, ST, false, false>);
            k<<<grid, kTx, 0, st>>>((const T *)src, (T *)dst, kp, sx, sy, sz);
            return;
        }
        if constexpr (ST != ST_FP64) {
            auto *k = W2 && c.walls ? (ref ? k_stream_collide<LAT, ST, W2, true> : k_stream_collide<LAT, ST, W2, false>)
                                    : (ref ? k_stream_collide<LAT, ST, false, true> : k_stream_collide<LAT, ST, false, false>);
            k<<<grid, kTx, 0, st>>>((const T *)src, (T *)dst, kp, sx, sy, sz);
        }
    }
    static void walls(const Ctx &c, void *buf, cudaStream_t st)
    {
        if constexpr (LAT == LAT_D2Q37 || LAT == LAT_D3Q103) {
            WallParamsT<R> wp;
            for (int b = 0; b < 2; ++b) {
                for (int d = 0; d < 3; ++d) wp.vw[b][d] = (R)(c.wall_u[b][d] / c.r);
                wp.thw[b] = (R)(c.wall_T[b] - 1.0);
            }
            k_walls<LAT, ST><<<dim3((c.nx + 63) / 64, 2, c.nz), 64, 0, st>>>((T *)buf, kparams(c), wp);
        }
    }
    static void moments(const Ctx &c, const void *buf, double *rho, double *u, double *T_, double *Pi, double *q,
                        cudaStream_t st)
    {
        k_moments<LAT, ST><<<rows_grid(c, c.ny, 64), 64, 0, st>>>((const T *)buf, kparams(c), rho, u, T_, Pi, q);
    }
    static void diag(const Ctx &c, const void *buf, void *snap, int have_snap, double *partials, int nblk,
                     cudaStream_t st)
    {
        k_diag<LAT, ST><<<nblk, kDiagThreads, 0, st>>>((const T *)buf, kparams(c), (R *)snap, have_snap, partials);
    }
    static void get_pops(const Ctx &c, const void *buf, double *g, double *h, cudaStream_t st)
    {
        k_get_pops<LAT, ST><<<rows_grid(c, c.ny, 64), 64, 0, st>>>((const T *)buf, kparams(c), g, h);
    }
    static void set_pops(const Ctx &c, void *buf, const double *g, const double *h, cudaStream_t st)
    {
        k_set_pops<LAT, ST><<<rows_grid(c, c.ny, 64), 64, 0, st>>>((T *)buf, kparams(c), g, h);
    }
};

template <int LAT, int ST> Ops make_ops_st()
{
    Ops o;
    o.init = &Launch<LAT, ST>::init;
    o.init_neq = &Launch<LAT, ST>::init_neq;
    o.step = &Launch<LAT, ST>::step;
    o.walls = &Launch<LAT, ST>::walls;
    o.moments = &Launch<LAT, ST>::moments;
    o.diag = &Launch<LAT, ST>::diag;
    o.get_pops = &Launch<LAT, ST>::get_pops;
    o.set_pops = &Launch<LAT, ST>::set_pops;
    o.staged_ok = &Launch<LAT, ST>::staged_ok;
    o.paired_ok = &Launch<LAT, ST>::paired_ok;
    return o;
}


} // namespace lbm
