// Host-side launch wrappers of the kernels for one lattice (included by one .cu per
// lattice, which instantiates them and exports an Ops table to the C-ABI layer).
#pragma once
#include <algorithm>

#include "tma_kernel.cuh"
#include "ops.h"

namespace lbm {

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
    const long long elem = storage_bytes(c.storage);
    for (int p = 0; p < 2 * KParams<LAT, S>::Q; ++p) {
        const int i = p % KParams<LAT, S>::Q;
        const long long cx = Lattice<LAT>::T.c[i][0], cy = Lattice<LAT>::T.c[i][1], cz = Lattice<LAT>::T.c[i][2];
        kp.soff[p] = (long long)p * c.plane * elem;
        kp.goff[p] = ((long long)p * c.plane - cz * (long long)c.nys * c.nx - cy * c.nx - cx) * elem;
    }
    return kp;
}

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
                if (c.walls)
                    k_stream_collide_pair<LAT, ST, true><<<grid, kTx, 0, st>>>((const T *)src, (T *)dst, kp, sy);
                else
                    k_stream_collide_pair<LAT, ST, false><<<grid, kTx, 0, st>>>((const T *)src, (T *)dst, kp, sy);
                return;
            }
        }
        const dim3 grid = rows_grid(c, kp.ny_comp, kTx);
        constexpr int kWrap = wrap_threshold<LAT>();
        const int sx = c.nx < kWrap, sy = c.ny < kWrap, sz = c.nz < kWrap;
        // walls on D2Q37 and D3Q103 (reach 3); the create call rejects them for D2Q33 and D2Q77
        constexpr bool W2 = LAT == LAT_D2Q37 || LAT == LAT_D3Q103;
        // FP64 storage: two-pass only (148 / 412 doubles per cell do not fit the registers)
        if (c.kernel == 4 || ST == ST_FP64) {
            if (W2 && c.walls)
                k_stream_collide_2p<LAT, ST, W2><<<grid, kTx, 0, st>>>((const T *)src, (T *)dst, kp, sx, sy, sz);
            else
                k_stream_collide_2p<LAT, ST, false><<<grid, kTx, 0, st>>>((const T *)src, (T *)dst, kp, sx, sy, sz);
            return;
        }
        if constexpr (ST != ST_FP64) {
            if (W2 && c.walls)
                k_stream_collide<LAT, ST, W2><<<grid, kTx, 0, st>>>((const T *)src, (T *)dst, kp, sx, sy, sz);
            else
                k_stream_collide<LAT, ST, false><<<grid, kTx, 0, st>>>((const T *)src, (T *)dst, kp, sx, sy, sz);
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
