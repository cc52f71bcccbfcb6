// Shared-memory-staged fused stream + collide (Sec. V, Eqs. DiscreteReductionG / H).
//
// A block owns TW consecutive cells of one row (a tile) and runs persistently over tiles.
// For the next tile, one warp issues bulk asynchronous copies (the TMA engine,
// cp.async.bulk) of every population plane's source row segment [x0 - H, x0 + TW + H)
// into a shared-memory stage, while the block computes the current tile from the other
// stage; an mbarrier with a transaction count signals arrival.  The pull-stream is then
// a shared-memory read at a compile-time offset: population i of cell x0 + tx is
// stage[plane i][H + tx - c_ix], and the source row y - c_iy (wrapped, or a wall ghost
// row) was chosen by the producer.  Population values are read from shared memory
// twice (moments, then relaxation), so they never occupy registers across the cell.
//
// Constraints of this path (the host falls back to the register kernel otherwise):
// nx a multiple of TW, row starts 16-byte aligned, D = 2.  H = 16 bytes of halo (4 FP32
// or 8 FP16/BF16 values) covers |c_x| <= 3 and keeps every copy 16-byte aligned.
#pragma once
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace lbm {

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(smem_u32(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}

// global -> shared bulk copy completing on `bar` (16-byte aligned, size a multiple of 16)
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// Bounded wait on an mbarrier phase: gives up after `limit` SM cycles (2^31, about a
// second, unless a test asks for less).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, long long limit = 1LL << 31)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}

template <int ST> struct TileGeom {
    using T = typename Storage<ST>::T;
    static constexpr int TW = 128;                    // cells per tile = threads per block
    static constexpr int H = 16 / (int)sizeof(T);     // halo values per side
    static constexpr int L = TW + 2 * H;              // staged values per plane row
};

template <int LAT, int ST> struct SmemPop {
    using G = TileGeom<ST>;
    using S = Storage<ST>;
    using V = float;
    static constexpr int Q = Lattice<LAT>::Q;
    const typename S::T *base; // stage + H + tx
    __device__ __forceinline__ void refresh() {}
    template <int P> __device__ __forceinline__ void prefetch() const {}
    template <int I> __device__ __forceinline__ float sv() const
    {
        constexpr int off = I * G::L - cv<LAT, I, 0>();
        return S::cvt(*reinterpret_cast<const typename S::Raw *>(base + off));
    }
    template <int I> __device__ __forceinline__ float tv() const
    {
        constexpr int off = (Q + I) * G::L - cv<LAT, I, 0>();
        return S::cvt(*reinterpret_cast<const typename S::Raw *>(base + off));
    }
};

// Shared-memory bytes of the kernel: two stages plus the two mbarriers.
template <int LAT, int ST> constexpr size_t tma_smem_bytes()
{
    using G = TileGeom<ST>;
    return 128 + 2 * (size_t)(2 * Lattice<LAT>::Q) * G::L * sizeof(typename G::T);
}

// Blocks per SM the kernel is compiled for: shared memory allows 2 stages of FP32 tiles
// for two blocks, of 16-bit tiles for four (registers then cap at 128 per thread).
template <int ST> constexpr int tma_min_blocks() { return ST == ST_FP32 ? 2 : 4; }

template <int LAT, int ST, bool WALLS>
__global__ void __launch_bounds__(128, tma_min_blocks<ST>()) k_stream_collide_tma(const typename Storage<ST>::T *__restrict__ src,
                                                              typename Storage<ST>::T *__restrict__ dst,
                                                              const KParams<LAT> kp, int ntiles, int *err)
{
    using G = TileGeom<ST>;
    using T = typename G::T;
    constexpr int Q = Lattice<LAT>::Q;
    constexpr int NP = 2 * Q;
    constexpr uint32_t STAGE_ELEMS = NP * G::L;
    constexpr uint32_t STAGE_BYTES = STAGE_ELEMS * sizeof(T);
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw);
    T *stage0 = reinterpret_cast<T *>(smem_raw + 128);
    const int tx = threadIdx.x;
    const int lane = tx & 31, warp = tx >> 5;
    const int tpr = kp.nx / G::TW;  // tiles per row
    const bool small_y = kp.ny < 4;
    // err[1] != 0: fault injection for the tests (lbm_debug_inject_stall): the producer
    // announces a stage's bytes but issues no copy, so every wait runs out, after a short
    // limit, and the launch reports LBM_ERR_TIMEOUT through err[0]
    const bool stall = err[1] != 0;
    const long long limit = stall ? (1LL << 22) : (1LL << 31);

    if (tx == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();

    // producer: warp 0 stages tile t into stage st
    auto produce = [&](int t, int st) {
        const int x0 = (t % tpr) * G::TW;
        const int rz = t / tpr;
        const int y = kp.y0 + rz % kp.ny_comp;
        const int z = rz / kp.ny_comp;
        T *sbase = stage0 + (size_t)st * STAGE_ELEMS;
        if (lane == 0) mbar_expect_tx(&bar[st], STAGE_BYTES);
        __syncwarp();
        if (stall) return;
        const bool interior = x0 >= G::H && x0 + G::TW + G::H <= kp.nx;
        for (int p = lane; p < NP; p += 32) {
            const int i = p < Q ? p : p - Q;
            const int cy = kp.cvel[i][1];
            int ys;
            if constexpr (WALLS) {
                ys = y - cy + kp.gh;
            } else {
                ys = y - cy;
                if (small_y) ys = ((ys % kp.ny) + kp.ny) % kp.ny;
                else ys += ys < 0 ? kp.ny : (ys >= kp.ny ? -kp.ny : 0);
            }
            const T *row = src + (long long)p * kp.plane + ((long long)z * kp.nys + ys) * kp.nx;
            T *srow = sbase + p * G::L;
            if (interior) {
                bulk_g2s(srow, row + (x0 - G::H), G::L * sizeof(T), &bar[st]);
            } else {
                const int xl = x0 == 0 ? kp.nx - G::H : x0 - G::H;
                const int xr = x0 + G::TW == kp.nx ? 0 : x0 + G::TW;
                bulk_g2s(srow, row + xl, G::H * sizeof(T), &bar[st]);
                bulk_g2s(srow + G::H, row + x0, G::TW * sizeof(T), &bar[st]);
                bulk_g2s(srow + G::H + G::TW, row + xr, G::H * sizeof(T), &bar[st]);
            }
        }
    };

    if (warp == 0 && (int)blockIdx.x < ntiles) produce(blockIdx.x, 0);
    int k = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++k) {
        const int st = k & 1;
        const int tn = t + gridDim.x;
        if (warp == 0 && tn < ntiles) {
            fence_proxy_async();
            produce(tn, st ^ 1);
        }
        const bool ok = mbar_wait_bounded(&bar[st], (k >> 1) & 1, limit);
        if (!__syncthreads_and(ok)) {
            // record the failure, let the copies this block issued land (bounded), leave
            if (tx == 0) {
                atomicExch(err, 1);
                if (tn < ntiles) mbar_wait_bounded(&bar[st ^ 1], ((k + 1) >> 1) & 1, limit);
                mbar_wait_bounded(&bar[st], (k >> 1) & 1, limit);
            }
            __syncthreads();
            return;
        }
        const int x0 = (t % tpr) * G::TW;
        const int rz = t / tpr;
        const int y = kp.y0 + rz % kp.ny_comp;
        const int z = rz / kp.ny_comp;
        const SmemPop<LAT, ST> pop{stage0 + (size_t)st * STAGE_ELEMS + G::H + tx};
        const long long o = cell_index<LAT>(kp, x0 + tx, y + kp.gh, z);
        collide_store<LAT, ST>(kp, pop, dst, o);
        __syncthreads();
    }
}

} // namespace lbm
