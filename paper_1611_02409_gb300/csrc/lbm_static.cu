// Conservation totals of caller-owned macroscopic fields, computed without allocating.
//
// Some callers cannot call cudaMalloc at the point where they need these totals: code
// running in a region whose device memory was reserved up front by a host framework
// (further allocations fail), or a time-critical loop that must not risk the implicit
// device synchronisation an allocation can cause.  Creating a handle allocates, so this
// entry point takes plain device arrays and reduces them with a block-partial scratch
// that lives in a file-scope __device__ array of fixed size: every GPU that loads the
// library holds it (2048 x 6 doubles, 96 KiB) until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/lbm.h"
#include "ops.h"

namespace {

constexpr int kBlocks = 2048;   // rows of the scratch: one per block
constexpr int kChunk = 16384;   // cells a block reduces
constexpr int kThreads = 256;
constexpr int kNV = 6;          // mass, momentum x y z, energy, bad cells
constexpr long long kMaxCells = (long long)kBlocks * kChunk;

static __device__ __align__(256) double g_scratch[kBlocks * kNV];

// Scratch device address per device ordinal, set on the first call on that device.
constexpr int kMaxDevices = 64;
double *g_scratch_ptr[kMaxDevices] = {};
std::mutex g_setup_mutex;

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block b reduces cells [b kChunk, min(n, (b+1) kChunk)) and writes row b of `partials`
// (every row it owns is overwritten, so nothing has to start at zero).
__global__ void __launch_bounds__(kThreads) k_field_totals(const double *__restrict__ rho,
                                                           const double *__restrict__ u,
                                                           const double *__restrict__ T, long long n, int D,
                                                           double half_dof, double *partials)
{
    double acc[kNV] = {0, 0, 0, 0, 0, 0};
    const long long c0 = (long long)blockIdx.x * kChunk;
    const long long c1 = c0 + kChunk < n ? c0 + kChunk : n;
    for (long long f = c0 + threadIdx.x; f < c1; f += kThreads) {
        const double r = rho[f], t = T[f];
        double u2 = 0.0;
        bool ok = isfinite(r) && isfinite(t) && r > 0.0 && t > 0.0;
        for (int a = 0; a < D; ++a) {
            const double ua = u[a * n + f];
            ok = ok && isfinite(ua);
            acc[1 + a] += r * ua;
            u2 += ua * ua;
        }
        acc[0] += r;
        acc[4] += r * (0.5 * u2 + half_dof * t);
        acc[5] += ok ? 0.0 : 1.0;
    }
    __shared__ double sh[kThreads / 32][kNV];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v < kNV; ++v) {
        const double x = warp_sum_d(acc[v]);
        if (lane == 0) sh[wid][v] = x;
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int v = 0; v < kNV; ++v) {
            double x = lane < kThreads / 32 ? sh[lane][v] : 0.0;
            x = warp_sum_d(x);
            if (lane == 0) partials[(long long)blockIdx.x * kNV + v] = x;
        }
    }
}

// One block sums rows [0, nblk) in a fixed order into the caller's out[0..5].
__global__ void __launch_bounds__(kThreads) k_field_totals_final(const double *__restrict__ partials, int nblk,
                                                                 double *out)
{
    double acc[kNV] = {0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblk; b += kThreads)
#pragma unroll
        for (int v = 0; v < kNV; ++v) acc[v] += partials[(long long)b * kNV + v];
    __shared__ double sh[kThreads / 32][kNV];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v < kNV; ++v) {
        const double x = warp_sum_d(acc[v]);
        if (lane == 0) sh[wid][v] = x;
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int v = 0; v < kNV; ++v) {
            double x = lane < kThreads / 32 ? sh[lane][v] : 0.0;
            x = warp_sum_d(x);
            if (lane == 0) out[v] = x;
        }
    }
}

// Device address of the scratch on the current device (host code must not pass the
// symbol itself: on the host it names a stand-in, not device memory).  The address is
// looked up again on every call made outside a stream capture, so a context that was
// torn down and recreated (cudaDeviceReset) gets the array's new address; inside a
// capture the address of the last call on this device is used.
int scratch_address(cudaStream_t st, double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return lbm::set_global_error(LBM_ERR_CUDA, "cudaGetDevice failed");
    if (dev < 0 || dev >= kMaxDevices) return lbm::set_global_error(LBM_ERR_ARG, "device ordinal out of range");
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(st, &cap);
    if (e != cudaSuccess) return lbm::set_global_error(LBM_ERR_CUDA, cudaGetErrorString(e));
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (cap == cudaStreamCaptureStatusNone) {
        double *p = nullptr;
        e = cudaGetSymbolAddress(reinterpret_cast<void **>(&p), g_scratch);
        if (e != cudaSuccess || !p)
            return lbm::set_global_error(LBM_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed");
        g_scratch_ptr[dev] = p;
    } else if (!g_scratch_ptr[dev]) {
        return lbm::set_global_error(LBM_ERR_ARG, "first call on this device made during a stream capture");
    }
    *out = g_scratch_ptr[dev];
    return LBM_OK;
}

} // namespace

extern "C" int lbm_field_totals_static(int D, double N_f, long long n, const double *rho, const double *u,
                                       const double *T, double *out, void *stream)
{
    if (D != 2 && D != 3) return lbm::set_global_error(LBM_ERR_ARG, "D must be 2 or 3");
    if (!(N_f >= 0.0) || !std::isfinite(N_f)) return lbm::set_global_error(LBM_ERR_ARG, "N_f must be >= 0");
    if (!rho || !u || !T || !out) return lbm::set_global_error(LBM_ERR_ARG, "null pointer");
    if (n < 1) return lbm::set_global_error(LBM_ERR_ARG, "n must be >= 1");
    if (n > kMaxCells)
        return lbm::set_global_error(LBM_ERR_ARG, "n exceeds the static scratch limit of 33554432 cells "
                                                  "(2048 blocks x 16384 cells)");
    cudaStream_t st = (cudaStream_t)stream;
    double *scratch = nullptr;
    int rc = scratch_address(st, &scratch);
    if (rc) return rc;
    const int nblk = (int)((n + kChunk - 1) / kChunk);
    k_field_totals<<<nblk, kThreads, 0, st>>>(rho, u, T, n, D, 0.5 * (D + N_f), scratch);
    k_field_totals_final<<<1, kThreads, 0, st>>>(scratch, nblk, out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return lbm::set_global_error(LBM_ERR_CUDA, cudaGetErrorString(e));
    return LBM_OK;
}
