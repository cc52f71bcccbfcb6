// Surrogate network kernels (include/lbm.h, lbm_mlp_*): a multilayer perceptron with
// GELU hidden layers and a linear output, trained with the mean squared error and Adam.
// Matrix products run on the tensor cores in bfloat16 with FP32 accumulation: by
// default as tcgen05 MMAs (operands staged in shared memory, the accumulator in tensor
// memory), or as warp-level mma.sync m16n8k16 (lbm_mlp_set_gemm); master weights, Adam
// moments, pre-activations and gradients are FP32.  The operands held in bfloat16 are: the network input, the weights, every hidden
// activation fed to the next layer, and the backward deltas fed to the two gradient
// products.  The GEMMs here are small (batch <= a few hundred, width <= 1024).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "ops.h"

namespace {

using bf16 = __nv_bfloat16;
constexpr int BM = 64, BN = 64, BK = 16;

__device__ __forceinline__ uint32_t pack_bf16(bf16 lo, bf16 hi)
{
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }

__device__ __forceinline__ float gelu_grad_f(float z)
{
    return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

// C[M x N] = op(A)[M x K] op(B)[K x N] (+ bias[N]); op(A)[m][k] = ta ? A[k lda + m] :
// A[m lda + k], op(B)[k][n] = tb ? B[n ldb + k] : B[k ldb + n].  Epilogue: Cpre (FP32,
// pre-activation) if given, C = act(...) (act 1 = GELU), and its bfloat16 copy Cbf if given.
__global__ void __launch_bounds__(128) k_gemm(int M, int N, int K, const bf16 *__restrict__ A, int lda, int ta,
                                              const bf16 *__restrict__ B, int ldb, int tb, float *C, int ldc,
                                              const float *__restrict__ bias, int act, float *Cpre, bf16 *Cbf)
{
    __shared__ bf16 As[BM][BK + 8];
    __shared__ bf16 Bs[BN][BK + 8];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int wm = w >> 1, wn = w & 1;
    const int g = lane >> 2, tq = lane & 3;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[i][j][k] = 0.f;
    const bf16 zero = __float2bfloat16(0.f);
    for (int k0 = 0; k0 < K; k0 += BK) {
        for (int e = tid; e < BM * BK; e += 128) {
            const int m = e / BK, k = e % BK, gm = m0 + m, gk = k0 + k;
            As[m][k] = (gm < M && gk < K) ? (ta ? A[(long long)gk * lda + gm] : A[(long long)gm * lda + gk]) : zero;
        }
        for (int e = tid; e < BN * BK; e += 128) {
            const int n = e / BK, k = e % BK, gn = n0 + n, gk = k0 + k;
            Bs[n][k] = (gn < N && gk < K) ? (tb ? B[(long long)gn * ldb + gk] : B[(long long)gk * ldb + gn]) : zero;
        }
        __syncthreads();
        uint32_t af[2][4], bfr[4][2];
#pragma unroll
        for (int mi = 0; mi < 2; ++mi) {
            const int r = wm * 32 + mi * 16 + g;
            af[mi][0] = pack_bf16(As[r][2 * tq], As[r][2 * tq + 1]);
            af[mi][1] = pack_bf16(As[r + 8][2 * tq], As[r + 8][2 * tq + 1]);
            af[mi][2] = pack_bf16(As[r][2 * tq + 8], As[r][2 * tq + 9]);
            af[mi][3] = pack_bf16(As[r + 8][2 * tq + 8], As[r + 8][2 * tq + 9]);
        }
#pragma unroll
        for (int ni = 0; ni < 4; ++ni) {
            const int c = wn * 32 + ni * 8 + g;
            bfr[ni][0] = pack_bf16(Bs[c][2 * tq], Bs[c][2 * tq + 1]);
            bfr[ni][1] = pack_bf16(Bs[c][2 * tq + 8], Bs[c][2 * tq + 9]);
        }
#pragma unroll
        for (int mi = 0; mi < 2; ++mi)
#pragma unroll
            for (int ni = 0; ni < 4; ++ni) {
                float *d = acc[mi][ni];
                asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                             "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                             : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                             : "r"(af[mi][0]), "r"(af[mi][1]), "r"(af[mi][2]), "r"(af[mi][3]), "r"(bfr[ni][0]),
                               "r"(bfr[ni][1]));
            }
        __syncthreads();
    }
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int r = m0 + wm * 32 + mi * 16 + g + (k >= 2 ? 8 : 0);
                const int c = n0 + wn * 32 + ni * 8 + 2 * tq + (k & 1);
                if (r < M && c < N) {
                    float v = acc[mi][ni][k] + (bias ? bias[c] : 0.f);
                    const long long o = (long long)r * ldc + c;
                    if (Cpre) Cpre[o] = v;
                    if (act == 1) v = gelu_f(v);
                    if (C) C[o] = v;
                    if (Cbf) Cbf[o] = __float2bfloat16_rn(v);
                }
            }
}

// ---- tcgen05 form -------------------------------------------------------------------
// One CTA (4 warps) computes a TM x TN tile of C (TN = 64, or 32 when 64-wide tiles would
// leave most SMs idle).  Per K step of TK, the threads stage
// op(A) (TM x TK) and op(B) (as TN rows of TK) in shared memory in the canonical
// no-swizzle K-major layout: 8-row x 16-byte core matrices, row group by row group, so
// K-adjacent core matrices are 128 bytes apart (the descriptors' leading byte offset) and
// 8-row groups TK / 8 x 128 bytes apart (the stride byte offset).  Staging moves 16-byte
// groups of eight values: eight consecutive k of one row when the operand is contiguous
// in k (one 16-byte load, one 16-byte store into its core-matrix row), eight consecutive
// rows at one k otherwise (one 16-byte load, eight 2-byte stores); groups that cross the
// matrix edge or an unaligned address are read element by element, zero outside.  Every
// thread holds its groups of the next K step in registers, loaded while the MMAs of the
// current step run.  One thread issues the TK / 16 MMAs (M = 128, N = 64, K = 16, BF16 x
// BF16 -> FP32 in tensor memory) and commits them to an mbarrier; every thread waits
// (bounded: on timeout the kernel sets *err and leaves C unwritten) before the tiles are
// restaged.  The epilogue reads each thread's row (TMEM lane) with tcgen05.ld and applies
// bias, GELU and the bfloat16 copy as k_gemm does.
constexpr int TM = 128, TK = 64;

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t core_off(int row, int k)
{
    return ((((row >> 3) * (TK / 8) + (k >> 3)) << 7) + ((row & 7) << 4) + ((k & 7) << 1));
}

// Shared-memory matrix descriptor: start, leading and stride byte offsets in 16-byte units,
// descriptor version 1, no swizzling.
__device__ __forceinline__ uint64_t mma_sdesc(uint32_t addr)
{
    constexpr uint32_t lbo = 128, sbo = (TK / 8) * 128;
    uint64_t d = (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Group g (0 <= g < ROWS TK / 8) of an operand for the K step at k0: its tile row r and
// first k (kmaj: eight consecutive k of row r; else eight consecutive rows from r at k),
// loaded from X (op(X)[r][k] = kmaj ? X[r ld + k] : X[k ld + r]; rows below rlim, k
// below klim; zero outside).
template <int ROWS> struct StageGroup {
    static __device__ __forceinline__ void place(int g, bool kmaj, int &r, int &k)
    {
        if (kmaj) {
            r = g / (TK / 8);
            k = (g % (TK / 8)) * 8;
        } else {
            k = g / (ROWS / 8);
            r = (g % (ROWS / 8)) * 8;
        }
    }
    static __device__ __forceinline__ uint4 load(const bf16 *__restrict__ X, int ld, bool kmaj, int r0, int rlim,
                                                 int k0, int klim, int g)
    {
        int r, k;
        place(g, kmaj, r, k);
        const int gr = r0 + r, gk = k0 + k;
        const bf16 *p = kmaj ? X + (long long)gr * ld + gk : X + (long long)gk * ld + gr;
        const bool full = kmaj ? (gr < rlim && gk + 8 <= klim) : (gk < klim && gr + 8 <= rlim);
        if (full && (reinterpret_cast<uintptr_t>(p) & 15) == 0) return __ldg(reinterpret_cast<const uint4 *>(p));
        uint32_t w[4];
#pragma unroll
        for (int j = 0; j < 8; j += 2) {
            unsigned short e[2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const bool in = kmaj ? (gr < rlim && gk + j + i < klim) : (gk < klim && gr + j + i < rlim);
                e[i] = in ? __bfloat16_as_ushort(p[kmaj ? j + i : (long long)(j + i)]) : (unsigned short)0;
            }
            w[j / 2] = (uint32_t)e[0] | ((uint32_t)e[1] << 16);
        }
        return make_uint4(w[0], w[1], w[2], w[3]);
    }
    static __device__ __forceinline__ void store(unsigned char *s, bool kmaj, int g, uint4 v)
    {
        int r, k;
        place(g, kmaj, r, k);
        if (kmaj) {
            *reinterpret_cast<uint4 *>(s + core_off(r, k)) = v;
        } else {
            const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int j = 0; j < 8; ++j)
                *reinterpret_cast<unsigned short *>(s + core_off(r + j, k)) =
                    (unsigned short)(j & 1 ? w[j / 2] >> 16 : w[j / 2] & 0xffffu);
        }
    }
};

__device__ __forceinline__ bool mbar_wait_limit(uint64_t *bar, uint32_t parity)
{
    const long long t0 = clock64();
    while (true) {
        uint32_t ok;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(ok)
                     : "r"(smem_addr(bar)), "r"(parity)
                     : "memory");
        if (ok) return true;
        if (clock64() - t0 > (1LL << 31)) return false;  // about a second of SM clock
    }
}

template <int TN>
__global__ void __launch_bounds__(128) k_gemm_tc(int M, int N, int K, const bf16 *__restrict__ A, int lda, int ta,
                                                 const bf16 *__restrict__ B, int ldb, int tb, float *C, int ldc,
                                                 const float *__restrict__ bias, int act, float *Cpre, bf16 *Cbf,
                                                 int *err)
{
    __shared__ __align__(1024) unsigned char sA[TM * TK * 2];
    __shared__ __align__(1024) unsigned char sB[TN * TK * 2];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tbase;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tbase)),
                     "r"(TN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tbase;
    // instruction descriptor: D FP32, A and B BF16, both K-major, N / 8, M / 16
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) |
                           ((uint32_t)(TM >> 4) << 24);
    uint32_t phase = 0;
    int ok = 1;
    // op(A) rows are m (contiguous in k unless ta); op(B) rows are n (contiguous in k if tb).
    // Group g of a thread: tid + 128 j, so consecutive threads read consecutive addresses.
    constexpr int GA = TM * TK / 8 / 128, GB = TN * TK / 8 / 128;
    const bool akm = !ta, bkm = tb != 0;
    uint4 va[GA], vb[GB];
#pragma unroll
    for (int j = 0; j < GA; ++j) va[j] = StageGroup<TM>::load(A, lda, akm, m0, M, 0, K, tid + 128 * j);
#pragma unroll
    for (int j = 0; j < GB; ++j) vb[j] = StageGroup<TN>::load(B, ldb, bkm, n0, N, 0, K, tid + 128 * j);
    for (int k0 = 0; k0 < K; k0 += TK) {
#pragma unroll
        for (int j = 0; j < GA; ++j) StageGroup<TM>::store(sA, akm, tid + 128 * j, va[j]);
#pragma unroll
        for (int j = 0; j < GB; ++j) StageGroup<TN>::store(sB, bkm, tid + 128 * j, vb[j]);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int s = 0; s < TK / 16; ++s) {
                const uint64_t da = mma_sdesc(smem_addr(sA) + s * 256), db = mma_sdesc(smem_addr(sB) + s * 256);
                const uint32_t accumulate = (k0 > 0 || s > 0) ? 1u : 0u;
                asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                             "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                             "l"(da), "l"(db), "r"(idesc), "r"(accumulate));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_addr(&bar))
                         : "memory");
        }
        // the next K step's groups load while the MMAs run
        if (k0 + TK < K) {
#pragma unroll
            for (int j = 0; j < GA; ++j) va[j] = StageGroup<TM>::load(A, lda, akm, m0, M, k0 + TK, K, tid + 128 * j);
#pragma unroll
            for (int j = 0; j < GB; ++j) vb[j] = StageGroup<TN>::load(B, ldb, bkm, n0, N, k0 + TK, K, tid + 128 * j);
        }
        const int w = mbar_wait_limit(&bar, phase) ? 1 : 0;
        phase ^= 1;
        ok = __syncthreads_and(w && ok);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (!ok) break;
    }
    if (ok) {
        const int r = m0 + warp * 32 + (tid & 31);
        for (int c = 0; c < TN; c += 8) {
            uint32_t v[8];
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                         : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                           "=r"(v[7])
                         : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int col = n0 + c + j;
                if (r < M && col < N) {
                    float x = __uint_as_float(v[j]) + (bias ? bias[col] : 0.f);
                    const long long o = (long long)r * ldc + col;
                    if (Cpre) Cpre[o] = x;
                    if (act == 1) x = gelu_f(x);
                    if (C) C[o] = x;
                    if (Cbf) Cbf[o] = __float2bfloat16_rn(x);
                }
            }
        }
    } else if (tid == 0) {
        atomicExch(err, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TN));
}

__global__ void k_f2bf(const float *__restrict__ s, bf16 *d, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        d[i] = __float2bfloat16_rn(s[i]);
}

// dz = 2 (y - t) / n, its bfloat16 copy, and per-block partial sums of (y - t)^2.
__global__ void __launch_bounds__(256) k_mse(const float *__restrict__ y, const float *__restrict__ t, float *dz,
                                             bf16 *dzb, long long n, double *partials)
{
    double acc = 0.0;
    for (long long i = blockIdx.x * 256LL + threadIdx.x; i < n; i += (long long)gridDim.x * 256) {
        const float d = y[i] - t[i];
        acc += (double)d * d;
        const float gz = 2.f * d / (float)n;
        dz[i] = gz;
        dzb[i] = __float2bfloat16_rn(gz);
    }
    __shared__ double sh[256];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = sh[0];
}

__global__ void k_sum_partials(const double *p, int n, double *out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += p[i];
        *out = s;
    }
}

// dz = da * GELU'(z) and its bfloat16 copy.
__global__ void k_gelu_bwd(const float *__restrict__ da, const float *__restrict__ z, float *dz, bf16 *dzb,
                           long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float v = da[i] * gelu_grad_f(z[i]);
        dz[i] = v;
        dzb[i] = __float2bfloat16_rn(v);
    }
}

// db[c] = sum_r dz[r][c] (fixed order per column).
__global__ void k_colsum(const float *__restrict__ dz, int rows, int cols, float *db)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    float s = 0.f;
    for (int r = 0; r < rows; ++r) s += dz[(long long)r * cols + c];
    db[c] = s;
}

__global__ void k_adam(float *w, const float *__restrict__ g, float *m, float *v, long long n, float lr, float b1,
                       float b2, float eps, float c1, float c2)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

} // namespace

struct lbm_mlp {
    int L = 0, maxb = 0;
    std::vector<int> sizes;
    std::vector<long long> woff, boff;  // offsets into the packed parameter vector
    long long nparam = 0;
    float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;  // packed FP32
    bf16 *wb = nullptr;                                            // bfloat16 weights (packed like p)
    bf16 *xb = nullptr;                                            // input [maxb][sizes[0]]
    std::vector<float *> z;                                        // pre-activations per layer
    std::vector<bf16 *> ab;                                        // hidden activations (bf16)
    float *dz = nullptr, *da = nullptr;
    bf16 *dzb = nullptr;
    double *partials = nullptr, *dloss = nullptr;
    int *err = nullptr;             // set by a tcgen05 GEMM whose MMA wait timed out
    int gemm_kind = LBM_MLP_GEMM_TCGEN05;
    int num_sms = 1;                // of the device the handle was created on
    int batch = 0;
    long long t = 0;
    cudaStream_t stream = nullptr;
};

namespace {

int mfail(const char *msg) { return lbm::set_global_error(LBM_ERR_ARG, msg); }

#define LBM_MCK(call)                                                                                          \
    do {                                                                                                       \
        cudaError_t e_ = (call);                                                                               \
        if (e_ != cudaSuccess) return lbm::set_global_error(LBM_ERR_CUDA, cudaGetErrorString(e_));             \
    } while (0)

void gemm(lbm_mlp *h, int M, int N, int K, const bf16 *A, int lda, int ta, const bf16 *B, int ldb, int tb, float *C,
          int ldc, const float *bias, int act, float *Cpre, bf16 *Cbf)
{
    if (h->gemm_kind == LBM_MLP_GEMM_TCGEN05) {
        // 64-wide tiles unless they would occupy fewer than half of the SMs
    const int tiles64 = ((N + 63) / 64) * ((M + TM - 1) / TM);
    if (tiles64 < h->num_sms / 2) {
        dim3 grid((N + 31) / 32, (M + TM - 1) / TM);
        k_gemm_tc<32><<<grid, 128, 0, h->stream>>>(M, N, K, A, lda, ta, B, ldb, tb, C, ldc, bias, act, Cpre, Cbf,
                                                  h->err);
        return;
    }
    dim3 grid((N + 63) / 64, (M + TM - 1) / TM);
        k_gemm_tc<64><<<grid, 128, 0, h->stream>>>(M, N, K, A, lda, ta, B, ldb, tb, C, ldc, bias, act, Cpre, Cbf,
                                                  h->err);
        return;
    }
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM);
    k_gemm<<<grid, 128, 0, h->stream>>>(M, N, K, A, lda, ta, B, ldb, tb, C, ldc, bias, act, Cpre, Cbf);
}

int grid1(long long n) { return (int)std::min<long long>((n + 255) / 256, 4096); }

// LBM_ERR_TIMEOUT once a tcgen05 GEMM gave up waiting for its MMAs (the word is then
// cleared); call after a synchronisation of the handle's stream.
int check_timeout(lbm_mlp *h)
{
    int e = 0;
    LBM_MCK(cudaMemcpy(&e, h->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (!e) return LBM_OK;
    LBM_MCK(cudaMemset(h->err, 0, sizeof(int)));
    return lbm::set_global_error(LBM_ERR_TIMEOUT, "tcgen05 GEMM: MMA completion wait timed out");
}

} // namespace

extern "C" {

int lbm_mlp_create(int nlayers, const int *sizes, int max_batch, void *stream, lbm_mlp **out)
{
    if (!out || !sizes || nlayers < 1 || max_batch < 1) return mfail("need nlayers >= 1, sizes, max_batch >= 1");
    for (int i = 0; i <= nlayers; ++i)
        if (sizes[i] < 1) return mfail("layer sizes must be >= 1");
    lbm_mlp *h = new lbm_mlp();
    h->L = nlayers;
    h->maxb = max_batch;
    h->sizes.assign(sizes, sizes + nlayers + 1);
    h->stream = (cudaStream_t)stream;
    {
        int dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess)
            cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (h->num_sms < 1) h->num_sms = 1;
    }
    int maxn = 0;
    for (int l = 0; l < nlayers; ++l) {
        h->woff.push_back(h->nparam);
        h->nparam += (long long)sizes[l] * sizes[l + 1];
        h->boff.push_back(h->nparam);
        h->nparam += sizes[l + 1];
        maxn = std::max(maxn, std::max(sizes[l], sizes[l + 1]));
    }
    cudaError_t e = cudaSuccess;
    auto al = [&](void **p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(p, bytes);
        if (e == cudaSuccess) e = cudaMemsetAsync(*p, 0, bytes, h->stream);
    };
    al((void **)&h->p, sizeof(float) * h->nparam);
    al((void **)&h->g, sizeof(float) * h->nparam);
    al((void **)&h->m, sizeof(float) * h->nparam);
    al((void **)&h->v, sizeof(float) * h->nparam);
    al((void **)&h->wb, sizeof(bf16) * h->nparam);
    al((void **)&h->xb, sizeof(bf16) * (size_t)max_batch * sizes[0]);
    h->z.resize(nlayers);
    h->ab.resize(nlayers);
    for (int l = 0; l < nlayers; ++l) {
        al((void **)&h->z[l], sizeof(float) * (size_t)max_batch * sizes[l + 1]);
        al((void **)&h->ab[l], sizeof(bf16) * (size_t)max_batch * sizes[l + 1]);
    }
    al((void **)&h->dz, sizeof(float) * (size_t)max_batch * maxn);
    al((void **)&h->da, sizeof(float) * (size_t)max_batch * maxn);
    al((void **)&h->dzb, sizeof(bf16) * (size_t)max_batch * maxn);
    al((void **)&h->partials, sizeof(double) * 4096);
    al((void **)&h->dloss, sizeof(double));
    al((void **)&h->err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(h->err, 0, sizeof(int));
    if (e != cudaSuccess) {
        lbm_mlp_destroy(h);
        return lbm::set_global_error(LBM_ERR_NOMEM, cudaGetErrorString(e));
    }
    *out = h;
    return LBM_OK;
}

int lbm_mlp_destroy(lbm_mlp *h)
{
    if (!h) return LBM_OK;
    cudaStreamSynchronize(h->stream);
    for (void *p : {(void *)h->p, (void *)h->g, (void *)h->m, (void *)h->v, (void *)h->wb, (void *)h->xb,
                    (void *)h->dz, (void *)h->da, (void *)h->dzb, (void *)h->partials, (void *)h->dloss,
                    (void *)h->err})
        if (p) cudaFree(p);
    for (auto *p : h->z)
        if (p) cudaFree(p);
    for (auto *p : h->ab)
        if (p) cudaFree(p);
    delete h;
    return LBM_OK;
}

long long lbm_mlp_num_params(const lbm_mlp *h) { return h ? h->nparam : -1; }

int lbm_mlp_set_params(lbm_mlp *h, const float *params)
{
    if (!h || !params) return mfail("null argument");
    LBM_MCK(cudaMemcpyAsync(h->p, params, sizeof(float) * h->nparam, cudaMemcpyHostToDevice, h->stream));
    LBM_MCK(cudaMemsetAsync(h->m, 0, sizeof(float) * h->nparam, h->stream));
    LBM_MCK(cudaMemsetAsync(h->v, 0, sizeof(float) * h->nparam, h->stream));
    k_f2bf<<<grid1(h->nparam), 256, 0, h->stream>>>(h->p, h->wb, h->nparam);
    h->t = 0;
    LBM_MCK(cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

int lbm_mlp_get_params(lbm_mlp *h, float *params, float *grads)
{
    if (!h) return mfail("null handle");
    if (params) LBM_MCK(cudaMemcpyAsync(params, h->p, sizeof(float) * h->nparam, cudaMemcpyDeviceToHost, h->stream));
    if (grads) LBM_MCK(cudaMemcpyAsync(grads, h->g, sizeof(float) * h->nparam, cudaMemcpyDeviceToHost, h->stream));
    LBM_MCK(cudaStreamSynchronize(h->stream));
    return check_timeout(h);
}

int lbm_mlp_set_gemm(lbm_mlp *h, int kind)
{
    if (!h) return mfail("null handle");
    if (kind != LBM_MLP_GEMM_TCGEN05 && kind != LBM_MLP_GEMM_MMA_SYNC) return mfail("unknown GEMM kind");
    h->gemm_kind = kind;
    return LBM_OK;
}

int lbm_mlp_forward(lbm_mlp *h, int batch, const float *x, float *y)
{
    if (!h || !x || batch < 1 || batch > h->maxb) return mfail("bad forward arguments");
    h->batch = batch;
    const int *S = h->sizes.data();
    k_f2bf<<<grid1((long long)batch * S[0]), 256, 0, h->stream>>>(x, h->xb, (long long)batch * S[0]);
    const bf16 *in = h->xb;
    for (int l = 0; l < h->L; ++l) {
        const bool last = l == h->L - 1;
        gemm(h, batch, S[l + 1], S[l], in, S[l], 0, h->wb + h->woff[l], S[l + 1], 0, last ? h->z[l] : nullptr,
             S[l + 1], h->p + h->boff[l], last ? 0 : 1, last ? nullptr : h->z[l], last ? nullptr : h->ab[l]);
        in = h->ab[l];
    }
    if (y)
        LBM_MCK(cudaMemcpyAsync(y, h->z[h->L - 1], sizeof(float) * (size_t)batch * S[h->L], cudaMemcpyDeviceToDevice,
                                h->stream));
    LBM_MCK(cudaGetLastError());
    return LBM_OK;
}

int lbm_mlp_backward(lbm_mlp *h, const float *target, double *loss)
{
    if (!h || !target || h->batch < 1) return mfail("bad backward arguments (run lbm_mlp_forward first)");
    const int B = h->batch;
    const int *S = h->sizes.data();
    const long long nout = (long long)B * S[h->L];
    const int nb = grid1(nout);
    k_mse<<<nb, 256, 0, h->stream>>>(h->z[h->L - 1], target, h->dz, h->dzb, nout, h->partials);
    k_sum_partials<<<1, 32, 0, h->stream>>>(h->partials, nb, h->dloss);
    for (int l = h->L - 1; l >= 0; --l) {
        const int K = S[l], N = S[l + 1];
        const bf16 *act = l == 0 ? h->xb : h->ab[l - 1];
        // dW = act^T dz   (K x N)
        gemm(h, K, N, B, act, K, 1, h->dzb, N, 0, h->g + h->woff[l], N, nullptr, 0, nullptr, nullptr);
        k_colsum<<<(N + 127) / 128, 128, 0, h->stream>>>(h->dz, B, N, h->g + h->boff[l]);
        if (l > 0) {
            // da = dz W^T   (B x K), then dz = da GELU'(z_{l-1})
            gemm(h, B, K, N, h->dzb, N, 0, h->wb + h->woff[l], N, 1, h->da, K, nullptr, 0, nullptr, nullptr);
            k_gelu_bwd<<<grid1((long long)B * K), 256, 0, h->stream>>>(h->da, h->z[l - 1], h->dz, h->dzb,
                                                                       (long long)B * K);
        }
    }
    LBM_MCK(cudaGetLastError());
    if (loss) {
        double v = 0.0;
        LBM_MCK(cudaMemcpyAsync(&v, h->dloss, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        LBM_MCK(cudaStreamSynchronize(h->stream));
        *loss = v / (double)nout;
        return check_timeout(h);
    }
    return LBM_OK;
}

int lbm_mlp_adam(lbm_mlp *h, float lr, float b1, float b2, float eps)
{
    if (!h) return mfail("null handle");
    h->t += 1;
    const float c1 = 1.f - powf(b1, (float)h->t), c2 = 1.f - powf(b2, (float)h->t);
    k_adam<<<grid1(h->nparam), 256, 0, h->stream>>>(h->p, h->g, h->m, h->v, h->nparam, lr, b1, b2, eps, c1, c2);
    k_f2bf<<<grid1(h->nparam), 256, 0, h->stream>>>(h->p, h->wb, h->nparam);
    LBM_MCK(cudaGetLastError());
    return LBM_OK;
}

} // extern "C"
