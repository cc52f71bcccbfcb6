// Per-cell arithmetic of the ES-BGK scheme on the GPU, FP32, in deviation form.
//
// Storage convention (all precisions): s_i = (g_i - w_i)/w_i and t_i = (h_i - w_i N_f/2)/w_i,
// i.e. deviations from the rest state rho = T = 1 (u = 0) scaled by the weight, so the
// small departures that carry the flow keep their full relative precision in FP32 and
// stay in the normal range of FP16/BF16.  A handle with a reference state (rho0, T0)
// stores them less that state's rest equilibrium (KParams::ref_*): the arithmetic below
// still works with deviations from rho = T = 1, the moment sums take the reference's
// constant share and the relaxation's target is shifted by it.
//
// Moments (Sec. V): rho = sum g_i, rho u = sum g_i xi_i, the second moment
// sum g_i xi_i xi_i, rho e_int = sum h_i; temperatures T_tr, T_int, T_eq, T_rel and the
// corrected tensor Lambda (Sec. II, Sec. V).  Equilibrium (Sec. IV, Eq. GExpansion):
// the truncated Hermite series sum_{n<=4} a^(n).H^(n)(xi)/n! with a^(n) from Eq. fESCoe
// is, as a function of xi, a polynomial P(xi) of degree 4.  Collecting the traces of
// a^(n) that the delta terms of H^(n) produce gives its monomial coefficients:
//   P(xi) = sum_m xi^m : C_m / m!,   C_m = sum_k (-1/2)^k / k!  tr^k a^(m+2k)
// so G_i = w_i rho P(r c_i), evaluated per velocity with integer c_i folded at compile
// time and the even / odd parts shared by each opposite pair.  With A = Lambda - delta,
// a^(n) is the n-th moment of a formal Gaussian of mean u and covariance A.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>
#include <string.h>

#include <type_traits>

#include "lattice.cuh"
#include "vec2.cuh"

namespace lbm {

enum : int { ST_FP32 = 0, ST_FP16 = 1, ST_BF16 = 2, ST_FP64 = 3 };

// raw(): the stored bits, cvt(): to the arithmetic type R (FP32, or FP64 for FP64
// storage).  The gather loads all raw values first and converts them afterwards, so every
// load of a cell is in flight at once.
template <int ST> struct Storage;
template <> struct Storage<ST_FP32> {
    using T = float;
    using Raw = float;
    using R = float;
    static __device__ __forceinline__ Raw raw(const T *p) { return __ldg(p); }
    static __device__ __forceinline__ float cvt(Raw r) { return r; }
    static __device__ __forceinline__ float ld(const T *p) { return __ldg(p); }
    static __device__ __forceinline__ void st(T *p, float v) { __stcs(p, v); }
};
template <> struct Storage<ST_FP16> {
    using T = __half;
    using Raw = unsigned short;
    using R = float;
    static __device__ __forceinline__ Raw raw(const T *p)
    {
        return __ldg(reinterpret_cast<const unsigned short *>(p));
    }
    static __device__ __forceinline__ float cvt(Raw r) { return __half2float(__ushort_as_half(r)); }
    static __device__ __forceinline__ float ld(const T *p) { return __half2float(__ldg(p)); }
    static __device__ __forceinline__ void st(T *p, float v) { __stcs(reinterpret_cast<unsigned short *>(p), __half_as_ushort(__float2half_rn(v))); }
    // two neighbouring cells' values in one 32-bit word (low half: the first cell)
    static __device__ __forceinline__ f2 cvt2(uint32_t r)
    {
        __half2 h;
        memcpy(&h, &r, 4);
        return as_f2(__half22float2(h));
    }
    static __device__ __forceinline__ void st2(T *p, f2 v)
    {
        const __half2 h = __float22half2_rn(as_float2(v));
        uint32_t r;
        memcpy(&r, &h, 4);
        __stcs(reinterpret_cast<unsigned int *>(p), r);
    }
};
template <> struct Storage<ST_BF16> {
    using T = __nv_bfloat16;
    using Raw = unsigned short;
    using R = float;
    static __device__ __forceinline__ Raw raw(const T *p)
    {
        return __ldg(reinterpret_cast<const unsigned short *>(p));
    }
    static __device__ __forceinline__ float cvt(Raw r) { return __bfloat162float(__ushort_as_bfloat16(r)); }
    static __device__ __forceinline__ float ld(const T *p) { return __bfloat162float(__ldg(p)); }
    static __device__ __forceinline__ void st(T *p, float v) { __stcs(reinterpret_cast<unsigned short *>(p), __bfloat16_as_ushort(__float2bfloat16_rn(v))); }
    static __device__ __forceinline__ f2 cvt2(uint32_t r)
    {
        __nv_bfloat162 h;
        memcpy(&h, &r, 4);
        return as_f2(__bfloat1622float2(h));
    }
    static __device__ __forceinline__ void st2(T *p, f2 v)
    {
        const __nv_bfloat162 h = __float22bfloat162_rn(as_float2(v));
        uint32_t r;
        memcpy(&r, &h, 4);
        __stcs(reinterpret_cast<unsigned int *>(p), r);
    }
};

// FP64 storage with FP64 arithmetic: for steady states that must agree with an FP64
// reference beyond the fixed-point wander of the FP32 iteration.
template <> struct Storage<ST_FP64> {
    using T = double;
    using Raw = double;
    using R = double;
    static __device__ __forceinline__ Raw raw(const T *p) { return __ldg(p); }
    static __device__ __forceinline__ double cvt(Raw r) { return r; }
    static __device__ __forceinline__ double ld(const T *p) { return __ldg(p); }
    static __device__ __forceinline__ void st(T *p, double v) { __stcs(p, v); }
};

// Per-launch parameters (passed by value; read from the constant bank).  S is the
// arithmetic type of the kernels they serve (float, or double for FP64 storage).
template <int LAT, class S = float> struct KParams {
    static constexpr int Q = Lattice<LAT>::Q;
    int nx, ny, nz;       // domain
    int nys;              // stored rows (ny + 2 gh)
    int gh;               // ghost rows beyond each wall row (0 when periodic)
    int y0, ny_comp;      // first computed domain row and number of computed rows
    int open_x;           // open (zero-gradient) ends in x instead of periodic
    long long plane;      // stored cells per population plane
    S omega;              // relaxation rate
    S kappa, a_tr, a_sig; // Lambda = (1-k)[(1-nu) T_tr d + nu sigma] + k T_eq d
    S Nf, halfNf, r;
    double r_d;           // r in FP64 (field input conversion)
    S R2_hi, R2_lo;       // r^2 as an unevaluated sum (hi + lo; lo = 0 in FP64)
    S w[Q];               // lattice weights, for the wall and flux sums
    // Shell weights as hi + lo float pairs.  Conservation of momentum rests on the
    // identity r^2 sum_i w_i c_i c_i = delta holding for the constants actually used:
    // FP32-rounded r^2 and w_i miss it by ~1e-8, which the over-relaxed collision turns
    // into a systematic drift j -> j (1 + omega eps) per step.  The moment sums therefore
    // use w_hi + w_lo and the linear equilibrium term uses R2_hi + R2_lo.
    S wsh_hi[Lattice<LAT>::NSHELL], wsh_lo[Lattice<LAT>::NSHELL];
    signed char cvel[Q][3]; // integer velocities, for runtime-indexed loops
    // Byte offsets, relative to a cell's own address in set 0 plane 0, of the source of
    // population p (p < Q: g_p, else h_{p-Q}) for a cell away from the periodic seams,
    // and of its destination; the gather then needs no per-population index arithmetic.
    long long goff[2 * Q], soff[2 * Q];
    // Reference state (rho0, T0) of the stored deviations: s_i = g_i/w_i - 1 - dg_i and
    // t_i = h_i/w_i - N_f/2 - dh_i, with dg_i = rho0 phi_i - 1, dh_i = (N_f/2)(rho0 T0 phi_i - 1)
    // and phi_i the rest equilibrium at T0 relative to the weight (a function of |c_i| only,
    // so one value per shell).  All zero for rho0 = T0 = 1.  ref_wg, ref_wh: omega dg, omega dh
    // (16-bit relaxation).  ref_hi + ref_lo: the reference's share of the raw moments,
    // sum_i w_i dg_i (drho), sum_i w_i dh_i (H) and sum_i w_i dg_i c_ia^2 (M_aa, a = 0..2),
    // from the rounded dg, dh, so that the collision conserves exactly what it sums.
    S ref_g[Lattice<LAT>::NSHELL], ref_h[Lattice<LAT>::NSHELL];
    S ref_wg[Lattice<LAT>::NSHELL], ref_wh[Lattice<LAT>::NSHELL];
    S ref_hi[5], ref_lo[5];
    // r - (S)r, and r^m / alpha! (m = |alpha| = 3, 4) as hi + lo for each monomial alpha of
    // the fourth-order polynomial: with them the lattice sums of the equilibrium close on
    // the exact constants (a rounded r^4 / 4! shifts the equilibrium's mass by that
    // rounding times its O((T - 1)^2) fourth-order part, the same in every cell and step).
    S r_lo;
    S cm_hi[Monos<Lattice<LAT>::D>::K], cm_lo[Monos<Lattice<LAT>::D>::K];
};

// State that the equilibrium needs, in deviation form.  The leading (first-order) parts
// are carried multiplied by rho (J = rho v, X = rho (A + u u), rho theta_rel) so that the
// equilibrium's conserved moments come out of the lattice sums without a division by
// rho: a rounded 1/rho is nearly the same in every cell of a smooth flow, and rho (1/rho)
// != 1 would scale momentum by the same factor every step.
// V = float for one cell, f2 for two neighbouring cells in the lanes of packed FP32 pairs.
template <int D, class V = float> struct EqState {
    V drho, rho, inv_rho;
    V J[D];               // rho v, v = u / r the lattice-unit velocity
    V u[D];               // velocity (xi units), for second-order terms
    V X[D][D];            // rho (A + u u), A = Lambda - delta
    V A[D][D];            // A, for second-order terms
    V rth_rel;            // rho (T_rel - 1)
    V th_rel;             // T_rel - 1
};

// Monomial coefficients of q(xi) = P(xi) - 1 at xi = r c, for the state s, up to the
// expansion's order N.
template <int D, class V = float, int N = 4> struct PolyCoef {
    static constexpr int K = Monos<D, N>::K;
    V k[K];
};

template <int D, class V>
__device__ __forceinline__ V c3_of(const V (&A)[D][D], const V (&u)[D], int a, int b, int c)
{
    return A[a][b] * u[c] + A[a][c] * u[b] + A[b][c] * u[a] + u[a] * u[b] * u[c];
}

template <int D, class V>
__device__ __forceinline__ V c4_of(const V (&A)[D][D], const V (&u)[D], int a, int b, int c, int d)
{
    return A[a][b] * A[c][d] + A[a][c] * A[b][d] + A[a][d] * A[b][c]
         + A[a][b] * u[c] * u[d] + A[a][c] * u[b] * u[d] + A[a][d] * u[b] * u[c]
         + A[b][c] * u[a] * u[d] + A[b][d] * u[a] * u[c] + A[c][d] * u[a] * u[b]
         + u[a] * u[b] * u[c] * u[d];
}

// Probabilists' Hermite polynomials He_k(x) = sum_j he_coef(k, j) x^j, from the
// recurrence He_k = x He_{k-1} - (k - 1) He_{k-2}, He_0 = 1, He_1 = x.
LBM_HD constexpr int he_coef(int k, int j)
{
    if (j < 0 || j > k) return 0;
    if (k == 0) return 1;
    if (k == 1) return j == 1 ? 1 : 0;
    return he_coef(k - 1, j - 1) - (k - 1) * he_coef(k - 2, j);
}

// Product of homogeneous polynomials in (t_x, t_y), f[a] the coefficient of t_x^a t_y^(n-a).
template <int NA, int NB, class V>
__device__ __forceinline__ void hmul(const V (&f)[NA], const V (&g)[NB], V (&out)[NA + NB - 1])
{
#pragma unroll
    for (int a = 0; a < NA + NB - 1; ++a) out[a] = 0.f;
#pragma unroll
    for (int a = 0; a < NA; ++a)
#pragma unroll
        for (int b = 0; b < NB; ++b) out[a + b] = vfma(f[a], g[b], out[a + b]);
}

// Fifth- and sixth-order terms of the 2-D expansion (Sec. IV: a^(5), a^(6), the Burnett
// order), added to the monomial coefficients.  With a^(n) . H^(n) / n! written over
// multi-indices alpha as b_alpha He_alpha(xi), b_alpha is the t^alpha coefficient of the
// generating function exp(u.t + t.(Lambda - delta).t / 2) of the Gaussian's Hermite
// coefficients (the same sums over Lambda^beta delta^(alpha-beta) u^(n-2 alpha) products as
// Eq. fESCoe): with P1 = u.t and P2 = t.A.t / 2, its degree-5 part is
// P1^5/120 + P1^3 P2/6 + P1 P2^2/2 and its degree-6 part P1^6/720 + P1^4 P2/24 +
// P1^2 P2^2/4 + P2^3/6.  He_alpha(xi) = He_{a}(xi_x) He_{n-a}(xi_y) then spreads each b_alpha
// over the monomials of degree n, n-2, ...; xi = r c scales degree m by r^m.
template <class V>
__device__ __forceinline__ void burnett_terms(const EqState<2, V> &s, float r, PolyCoef<2, V, 6> &pc)
{
    const V p1[2] = {s.u[1], s.u[0]};
    const V p2[3] = {0.5f * s.A[1][1], s.A[0][1], 0.5f * s.A[0][0]};
    V p1_2[3], p1_3[4], p1_4[5], p1_5[6], p1_6[7], p2_2[5], p2_3[7];
    hmul(p1, p1, p1_2);
    hmul(p1_2, p1, p1_3);
    hmul(p1_3, p1, p1_4);
    hmul(p1_4, p1, p1_5);
    hmul(p1_5, p1, p1_6);
    hmul(p2, p2, p2_2);
    hmul(p2_2, p2, p2_3);
    V t5a[6], t5b[6], t6a[7], t6b[7];
    hmul(p1_3, p2, t5a);
    hmul(p1, p2_2, t5b);
    hmul(p1_4, p2, t6a);
    hmul(p1_2, p2_2, t6b);
    V b5[6], b6[7];
#pragma unroll
    for (int a = 0; a < 6; ++a) b5[a] = (1.f / 120.f) * p1_5[a] + (1.f / 6.f) * t5a[a] + 0.5f * t5b[a];
#pragma unroll
    for (int a = 0; a < 7; ++a)
        b6[a] = (1.f / 720.f) * p1_6[a] + (1.f / 24.f) * t6a[a] + 0.25f * t6b[a] + (1.f / 6.f) * p2_3[a];
    // monomial xi_x^i xi_y^j: odd degrees from n = 5, even degrees from n = 6
    float rp[7] = {1.f, r, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int m = 2; m < 7; ++m) rp[m] = rp[m - 1] * r;
    static_for<0, 7>([&](auto II) {
        constexpr int i = decltype(II)::value;
        static_for<0, 7 - i>([&](auto JJ) {
            constexpr int j = decltype(JJ)::value;
            constexpr int n = (i + j) % 2 ? 5 : 6;
            if constexpr (i + j <= n) {
                V acc = 0.f;
                static_for<0, n + 1>([&](auto AA) {
                    constexpr int a = decltype(AA)::value;
                    constexpr int h = he_coef(a, i) * he_coef(n - a, j);
                    if constexpr (h != 0) {
                        if constexpr (n == 5) acc = vfma(V((float)h), b5[a], acc);
                        else acc = vfma(V((float)h), b6[a], acc);
                    }
                });
                constexpr int K = mono_k2(i, j);
                static_assert(Monos<2, 6>::M.e[K][0] == i && Monos<2, 6>::M.e[K][1] == j, "monomial order");
                if constexpr (i + j <= 4) pc.k[K] = vfma(s.rho * rp[i + j], acc, pc.k[K]);
                else pc.k[K] = s.rho * rp[i + j] * acc;
            }
        });
    });
}

// Coefficients of rho q(xi) in the monomials of c (xi = r c): K_alpha = rho r^|alpha| C_alpha / alpha!
// for the fourth-order expansion (Eq. GExpansion); with N = 6 (2-D) the fifth- and
// sixth-order terms are added.
// PRECISE: r^2 as hi + lo (FP32 storage).  EXACT (with PRECISE): the third- and
// fourth-order constants r^m / alpha! as hi + lo too; their rounding shifts the
// equilibrium's mass, momentum and energy in proportion to its (T - 1) terms, negligible
// near the lattice's unit temperature and compiled in for handles with a reference state.
// Otherwise CM: the constants r^m / alpha! from the launch parameters (one product per
// coefficient), else r^m and 1/alpha! formed in the kernel.
template <bool PRECISE, bool EXACT, bool CM = true, int D, class V, int N, class KP>
__device__ __forceinline__ void poly_coeffs(const EqState<D, V> &s, const KP &kp, PolyCoef<D, V, N> &pc)
{
    using S = typename ScalarOf<V>::type;
    const S r = kp.r, R2_hi = kp.R2_hi, R2_lo = PRECISE ? kp.R2_lo : S(0);
    const auto &A = s.A;
    const auto &u = s.u;
    const V rho = s.rho;
    V trA = 0.f, u2 = 0.f, trA2 = 0.f, uAu = 0.f, trX = 0.f;
    V Au[D], AJ[D], A2[D][D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
        trA += A[a][a];
        trX += s.X[a][a];
        u2 += u[a] * u[a];
        V t = 0.f, tj = 0.f;
#pragma unroll
        for (int b = 0; b < D; ++b) {
            t += A[a][b] * u[b];
            tj += A[a][b] * s.J[b];
        }
        Au[a] = t;
        AJ[a] = tj;
    }
#pragma unroll
    for (int a = 0; a < D; ++a) {
        uAu += u[a] * Au[a];
#pragma unroll
        for (int b = 0; b < D; ++b) {
            V t = 0.f;
#pragma unroll
            for (int c = 0; c < D; ++c) t += A[a][c] * A[c][b];
            A2[a][b] = t;
            trA2 += A[a][b] * A[a][b];
        }
    }
    // rho (C_0 - 1) = -rho tr a2 / 2 + rho tr^2 a4 / 8,  rho tr a2 = tr X
    const V k0 = -0.5f * trX + 0.125f * rho * (trA * trA + 2.f * trA2 + 2.f * u2 * trA + 4.f * uAu + u2 * u2);
    // rho r C_1 = r^2 (J - (tr A J + 2 A J + u^2 J)/2)
    V k1[D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const V y = s.J[a] - 0.5f * (trA * s.J[a] + 2.f * AJ[a] + u2 * s.J[a]);
        k1[a] = vfma(R2_hi, y, R2_lo * y);
    }
    // rho C_2 = X - rho tr a4 / 2 (the trace part is second order)
    V c2[D][D];
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b)
            c2[a][b] = s.X[a][b]
                     - 0.5f * rho * (trA * A[a][b] + 2.f * A2[a][b] + trA * u[a] * u[b] + 2.f * Au[a] * u[b]
                                     + 2.f * Au[b] * u[a] + u2 * A[a][b] + u2 * u[a] * u[b]);
    const S r3 = R2_hi * r, r4 = R2_hi * R2_hi;
    static_for<0, Monos<D>::K>([&](auto KK) {
        constexpr int K = decltype(KK)::value;
        constexpr int m = Monos<D>::M.deg[K];
        constexpr S inv = (S)inv_alpha_factorial<D, K>();
        constexpr int i0 = mono_index<D, K>(0), i1 = mono_index<D, K>(1);
        constexpr int i2 = mono_index<D, K>(2), i3 = mono_index<D, K>(3);
        V v;
        if constexpr (m == 0) v = k0;
        else if constexpr (m == 1) v = k1[i0];
        else if constexpr (m == 2) {
            // r^2 in hi + lo so that the mass and energy sums close on the same constant
            // (inv = 1 or 1/2, exact)
            const V x = inv * c2[i0][i1];
            v = vfma(R2_hi, x, R2_lo * x);
        } else if constexpr (PRECISE && EXACT) {
            const V y = rho * (m == 3 ? c3_of<D, V>(A, u, i0, i1, i2) : c4_of<D, V>(A, u, i0, i1, i2, i3));
            v = vfma(kp.cm_hi[K], y, kp.cm_lo[K] * y);
        } else if constexpr (!PRECISE && CM) {
            v = kp.cm_hi[K] * (rho * (m == 3 ? c3_of<D, V>(A, u, i0, i1, i2) : c4_of<D, V>(A, u, i0, i1, i2, i3)));
        }
        else if constexpr (m == 3) v = r3 * inv * rho * c3_of<D, V>(A, u, i0, i1, i2);
        else v = r4 * inv * rho * c4_of<D, V>(A, u, i0, i1, i2, i3);
        pc.k[K] = v;
    });
    if constexpr (N == 6) {
        static_assert(D == 2, "the sixth-order expansion is built for the 2-D lattice");
        burnett_terms<V>(s, r, pc);
    }
}

// Even and odd parts of q at velocity I (compile-time), q(c_I) = E + O, q(-c_I) = E - O.
template <int LAT, int I, class V>
__device__ __forceinline__ void poly_eval_pair(const PolyCoef<Lattice<LAT>::D, V, Lattice<LAT>::ORDER> &pc, V &E,
                                               V &O)
{
    constexpr int D = Lattice<LAT>::D;
    using M = Monos<D, Lattice<LAT>::ORDER>;
    V e = 0.f, o = 0.f;
    static_for<0, M::K>([&](auto KK) {
        constexpr int K = decltype(KK)::value;
        constexpr int mv = mono_at<LAT, I, K>();
        if constexpr (mv != 0) {
            if constexpr (M::M.deg[K] % 2 == 0) {
                if constexpr (mv == 1) e += pc.k[K];
                else if constexpr (mv == -1) e -= pc.k[K];
                else e = vfma(V((float)mv), pc.k[K], e);
            } else {
                if constexpr (mv == 1) o += pc.k[K];
                else if constexpr (mv == -1) o -= pc.k[K];
                else o = vfma(V((float)mv), pc.k[K], o);
            }
        }
    });
    E = e;
    O = o;
}

// Raw deviation moments of one cell's populations (s = g~/w, t = h~/w).
template <int D, class V = float> struct RawMoments {
    V drho;               // sum g~
    V J[D];               // sum g~ c
    V M[D][D];            // sum g~ c c
    V H;                  // sum h~
};

// The reference state's share of the raw moments (see KParams::ref_*), added as hi + lo
// so that no constant rounding error enters the conserved sums.
template <int LAT, class S, class V>
__device__ __forceinline__ void add_reference(const KParams<LAT, S> &kp, RawMoments<Lattice<LAT>::D, V> &m)
{
    constexpr int D = Lattice<LAT>::D;
    m.drho = (m.drho + V(kp.ref_lo[0])) + V(kp.ref_hi[0]);
    m.H = (m.H + V(kp.ref_lo[1])) + V(kp.ref_hi[1]);
#pragma unroll
    for (int a = 0; a < D; ++a) m.M[a][a] = (m.M[a][a] + V(kp.ref_lo[2 + a])) + V(kp.ref_hi[2 + a]);
}

// Population accessors: pop.template sv<I>() / tv<I>() return the scaled deviations s_I,
// t_I of one cell (from registers, or from a shared-memory tile) as V; refresh() is
// called between the moment sums and the relaxation (a no-op unless the accessor
// re-converts or re-reads stored values there instead of keeping them live), and
// prefetch<P>() before the opposite pair P is used (a no-op unless the accessor reads
// memory in chunks of pairs).
template <class R = float> struct ArrayPopT {
    using V = R;
    const R *s, *t;
    __device__ __forceinline__ void refresh() {}
    template <int P> __device__ __forceinline__ void prefetch() const {}
    template <int I> __device__ __forceinline__ R sv() const { return s[I]; }
    template <int I> __device__ __forceinline__ R tv() const { return t[I]; }
};
using ArrayPop = ArrayPopT<float>;

// PRECISE (FP32 storage): hi + lo shell weights and an error-free momentum fold.  The
// 16-bit storage forms round every population to 2^-11 (FP16) or 2^-8 (BF16) each step,
// far above these 1e-8 effects, and fold with the FP32 weights alone; FP64 storage folds
// with the FP64 weights (plain double sums).
template <int LAT, bool PRECISE = true, class Pop, class S>
__device__ __forceinline__ void raw_moments(const KParams<LAT, S> &kp, const Pop &pop,
                                            RawMoments<Lattice<LAT>::D, typename Pop::V> &m)
{
    constexpr int D = Lattice<LAT>::D;
    constexpr int Q = Lattice<LAT>::Q;
    using V = typename Pop::V;
    static_assert(!PRECISE || std::is_same<V, float>::value, "the compensated sums are scalar");
    constexpr int NM = 2 + D + D * (D + 1) / 2; // drho, H, J, M (upper triangle)
    // hi and lo accumulators of the weighted sums
    V hi[NM], lo[NM];
#pragma unroll
    for (int k = 0; k < NM; ++k) hi[k] = lo[k] = 0.f;
    // unweighted partial sums of the current shell (velocities come shell by shell)
    V part[NM];
#pragma unroll
    for (int k = 0; k < NM; ++k) part[k] = 0.f;
    part[0] = pop.template sv<0>();
    part[1] = pop.template tv<0>();
    // Weighted fold of one shell's partial sums.  The momentum components (k = 2..D+1) fold
    // error-free (TwoProduct + TwoSum into lo): their rounding on a smooth flow is coherent
    // from cell to cell and from step to step, and the collision would inject it into the
    // conserved momentum as a slow systematic drift.
    auto fold = [&](int sh) {
        const S wh = kp.wsh_hi[sh], wl = kp.wsh_lo[sh];
        if constexpr (!PRECISE) {
#pragma unroll
            for (int k = 0; k < NM; ++k) {
                hi[k] = vfma(V(wh), part[k], hi[k]);
                part[k] = 0.f;
            }
            return;
        } else {
#pragma unroll
            for (int k = 0; k < NM; ++k) {
                if (k >= 2 && k < 2 + D) {
                    // _rn intrinsics: never contracted into FMAs, which would break the
                    // error-free transformations
                    const float p = __fmul_rn(wh, part[k]);
                    const float pe = fmaf(wh, part[k], -p);
                    const float sum = __fadd_rn(hi[k], p);
                    const float bv = __fsub_rn(sum, hi[k]);
                    const float e = __fadd_rn(__fsub_rn(hi[k], __fsub_rn(sum, bv)), __fsub_rn(p, bv));
                    hi[k] = sum;
                    lo[k] = fmaf(wl, part[k], lo[k] + (pe + e));
                } else {
                    hi[k] = fmaf(wh, part[k], hi[k]);
                    lo[k] = fmaf(wl, part[k], lo[k]);
                }
                part[k] = 0.f;
            }
        }
    };
    fold(0);
    // opposite pairs: the sum feeds the even moments, the difference the odd ones
    static_for<0, (Q - 1) / 2>([&](auto PP) {
        constexpr int I = 1 + 2 * decltype(PP)::value;
        constexpr int sh = Lattice<LAT>::T.shell[I];
        pop.template prefetch<decltype(PP)::value>();
        const V sa = pop.template sv<I>(), sb = pop.template sv<I + 1>();
        const V ev = sa + sb;
        const V od = sa - sb;
        part[0] += ev;
        part[1] += pop.template tv<I>() + pop.template tv<I + 1>();
        int k = 2;
        static_for<0, D>([&](auto AA) {
            constexpr int a = decltype(AA)::value;
            constexpr int ca = cv<LAT, I, a>();
            if constexpr (ca == 1) part[2 + a] += od;
            else if constexpr (ca == -1) part[2 + a] -= od;
            else if constexpr (ca != 0) part[2 + a] = vfma(V((float)ca), od, part[2 + a]);
        });
        k = 2 + D;
        static_for<0, D>([&](auto AA) {
            constexpr int a = decltype(AA)::value;
            static_for<a, D>([&](auto BB) {
                constexpr int b = decltype(BB)::value;
                constexpr int idx = 2 + D + a * D - a * (a - 1) / 2 + (b - a);
                constexpr int cab = cv<LAT, I, a>() * cv<LAT, I, b>();
                if constexpr (cab == 1) part[idx] += ev;
                else if constexpr (cab == -1) part[idx] -= ev;
                else if constexpr (cab != 0) part[idx] = vfma(V((float)cab), ev, part[idx]);
            });
        });
        (void)k;
        constexpr bool last = (I + 2 >= Q) || (Lattice<LAT>::T.shell[I + 2] != sh);
        if constexpr (last) fold(sh);
    });
    V tot[NM];
#pragma unroll
    for (int k = 0; k < NM; ++k) tot[k] = hi[k] + lo[k];
    m.drho = tot[0];
    m.H = tot[1];
#pragma unroll
    for (int a = 0; a < D; ++a) m.J[a] = tot[2 + a];
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = a; b < D; ++b) {
            const V v = tot[2 + D + a * D - a * (a - 1) / 2 + (b - a)];
            m.M[a][b] = v;
            m.M[b][a] = v;
        }
}

// Macroscopic state from raw moments, rho-weighted: P = r^2 M - drho delta =
// rho (sigma - delta) + rho u u, rho sdev = rho (sigma - delta), rho theta = rho (T - 1).
template <int D, class V = float> struct CellState {
    V drho, rho, inv_rho;
    V J[D];               // rho v
    V v[D];               // lattice-unit velocity J / rho
    V u[D];               // r v
    V ruu[D][D];          // rho u u
    V rsdev[D][D];        // rho (sigma - delta)
    V rth_tr, rth_int, rth_eq, rth_rel;
    V th_eq;              // T_eq - 1
};

// FASTDIV (the packed-lane collision of 16-bit storage): divisions by the fast reciprocal,
// whose ~2-ulp error is far below the storage rounding (2^-11, 2^-8); otherwise IEEE division.
template <class V> __device__ __forceinline__ V fast_inv(V x);
template <> __device__ __forceinline__ float fast_inv<float>(float x) { return __fdividef(1.f, x); }
template <> __device__ __forceinline__ f2 fast_inv<f2>(f2 x) { return f2(__fdividef(1.f, x.x), __fdividef(1.f, x.y)); }

// PRECISE: u = r v with r as hi + lo (a rounded r scales the velocity of the equilibrium's
// third- and fourth-order terms by the same factor in every cell, a momentum bias in
// proportion to T - 1: used with the exact constants of poly_coeffs).
template <int LAT, bool FASTDIV = false, bool PRECISE = false, class V, class S>
__device__ __forceinline__ void cell_state(const KParams<LAT, S> &kp, const RawMoments<Lattice<LAT>::D, V> &m,
                                           CellState<Lattice<LAT>::D, V> &c)
{
    constexpr int D = Lattice<LAT>::D;
    c.drho = m.drho;
    c.rho = 1.f + m.drho;
    if constexpr (FASTDIV) c.inv_rho = fast_inv(c.rho);
    else c.inv_rho = 1.f / c.rho;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        c.J[a] = m.J[a];
        c.v[a] = m.J[a] * c.inv_rho;
        if constexpr (PRECISE) c.u[a] = vfma(V(kp.r), c.v[a], V(kp.r_lo) * c.v[a]);
        else c.u[a] = kp.r * c.v[a];
    }
    V tr = 0.f;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = a; b < D; ++b) {
            // r^2 M in hi + lo: the temperature sees the r^2 the energy sums use
            const V R2M = vfma(kp.R2_hi, m.M[a][b], kp.R2_lo * m.M[a][b]);
            const V ruu = kp.R2_hi * (c.J[a] * c.v[b]);
            const V v = (R2M - (a == b ? m.drho : V(0.f))) - ruu;
            c.ruu[a][b] = c.ruu[b][a] = ruu;
            c.rsdev[a][b] = c.rsdev[b][a] = v;
            if (a == b) tr += v;
        }
    c.rth_tr = tr * (S(1) / S(D));
    if (kp.Nf > 0.f) {
        if constexpr (FASTDIV) {
            c.rth_int = __fdividef(2.f, kp.Nf) * m.H - m.drho;
            c.rth_eq = (D * c.rth_tr + kp.Nf * c.rth_int) * __fdividef(1.f, D + kp.Nf);
        } else {
            c.rth_int = 2.f * m.H / kp.Nf - m.drho;
            c.rth_eq = (D * c.rth_tr + kp.Nf * c.rth_int) / (D + kp.Nf);
        }
        // T_rel = T_int + kappa (T_eq - T_int): equal to T_int at equilibrium whatever the
        // rounding of kappa
        c.rth_rel = vfma(kp.kappa, c.rth_eq - c.rth_int, c.rth_int);
    } else {
        c.rth_int = 0.f;
        c.rth_eq = c.rth_tr;
        c.rth_rel = c.rth_tr;
    }
    c.th_eq = c.rth_eq * c.inv_rho;
}

// Lambda - delta = theta_tr delta + (1-kappa) nu (sigma - T_tr delta) + kappa (theta_eq - theta_tr) delta,
// the same tensor as (1-kappa)[(1-nu) T_tr delta + nu sigma] + kappa T_eq delta - delta written so
// that its trace, D theta_tr + kappa D (theta_eq - theta_tr), does not depend on rounded
// complements of kappa (energy closes exactly in the collision).
template <int LAT, class V, class S>
__device__ __forceinline__ void es_state(const KParams<LAT, S> &kp, const CellState<Lattice<LAT>::D, V> &c,
                                         EqState<Lattice<LAT>::D, V> &e)
{
    constexpr int D = Lattice<LAT>::D;
    e.drho = c.drho;
    e.rho = c.rho;
    e.inv_rho = c.inv_rho;
    e.rth_rel = c.rth_rel;
    e.th_rel = c.rth_rel * c.inv_rho;
    const V iso = vfma(kp.kappa, c.rth_eq - c.rth_tr, c.rth_tr);
#pragma unroll
    for (int a = 0; a < D; ++a) {
        e.J[a] = c.J[a];
        e.u[a] = c.u[a];
#pragma unroll
        for (int b = 0; b < D; ++b) {
            const V rA = kp.a_sig * (c.rsdev[a][b] - (a == b ? c.rth_tr : V(0.f))) + (a == b ? iso : V(0.f));
            e.X[a][b] = rA + c.ruu[a][b];
            e.A[a][b] = rA * c.inv_rho;
        }
    }
}

// Maxwellian state (Lambda = T delta) of (rho, u = r v, T) given the lattice velocity v.
template <int D, class R>
__device__ __forceinline__ void maxwell_state(R drho, const R (&v)[D], R r, R r_lo, R R2_hi, R th, EqState<D, R> &e)
{
    e.drho = drho;
    e.rho = 1.f + drho;
    e.inv_rho = 1.f / e.rho;
    e.th_rel = th;
    e.rth_rel = e.rho * th;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        e.J[a] = e.rho * v[a];
        e.u[a] = vfma(r, v[a], r_lo * v[a]);
    }
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) {
            e.A[a][b] = a == b ? th : 0.f;
            e.X[a][b] = (a == b ? e.rth_rel : 0.f) + R2_hi * (e.J[a] * v[b]);
        }
}

// Scaled equilibrium deviations at velocity I given Pq = rho q(c_I):
//   G~_I / w_I = drho + Pq,   H~_I / w_I = (N_f/2)(drho + rho th_rel) + (N_f/2)(1 + th_rel) Pq
template <class V = float> struct EqScalT {
    V drho, hb, hr;
    typename ScalarOf<V>::type om1; // 1 - omega
    V wdrho, whb, whr;    // omega-scaled terms (16-bit storage relaxation)
};
using EqScal = EqScalT<float>;

template <int D, class V, class S>
__device__ __forceinline__ EqScalT<V> eq_scalars(const EqState<D, V> &e, S halfNf)
{
    EqScalT<V> z;
    z.drho = e.drho;
    z.hb = halfNf * (e.drho + e.rth_rel);
    z.hr = halfNf * (1.f + e.th_rel);
    return z;
}

} // namespace lbm
