// Per-cell arithmetic of the ES-BGK scheme on the GPU, FP32, in deviation form.
//
// Storage convention (all precisions): s_i = (g_i - w_i)/w_i and t_i = (h_i - w_i N_f/2)/w_i,
// i.e. deviations from the rest state rho = T = 1 (u = 0) scaled by the weight, so the
// small departures that carry the flow keep their full relative precision in FP32 and
// stay in the normal range of FP16/BF16.
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

#include "lattice.cuh"

namespace lbm {

enum : int { ST_FP32 = 0, ST_FP16 = 1, ST_BF16 = 2 };

template <int ST> struct Storage;
template <> struct Storage<ST_FP32> {
    using T = float;
    static __device__ __forceinline__ float ld(const T *p) { return __ldg(p); }
    static __device__ __forceinline__ void st(T *p, float v) { __stcs(p, v); }
};
template <> struct Storage<ST_FP16> {
    using T = __half;
    static __device__ __forceinline__ float ld(const T *p) { return __half2float(__ldg(p)); }
    static __device__ __forceinline__ void st(T *p, float v) { *p = __float2half_rn(v); }
};
template <> struct Storage<ST_BF16> {
    using T = __nv_bfloat16;
    static __device__ __forceinline__ float ld(const T *p) { return __bfloat162float(__ldg(p)); }
    static __device__ __forceinline__ void st(T *p, float v) { *p = __float2bfloat16_rn(v); }
};

// Per-launch parameters (passed by value; read from the constant bank).
template <int LAT> struct KParams {
    static constexpr int Q = Lattice<LAT>::Q;
    int nx, ny, nz;       // domain
    int nys;              // stored rows (ny + 2 gh)
    int gh;               // ghost rows beyond each wall row (0 when periodic)
    int y0, ny_comp;      // first computed domain row and number of computed rows
    long long plane;      // stored cells per population plane
    float omega;          // relaxation rate
    float kappa, a_tr, a_sig; // Lambda = (1-k)[(1-nu) T_tr d + nu sigma] + k T_eq d
    float Nf, halfNf, r;
    double r_d;           // r in FP64 (field input conversion)
    float R2_hi, R2_lo;   // r^2 as an unevaluated float sum (hi + lo)
    float w[Q];           // lattice weights (FP32), for the wall and flux sums
    // Shell weights as hi + lo float pairs.  Conservation of momentum rests on the
    // identity r^2 sum_i w_i c_i c_i = delta holding for the constants actually used:
    // FP32-rounded r^2 and w_i miss it by ~1e-8, which the over-relaxed collision turns
    // into a systematic drift j -> j (1 + omega eps) per step.  The moment sums therefore
    // use w_hi + w_lo and the linear equilibrium term uses R2_hi + R2_lo.
    float wsh_hi[Lattice<LAT>::NSHELL], wsh_lo[Lattice<LAT>::NSHELL];
};

// State that the equilibrium needs, in deviation form.
template <int D> struct EqState {
    float drho, rho;      // rho - 1, rho
    float u[D];           // velocity (xi units)
    float v[D];           // velocity in lattice units, u / r
    float A[D][D];        // Lambda - delta
    float th_rel;         // T_rel - 1
};

// Monomial coefficients of q(xi) = P(xi) - 1 at xi = r c, for the state s.
template <int D> struct PolyCoef {
    static constexpr int K = Monos<D>::K;
    float k[K];
};

template <int D>
__device__ __forceinline__ float c3_of(const float (&A)[D][D], const float (&u)[D], int a, int b, int c)
{
    return A[a][b] * u[c] + A[a][c] * u[b] + A[b][c] * u[a] + u[a] * u[b] * u[c];
}

template <int D>
__device__ __forceinline__ float c4_of(const float (&A)[D][D], const float (&u)[D], int a, int b, int c, int d)
{
    return A[a][b] * A[c][d] + A[a][c] * A[b][d] + A[a][d] * A[b][c]
         + A[a][b] * u[c] * u[d] + A[a][c] * u[b] * u[d] + A[a][d] * u[b] * u[c]
         + A[b][c] * u[a] * u[d] + A[b][d] * u[a] * u[c] + A[c][d] * u[a] * u[b]
         + u[a] * u[b] * u[c] * u[d];
}

template <int D>
__device__ __forceinline__ void poly_coeffs(const EqState<D> &s, float r, float R2_hi, float R2_lo,
                                            PolyCoef<D> &pc)
{
    const auto &A = s.A;
    const auto &u = s.u;
    float trA = 0.f, u2 = 0.f, trA2 = 0.f, uAu = 0.f;
    float Au[D], A2[D][D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
        trA += A[a][a];
        u2 += u[a] * u[a];
        float t = 0.f;
#pragma unroll
        for (int b = 0; b < D; ++b) t += A[a][b] * u[b];
        Au[a] = t;
    }
#pragma unroll
    for (int a = 0; a < D; ++a) {
        uAu += u[a] * Au[a];
#pragma unroll
        for (int b = 0; b < D; ++b) {
            float t = 0.f;
#pragma unroll
            for (int c = 0; c < D; ++c) t += A[a][c] * A[c][b];
            A2[a][b] = t;
            trA2 += A[a][b] * A[a][b];
        }
    }
    // C_0 - 1 = -tr a2 / 2 + tr^2 a4 / 8
    const float c0 = -0.5f * (trA + u2)
                   + 0.125f * (trA * trA + 2.f * trA2 + 2.f * u2 * trA + 4.f * uAu + u2 * u2);
    // r C_1 = r (a1 - tr a3 / 2) = r^2 y with y = v - (tr A v + 2 A v + u^2 v)/2, v = u/r
    float k1[D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
        float Av = 0.f;
#pragma unroll
        for (int b = 0; b < D; ++b) Av += A[a][b] * s.v[b];
        const float y = s.v[a] - 0.5f * (trA * s.v[a] + 2.f * Av + u2 * s.v[a]);
        k1[a] = fmaf(R2_hi, y, R2_lo * y);
    }
    // C_2 = a2 - tr a4 / 2
    float c2[D][D];
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b)
            c2[a][b] = A[a][b] + u[a] * u[b]
                     - 0.5f * (trA * A[a][b] + 2.f * A2[a][b] + trA * u[a] * u[b] + 2.f * Au[a] * u[b]
                               + 2.f * Au[b] * u[a] + u2 * A[a][b] + u2 * u[a] * u[b]);
    const float r3 = R2_hi * r, r4 = R2_hi * R2_hi;
    static_for<0, PolyCoef<D>::K>([&](auto KK) {
        constexpr int K = decltype(KK)::value;
        constexpr int m = Monos<D>::M.deg[K];
        constexpr float inv = (float)inv_alpha_factorial<D, K>();
        constexpr int i0 = mono_index<D, K>(0), i1 = mono_index<D, K>(1);
        constexpr int i2 = mono_index<D, K>(2), i3 = mono_index<D, K>(3);
        float v;
        if constexpr (m == 0) v = c0;
        else if constexpr (m == 1) v = k1[i0];
        else if constexpr (m == 2) {
            // leading even term: r^2 in hi + lo so that mass and energy sums close exactly
            const float x = inv * c2[i0][i1];
            v = fmaf(R2_hi, x, R2_lo * x);
        }
        else if constexpr (m == 3) v = r3 * inv * c3_of<D>(A, u, i0, i1, i2);
        else v = r4 * inv * c4_of<D>(A, u, i0, i1, i2, i3);
        pc.k[K] = v;
    });
}

// Even and odd parts of q at velocity I (compile-time), q(c_I) = E + O, q(-c_I) = E - O.
template <int LAT, int I>
__device__ __forceinline__ void poly_eval_pair(const PolyCoef<Lattice<LAT>::D> &pc, float &E, float &O)
{
    constexpr int D = Lattice<LAT>::D;
    float e = 0.f, o = 0.f;
    static_for<0, Monos<D>::K>([&](auto KK) {
        constexpr int K = decltype(KK)::value;
        constexpr int mv = mono_at<LAT, I, K>();
        if constexpr (mv != 0) {
            if constexpr (Monos<D>::M.deg[K] % 2 == 0) {
                if constexpr (mv == 1) e += pc.k[K];
                else if constexpr (mv == -1) e -= pc.k[K];
                else e = fmaf((float)mv, pc.k[K], e);
            } else {
                if constexpr (mv == 1) o += pc.k[K];
                else if constexpr (mv == -1) o -= pc.k[K];
                else o = fmaf((float)mv, pc.k[K], o);
            }
        }
    });
    E = e;
    O = o;
}

// Raw deviation moments of one cell's populations (s = g~/w, t = h~/w).
template <int D> struct RawMoments {
    float drho;           // sum g~
    float J[D];           // sum g~ c
    float M[D][D];        // sum g~ c c
    float H;              // sum h~
};

template <int LAT>
__device__ __forceinline__ void raw_moments(const KParams<LAT> &kp, const float *s, const float *t,
                                            RawMoments<Lattice<LAT>::D> &m)
{
    constexpr int D = Lattice<LAT>::D;
    constexpr int Q = Lattice<LAT>::Q;
    constexpr int NM = 2 + D + D * (D + 1) / 2; // drho, H, J, M (upper triangle)
    // hi and lo accumulators of the weighted sums
    float hi[NM], lo[NM];
#pragma unroll
    for (int k = 0; k < NM; ++k) hi[k] = lo[k] = 0.f;
    // unweighted partial sums of the current shell (velocities come shell by shell)
    float part[NM];
#pragma unroll
    for (int k = 0; k < NM; ++k) part[k] = 0.f;
    part[0] = s[0];
    part[1] = t[0];
    auto fold = [&](int sh) {
#pragma unroll
        for (int k = 0; k < NM; ++k) {
            hi[k] = fmaf(kp.wsh_hi[sh], part[k], hi[k]);
            lo[k] = fmaf(kp.wsh_lo[sh], part[k], lo[k]);
            part[k] = 0.f;
        }
    };
    fold(0);
    // opposite pairs: the sum feeds the even moments, the difference the odd ones
    static_for<0, (Q - 1) / 2>([&](auto PP) {
        constexpr int I = 1 + 2 * decltype(PP)::value;
        constexpr int sh = Lattice<LAT>::T.shell[I];
        const float ev = s[I] + s[I + 1];
        const float od = s[I] - s[I + 1];
        part[0] += ev;
        part[1] += t[I] + t[I + 1];
        int k = 2;
        static_for<0, D>([&](auto AA) {
            constexpr int a = decltype(AA)::value;
            constexpr int ca = cv<LAT, I, a>();
            if constexpr (ca == 1) part[2 + a] += od;
            else if constexpr (ca == -1) part[2 + a] -= od;
            else if constexpr (ca != 0) part[2 + a] = fmaf((float)ca, od, part[2 + a]);
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
                else if constexpr (cab != 0) part[idx] = fmaf((float)cab, ev, part[idx]);
            });
        });
        (void)k;
        constexpr bool last = (I + 2 >= Q) || (Lattice<LAT>::T.shell[I + 2] != sh);
        if constexpr (last) fold(sh);
    });
    float tot[NM];
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
            const float v = tot[2 + D + a * D - a * (a - 1) / 2 + (b - a)];
            m.M[a][b] = v;
            m.M[b][a] = v;
        }
}

// Macroscopic state from raw moments: u, sigma - delta, theta = T - 1 for T_tr, T_int,
// T_eq, T_rel, and Lambda - delta.
template <int D> struct CellState {
    float drho, rho, inv_rho;
    float v[D];           // lattice-unit velocity J / rho
    float u[D];           // r v
    float sdev[D][D];     // sigma - delta
    float th_tr, th_int, th_eq, th_rel;
};

template <int LAT>
__device__ __forceinline__ void cell_state(const KParams<LAT> &kp, const RawMoments<Lattice<LAT>::D> &m,
                                           CellState<Lattice<LAT>::D> &c)
{
    constexpr int D = Lattice<LAT>::D;
    c.drho = m.drho;
    c.rho = 1.f + m.drho;
    c.inv_rho = 1.f / c.rho;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        c.v[a] = m.J[a] * c.inv_rho;
        c.u[a] = kp.r * c.v[a];
    }
    float tr = 0.f;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) {
            // r^2 M in hi + lo: the temperature must see the same r^2 the energy sum uses
            const float R2M = fmaf(kp.R2_hi, m.M[a][b], kp.R2_lo * m.M[a][b]);
            float v = (R2M - (a == b ? m.drho : 0.f)) * c.inv_rho - c.u[a] * c.u[b];
            c.sdev[a][b] = v;
            if (a == b) tr += v;
        }
    c.th_tr = tr * (1.f / D);
    if (kp.Nf > 0.f) {
        c.th_int = (2.f * m.H / kp.Nf - m.drho) * c.inv_rho;
        c.th_eq = (D * c.th_tr + kp.Nf * c.th_int) / (D + kp.Nf);
        c.th_rel = kp.kappa * c.th_eq + (1.f - kp.kappa) * c.th_int;
    } else {
        c.th_int = 0.f;
        c.th_eq = c.th_tr;
        c.th_rel = c.th_tr;
    }
}

template <int LAT>
__device__ __forceinline__ void es_state(const KParams<LAT> &kp, const CellState<Lattice<LAT>::D> &c,
                                         EqState<Lattice<LAT>::D> &e)
{
    constexpr int D = Lattice<LAT>::D;
    e.drho = c.drho;
    e.rho = c.rho;
    e.th_rel = c.th_rel;
    const float iso = kp.a_tr * c.th_tr + kp.kappa * c.th_eq;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        e.u[a] = c.u[a];
        e.v[a] = c.v[a];
#pragma unroll
        for (int b = 0; b < D; ++b) e.A[a][b] = kp.a_sig * c.sdev[a][b] + (a == b ? iso : 0.f);
    }
}

// Maxwellian state (Lambda = T delta) of (rho, u = r v, T) given the lattice velocity v.
template <int D>
__device__ __forceinline__ void maxwell_state(float drho, const float (&v)[D], float r, float th, EqState<D> &e)
{
    e.drho = drho;
    e.rho = 1.f + drho;
    e.th_rel = th;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        e.v[a] = v[a];
        e.u[a] = r * v[a];
#pragma unroll
        for (int b = 0; b < D; ++b) e.A[a][b] = a == b ? th : 0.f;
    }
}

// Scaled equilibrium deviations at velocity I given q_I:
//   G~_I / w_I = drho + rho q,   H~_I / w_I = (N_f/2)(drho + rho th_rel + rho T_rel q)
struct EqScal {
    float drho, rho, hb, hr; // hb = (N_f/2)(drho + rho th_rel), hr = (N_f/2) rho (1 + th_rel)
};

template <int D> __device__ __forceinline__ EqScal eq_scalars(const EqState<D> &e, float halfNf)
{
    EqScal z;
    z.drho = e.drho;
    z.rho = e.rho;
    z.hb = halfNf * fmaf(e.rho, e.th_rel, e.drho);
    z.hr = halfNf * e.rho * (1.f + e.th_rel);
    return z;
}

} // namespace lbm
