// Kernels of the ES-BGK lattice Boltzmann step, templated on lattice and storage.
//
// Layout in HBM: two population buffers (ping-pong), each holding 2Q planes
// [set][i][z][y][x] (set 0 = g, set 1 = h), x fastest.  In wall mode each plane has
// ny + 2 gh rows: gh = 2 ghost rows beyond each wall row (rows y = 0 and y = ny-1).
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

#include "physics.cuh"

namespace lbm {

constexpr int kDiagNV = 10;      // diagnostics partial sums per block
constexpr int kDiagThreads = 256;

// x - C wrapped into [0, n); `small` grids (n < max(4, reach): one add would not reach
// [0, n)) take the general modulo path.
template <int C> LBM_HD __forceinline__ int wrap_sub(int x, int n, bool small)
{
    int v = x - C;
    if (small) return ((v % n) + n) % n;
    if constexpr (C > 0) {
        if (v < 0) v += n;
    } else if constexpr (C < 0) {
        if (v >= n) v -= n;
    }
    return v;
}

// Source column x - C of the gather: wrapped (periodic) or, with open ends, clamped to the
// domain (zero gradient: a population from beyond an end is the end cell's own).
template <int C> LBM_HD __forceinline__ int src_x(int x, int n, bool small, bool open)
{
    if (open) {
        const int v = x - C;
        return v < 0 ? 0 : (v >= n ? n - 1 : v);
    }
    return wrap_sub<C>(x, n, small);
}

// Launch parameters of the kernels of storage form ST (FP64 constants for FP64 storage).
template <int LAT, int ST> using KParamsOf = KParams<LAT, typename Storage<ST>::R>;

template <int LAT, class S>
LBM_HD __forceinline__ long long cell_index(const KParams<LAT, S> &kp, int x, int ys, int z)
{
    return ((long long)z * kp.nys + ys) * kp.nx + x;
}

// Byte offsets of the 2Q destination planes from a cell's set-0 plane-0 address: a
// per-population table (the single-domain kernels' constant-bank offsets) ...
struct TableOff {
    const long long *soff;
    __device__ __forceinline__ long long operator()(int I) const { return soff[I]; }
};
// ... or the plane stride (batched instances: per-instance planes, 32-bit offsets).
template <int ELEM> struct StrideOff {
    int plane;
    __device__ __forceinline__ long long operator()(int I) const { return (long long)(I * plane) * ELEM; }
};

// Relax population I of a cell and store it: s' = s + omega(G~/w - dg - s), same for t
// with dh (dg, dh: the reference state's shift of velocity I's shell, see shift_g/shift_h).
// `cell` is the destination cell's address in set 0 plane 0; off(I) the planes' byte offsets.
// With V = f2 (two neighbouring cells, 16-bit storage) both lanes are relaxed by packed
// FMAs and stored as one 32-bit word at the first cell's address.
// SHIFT = false (the kernels of a handle without a reference state) drops dg, dh.
template <int LAT, int ST, bool SHIFT = true, class Off, class V, class S>
__device__ __forceinline__ void relax_store(typename Storage<ST>::T *__restrict__ cell, const Off &off, int I,
                                            S om, const EqScalT<V> &z, V q, V s, V t, S dg, S dh)
{
    using T = typename Storage<ST>::T;
    constexpr int Q = Lattice<LAT>::Q;
    char *b = reinterpret_cast<char *>(cell);
    if constexpr (std::is_same<V, f2>::value) {
        static_assert(ST != ST_FP32, "paired cells use 16-bit storage");
        const f2 wg = SHIFT ? z.wdrho - f2(dg) : z.wdrho, wh = SHIFT ? z.whb - f2(dh) : z.whb;
        Storage<ST>::st2(reinterpret_cast<T *>(b + off(I)), vfma(f2(z.om1), s, vfma(f2(om), q, wg)));
        Storage<ST>::st2(reinterpret_cast<T *>(b + off(Q + I)), vfma(f2(z.om1), t, vfma(z.whr, q, wh)));
    } else if constexpr (ST == ST_FP32 || ST == ST_FP64) {
        // difference form: the non-equilibrium part G~/w - s is formed exactly
        const V Gs = SHIFT ? (z.drho + q) - dg : z.drho + q;
        const V Ht = SHIFT ? vfma(z.hr, q, z.hb) - dh : vfma(z.hr, q, z.hb);
        Storage<ST>::st(reinterpret_cast<T *>(b + off(I)), vfma(om, Gs - s, s));
        Storage<ST>::st(reinterpret_cast<T *>(b + off(Q + I)), vfma(om, Ht - t, t));
    } else {
        // (1 - omega) s + omega G~/w in two FMAs (z carries omega-scaled terms); its extra
        // FP32 rounding is far below the 16-bit storage rounding
        const float wg = SHIFT ? z.wdrho - dg : z.wdrho, wh = SHIFT ? z.whb - dh : z.whb;
        Storage<ST>::st(reinterpret_cast<T *>(b + off(I)), fmaf(z.om1, s, fmaf(om, q, wg)));
        Storage<ST>::st(reinterpret_cast<T *>(b + off(Q + I)), fmaf(z.om1, t, fmaf(z.whr, q, wh)));
    }
}

// The reference state's shift of the relaxation target for shell `sh`, in the form
// relax_store takes: omega-scaled for 16-bit storage.
template <int ST, int LAT, class S> __device__ __forceinline__ S shift_g(const KParams<LAT, S> &kp, int sh)
{
    return (ST == ST_FP16 || ST == ST_BF16) ? kp.ref_wg[sh] : kp.ref_g[sh];
}
template <int ST, int LAT, class S> __device__ __forceinline__ S shift_h(const KParams<LAT, S> &kp, int sh)
{
    return (ST == ST_FP16 || ST == ST_BF16) ? kp.ref_wh[sh] : kp.ref_h[sh];
}

// Collide one cell's streamed populations (accessor `pop`) and store them at offset o.
// REF: the handle has a reference state (rho0, T0) != (1, 1); without one the kernels
// compile without the reference's moment share and relaxation shifts.
template <int LAT, int ST, bool REF = true, class Pop, class Off = TableOff, class S = float>
__device__ __forceinline__ void collide_store(const KParams<LAT, S> &kp, const Pop &pop,
                                              typename Storage<ST>::T *__restrict__ dst, long long o,
                                              const Off &off = Off{nullptr})
{
    constexpr int D = Lattice<LAT>::D;
    constexpr int Q = Lattice<LAT>::Q;
    constexpr bool PRECISE = ST == ST_FP32;
    using V = typename Pop::V;
    RawMoments<D, V> m;
    raw_moments<LAT, PRECISE>(kp, pop, m);
    if constexpr (REF) add_reference(kp, m);
    CellState<D, V> c;
    // packed lanes (16-bit storage) divide with the fast reciprocal; one-cell lanes keep
    // IEEE division (on the 3-D two-pass kernel the fast form costs registers and spills)
    cell_state<LAT, std::is_same<V, f2>::value, PRECISE && REF>(kp, m, c);
    EqState<D, V> e;
    es_state<LAT>(kp, c, e);
    PolyCoef<D, V, Lattice<LAT>::ORDER> pc;
    poly_coeffs<PRECISE, REF>(e, kp, pc);
    EqScalT<V> z = eq_scalars<D>(e, kp.halfNf);
    z.om1 = 1.f - kp.omega;
    z.wdrho = kp.omega * z.drho;
    z.whb = kp.omega * z.hb;
    z.whr = kp.omega * z.hr;
    typename Storage<ST>::T *cell = dst + o;
    Off so = off;
    if constexpr (std::is_same<Off, TableOff>::value) so.soff = kp.soff;
    Pop rp = pop;
    rp.refresh();
    relax_store<LAT, ST, REF>(cell, so, 0, kp.omega, z, pc.k[0], rp.template sv<0>(), rp.template tv<0>(),
                              shift_g<ST>(kp, 0), shift_h<ST>(kp, 0));
    static_for<0, (Q - 1) / 2>([&](auto PP) {
        constexpr int I = 1 + 2 * decltype(PP)::value;
        constexpr int sh = Lattice<LAT>::T.shell[I];
        rp.template prefetch<decltype(PP)::value>();
        V E, O;
        poly_eval_pair<LAT, I>(pc, E, O);
        const S dg = shift_g<ST>(kp, sh), dh = shift_h<ST>(kp, sh);
        relax_store<LAT, ST, REF>(cell, so, I, kp.omega, z, E + O, rp.template sv<I>(), rp.template tv<I>(), dg,
                                  dh);
        relax_store<LAT, ST, REF>(cell, so, I + 1, kp.omega, z, E - O, rp.template sv<I + 1>(),
                                  rp.template tv<I + 1>(), dg, dh);
    });
}

// Fused pull-stream + collide (Eqs. DiscreteReductionG / DiscreteReductionH): one thread
// per cell of row y = y0 + blockIdx.y (plane z = blockIdx.z), all 2Q populations in
// registers.  Periodic in x (and z, y when !WALLS); with WALLS the rows y - c_y reach
// into the ghost rows, which the wall kernel filled after the previous step.
// Four resident 128-thread blocks per SM (<= 128 registers) for the 2-D lattice: enough
// loads in flight for FP32 and better latency hiding for the compute-bound 16-bit forms.
template <int LAT, int ST> constexpr int direct_min_blocks() { return Lattice<LAT>::D == 2 ? 4 : 1; }

template <int LAT, int ST, bool WALLS, bool REF>
__global__ void __launch_bounds__(128, direct_min_blocks<LAT, ST>()) k_stream_collide(const typename Storage<ST>::T *__restrict__ src,
                                                        typename Storage<ST>::T *__restrict__ dst,
                                                        const KParamsOf<LAT, ST> kp, int small_x, int small_y,
                                                        int small_z)
{
    constexpr int D = Lattice<LAT>::D;
    constexpr int Q = Lattice<LAT>::Q;
    using S = Storage<ST>;
    using T = typename S::T;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= kp.nx) return;
    const int y = blockIdx.y + kp.y0;
    const int z = blockIdx.z;
    const long long o = cell_index<LAT>(kp, x, y + kp.gh, z);
    // a cell at least the stencil's reach R away from every periodic seam or open end
    // gathers at fixed byte offsets; only the warps holding the first and last R cells of
    // a row diverge
    constexpr int R = Lattice<LAT>::R;
    bool interior = x >= R && x + R < kp.nx;
    if constexpr (!WALLS) interior = interior && y >= R && y + R < kp.ny;
    if constexpr (D == 3) interior = interior && z >= R && z + R < kp.nz;
    typename S::Raw rs[Q], rt[Q];
    if (interior) {
        const char *base = reinterpret_cast<const char *>(src + o);
        static_for<0, Q>([&](auto II) {
            constexpr int I = decltype(II)::value;
            rs[I] = S::raw(reinterpret_cast<const T *>(base + kp.goff[I]));
            rt[I] = S::raw(reinterpret_cast<const T *>(base + kp.goff[Q + I]));
        });
    } else {
        static_for<0, Q>([&](auto II) {
            constexpr int I = decltype(II)::value;
            constexpr int cx = cv<LAT, I, 0>(), cy = cv<LAT, I, 1>(), cz = cv<LAT, I, 2>();
            const int xs = src_x<cx>(x, kp.nx, small_x, kp.open_x);
            int ys;
            if constexpr (WALLS) ys = y - cy + kp.gh;
            else ys = wrap_sub<cy>(y, kp.ny, small_y);
            int zs = z;
            if constexpr (D == 3) zs = wrap_sub<cz>(z, kp.nz, small_z);
            const long long idx = cell_index<LAT>(kp, xs, ys, zs);
            rs[I] = S::raw(src + (long long)I * kp.plane + idx);
            rt[I] = S::raw(src + (long long)(Q + I) * kp.plane + idx);
        });
    }
    (void)small_z;
    // keep the conversions (and everything after) below the whole gather
    asm volatile("" ::: "memory");
    typename S::R s[Q], t[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        s[i] = S::cvt(rs[i]);
        t[i] = S::cvt(rt[i]);
    }
    collide_store<LAT, ST, REF>(kp, ArrayPopT<typename S::R>{s, t}, dst, o);
}

// Populations read from the source buffer where they are used (two-pass kernel): a cell's
// wrapped source columns, rows and planes for the displacements -R..R (R the stencil's
// reach) are tabulated once.
// Opposite pairs are read in chunks of CH pairs: prefetch<P>() at the first pair of a
// chunk issues the chunk's 4 CH loads (g and h of both members) into registers before any
// of them is used, so each warp keeps a chunk of loads in flight; sv<I>() / tv<I>() then
// return the buffered values (the rest population is read directly).  With DB (double
// buffering) the first prefetch issues chunks 0 and 1 and every later one the chunk after
// the next, into the other of two buffers, so the next chunk's loads are in flight while
// the current one is summed or relaxed.  refresh() makes the buffer address opaque, so
// the relaxation reads the values again (from L1 / L2) instead of keeping the moment
// pass's values live across the cell.
template <int LAT, int ST, int CH, bool DB = false, bool PK = false> struct GatherPop {
    using S = Storage<ST>;
    using V = typename S::R;
    using T = typename S::T;
    static constexpr int Q = Lattice<LAT>::Q;
    static constexpr int NP = (Q - 1) / 2;
    static constexpr int NB = DB ? 2 : 1;   // chunk buffers
    static_assert(!PK || (sizeof(typename S::Raw) == 2 && !DB), "packing keeps 16-bit values");
    // PK (16-bit storage): the moment pass packs each opposite pair's two stored values into
    // one 32-bit word that stays in registers, so the relaxation pass reads nothing again
    mutable uint32_t wg[PK ? NP : 1], wh[PK ? NP : 1];
    mutable typename S::Raw g0, h0;
    bool second = false;                    // set by refresh(): the relaxation pass
    const T *src;
    long long plane;
    static constexpr int R = Lattice<LAT>::R;
    int col[2 * R + 1], row[2 * R + 1], pln[2 * R + 1];   // element offsets within a plane
    mutable typename S::Raw bs[NB][2 * CH], bt[NB][2 * CH];
    template <int I> __device__ __forceinline__ int at() const
    {
        return pln[cv<LAT, I, 2>() + R] + row[cv<LAT, I, 1>() + R] + col[cv<LAT, I, 0>() + R];
    }
    // source of population p (set p / Q, velocity p % Q) whose velocity is I
    template <int P, int I> __device__ __forceinline__ const T *addr() const { return src + P * plane + at<I>(); }
    // the loads of chunk C (pairs [C CH, (C + 1) CH)) into buffer C % NB
    template <int C> __device__ __forceinline__ void issue() const
    {
        static_for<0, CH>([&](auto KK) {
            constexpr int k = decltype(KK)::value;
            constexpr int P = C * CH + k;
            constexpr int I = 1 + 2 * P;
            if constexpr (P < NP) {
                bs[C % NB][2 * k] = S::raw(addr<I, I>());
                bs[C % NB][2 * k + 1] = S::raw(addr<I + 1, I + 1>());
                bt[C % NB][2 * k] = S::raw(addr<Q + I, I>());
                bt[C % NB][2 * k + 1] = S::raw(addr<Q + I + 1, I + 1>());
            }
        });
    }
    template <int P> __device__ __forceinline__ void prefetch() const
    {
        if constexpr (P % CH == 0) {
            constexpr int C = P / CH;
            if constexpr (PK) {
                if (second) return;
            }
            if constexpr (!DB) {
                issue<C>();
            } else {
                if constexpr (C == 0) issue<0>();
                if constexpr ((C + 1) * CH < NP) issue<C + 1>();
            }
            asm volatile("" ::: "memory");
            if constexpr (PK) {
                static_for<0, CH>([&](auto KK) {
                    constexpr int k = decltype(KK)::value;
                    constexpr int Pk = C * CH + k;
                    if constexpr (Pk < NP) {
                        wg[Pk] = (uint32_t)bs[0][2 * k] | ((uint32_t)bs[0][2 * k + 1] << 16);
                        wh[Pk] = (uint32_t)bt[0][2 * k] | ((uint32_t)bt[0][2 * k + 1] << 16);
                    }
                });
            }
        }
    }
    // the stored value of population I of the set (g: w = wg, b = bs; h: wh, bt)
    template <int I> __device__ __forceinline__ V packed(const uint32_t (&w)[PK ? NP : 1]) const
    {
        const uint32_t word = w[(I - 1) / 2];
        return S::cvt((typename S::Raw)((I - 1) % 2 ? word >> 16 : word & 0xffffu));
    }
    template <int I> __device__ __forceinline__ V sv() const
    {
        if constexpr (PK) {
            if constexpr (I == 0) {
                if (!second) g0 = S::raw(addr<0, 0>());
                return S::cvt(g0);
            } else if (second) {
                return packed<I>(wg);
            }
        }
        if constexpr (I == 0) return S::ld(addr<0, 0>());
        else return S::cvt(bs[(((I - 1) / 2) / CH) % NB][2 * (((I - 1) / 2) % CH) + (I - 1) % 2]);
    }
    template <int I> __device__ __forceinline__ V tv() const
    {
        if constexpr (PK) {
            if constexpr (I == 0) {
                if (!second) h0 = S::raw(addr<Q, 0>());
                return S::cvt(h0);
            } else if (second) {
                return packed<I>(wh);
            }
        }
        if constexpr (I == 0) return S::ld(addr<Q, 0>());
        else return S::cvt(bt[(((I - 1) / 2) / CH) % NB][2 * (((I - 1) / 2) % CH) + (I - 1) % 2]);
    }
    __device__ __forceinline__ void refresh()
    {
        if constexpr (PK) second = true;
        else asm volatile("" : "+l"(src));
    }
};

// Pairs per prefetch chunk of the two-pass kernel, and whether the chunks are
// double-buffered: D2Q37's 18 pairs in two chunks; D3Q103's 51 in three, or with FP32
// storage in four double-buffered chunks of 13 (measured at 256^3: +2.4 % for FP32, -2 %
// for FP16, whose chunks stay single; chunks of 6 or 9 pairs, double-buffered or not,
// and double-buffered chunks on D2Q77 measured no better; the packed 16-bit form with the
// reference shifts compiled in: chunks of 9, 13 and 17 within 0.5 % of each other).
template <int LAT, int ST> constexpr bool twopass_db() { return LAT == LAT_D3Q103 && ST == ST_FP32; }
// 16-bit storage on the large lattices: the relaxation reuses the moment pass's values,
// packed two per register, instead of reading them again
template <int LAT, int ST> constexpr bool twopass_pack()
{
    return (ST == ST_FP16 || ST == ST_BF16) && LAT == LAT_D3Q103;
}
template <int LAT, int ST> constexpr int twopass_chunk()
{
    return Lattice<LAT>::D == 2 ? 9 : (twopass_db<LAT, ST>() ? 13 : 17);
}

// The fused step with the populations read twice: once streamed into the moment sums,
// once more for the relaxation.  Nothing of the cell stays in registers between the
// passes, so the kernel fits a lattice whose 2Q values would not (D3Q103, 206 values):
// more resident warps in exchange for a second, cache-served read.  Every cell takes the
// same tabulated-offset gather (no seam divergence).
// FP64 storage (double arithmetic, twice the registers per value): two blocks per SM.
template <int LAT, int ST> constexpr int twopass_min_blocks()
{
    return ST == ST_FP64 || twopass_pack<LAT, ST>() ? 2 : (Lattice<LAT>::D == 2 ? 4 : 2);
}

template <int LAT, int ST, bool WALLS, bool REF>
__global__ void __launch_bounds__(128, twopass_min_blocks<LAT, ST>()) k_stream_collide_2p(
    const typename Storage<ST>::T *__restrict__ src, typename Storage<ST>::T *__restrict__ dst,
    const KParamsOf<LAT, ST> kp, int small_x, int small_y, int small_z)
{
    constexpr int D = Lattice<LAT>::D;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= kp.nx) return;
    const int y = blockIdx.y + kp.y0;
    const int z = blockIdx.z;
    GatherPop<LAT, ST, twopass_chunk<LAT, ST>(), twopass_db<LAT, ST>(), twopass_pack<LAT, ST>()> pop;
    pop.src = src;
    pop.plane = kp.plane;
    constexpr int R = Lattice<LAT>::R;
    static_for<0, 2 * R + 1>([&](auto KK) {
        constexpr int C = decltype(KK)::value - R;
        pop.col[KK] = src_x<C>(x, kp.nx, small_x, kp.open_x);
        int ys;
        if constexpr (WALLS) ys = y - C + kp.gh;
        else ys = wrap_sub<C>(y, kp.ny, small_y);
        pop.row[KK] = ys * kp.nx;
        if constexpr (D == 3) pop.pln[KK] = wrap_sub<C>(z, kp.nz, small_z) * kp.nys * kp.nx;
        else pop.pln[KK] = 0;
    });
    collide_store<LAT, ST, REF>(kp, pop, dst, cell_index<LAT>(kp, x, y + kp.gh, z));
}

// Two neighbouring cells' stored 16-bit values, one 32-bit word per population (low
// half: the even cell).  Values are converted to FP32 pairs where they are used; refresh()
// makes the words opaque between the moment sums and the relaxation, so the converted
// pairs are formed again there instead of being held in registers across the cell.
template <int ST, int Q> struct RawPop2 {
    using V = f2;
    uint32_t *s, *t;
    template <int I> __device__ __forceinline__ f2 sv() const { return Storage<ST>::cvt2(s[I]); }
    template <int I> __device__ __forceinline__ f2 tv() const { return Storage<ST>::cvt2(t[I]); }
    template <int P> __device__ __forceinline__ void prefetch() const {}
    __device__ __forceinline__ void refresh()
    {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            asm volatile("" : "+r"(s[i]));
            asm volatile("" : "+r"(t[i]));
        }
    }
};

// Values of the degree-<=4 monomials at each velocity of a 2-D lattice, for the paired
// kernel's rolled relaxation: one loop body for every opposite pair, the velocity's
// monomial values read from the constant bank instead of compiled into 18 copies.  The
// paired kernel is bound by instruction fetch (its unrolled cell is larger than the
// instruction cache holds for three warps per scheduler at different points); the rolled
// relaxation executes more instructions (multiplications by 0 and 1, a loop) from a
// smaller footprint, +2 % (FP16) / +5 % (BF16) at 4096^2.
template <int LAT> struct MonoVals {
    float m[Lattice<LAT>::Q][Monos<2>::K];
    int shell[Lattice<LAT>::Q];   // the velocity's shell (reference-state shift)
};
template <int LAT> constexpr MonoVals<LAT> make_mono_vals()
{
    MonoVals<LAT> v{};
    for (int i = 0; i < Lattice<LAT>::Q; ++i) {
        for (int k = 0; k < Monos<2>::K; ++k)
            v.m[i][k] = (float)(ipow(Lattice<LAT>::T.c[i][0], Monos<2>::M.e[k][0]) *
                                ipow(Lattice<LAT>::T.c[i][1], Monos<2>::M.e[k][1]));
        v.shell[i] = Lattice<LAT>::T.shell[i];
    }
    return v;
}
static __constant__ MonoVals<LAT_D2Q37> c_mono_d2q37 = make_mono_vals<LAT_D2Q37>();

// The paired cells' collision (packed FP32 lanes, the non-compensated sums of 16-bit
// storage): the moment sums read the gathered words from registers (unrolled), the
// relaxation, a rolled loop over opposite pairs, from their shared-memory column (word I
// at col[I * 128]).  Per lane the arithmetic and its order are collide_store's.
template <int LAT, int ST, bool REF>
__device__ __forceinline__ void collide_store_paired(const KParams<LAT> &kp, uint32_t (&rs)[Lattice<LAT>::Q],
                                                     uint32_t (&rt)[Lattice<LAT>::Q], const uint32_t *col,
                                                     typename Storage<ST>::T *__restrict__ dst, long long o)
{
    static_assert(LAT == LAT_D2Q37, "rolled relaxation: D2Q37 monomial table");
    constexpr int D = 2;
    constexpr int Q = Lattice<LAT>::Q;
    using V = f2;
    RawMoments<D, V> m;
    raw_moments<LAT, false>(kp, RawPop2<ST, Q>{rs, rt}, m);
    if constexpr (REF) add_reference(kp, m);
    CellState<D, V> c;
    cell_state<LAT, true>(kp, m, c);
    EqState<D, V> e;
    es_state<LAT>(kp, c, e);
    PolyCoef<D, V, 4> pc;
    poly_coeffs<false, false, false>(e, kp, pc);
    EqScalT<V> z = eq_scalars<D>(e, kp.halfNf);
    z.om1 = 1.f - kp.omega;
    z.wdrho = kp.omega * z.drho;
    z.whb = kp.omega * z.hb;
    z.whr = kp.omega * z.hr;
    typename Storage<ST>::T *cell = dst + o;
    const TableOff so{kp.soff};
    relax_store<LAT, ST, REF>(cell, so, 0, kp.omega, z, pc.k[0], Storage<ST>::cvt2(col[0]),
                              Storage<ST>::cvt2(col[Q * 128]), kp.ref_wg[0], kp.ref_wh[0]);
#pragma unroll 1
    for (int I = 1; I < Q; I += 2) {
        V E = 0.f, O = 0.f;
        static_for<0, Monos<2>::K>([&](auto KK) {
            constexpr int K = decltype(KK)::value;
            const float mv = c_mono_d2q37.m[I][K];
            if constexpr (Monos<2>::M.deg[K] % 2 == 0) E = vfma(V(mv), pc.k[K], E);
            else O = vfma(V(mv), pc.k[K], O);
        });
        float dg = 0.f, dh = 0.f;
        if constexpr (REF) {
            const int sh = c_mono_d2q37.shell[I];
            dg = kp.ref_wg[sh];
            dh = kp.ref_wh[sh];
        }
        relax_store<LAT, ST, REF>(cell, so, I, kp.omega, z, E + O, Storage<ST>::cvt2(col[I * 128]),
                                  Storage<ST>::cvt2(col[(Q + I) * 128]), dg, dh);
        relax_store<LAT, ST, REF>(cell, so, I + 1, kp.omega, z, E - O, Storage<ST>::cvt2(col[(I + 1) * 128]),
                                  Storage<ST>::cvt2(col[(Q + I + 1) * 128]), dg, dh);
    }
}

// 32-bit word of the 16-bit values at element offsets e and e + 1 from p, for an odd e:
// the two aligned words around them, then a byte permute.
__device__ __forceinline__ uint32_t ld_pair_odd(const char *p)
{
    const uint32_t w0 = __ldg(reinterpret_cast<const unsigned int *>(p - 2));
    const uint32_t w1 = __ldg(reinterpret_cast<const unsigned int *>(p + 2));
    return __byte_perm(w0, w1, 0x5432);
}

// The fused step for 16-bit storage on the 2-D lattice with two neighbouring cells
// (x, x + 1; x even) per thread: each population's two source values come in one 32-bit
// load when c_x is even (the pair stays word-aligned) and in two loads and a byte permute
// when it is odd; the collision of both cells runs in packed FP32 pairs (one FFMA2 per
// pair of FMAs) and both results leave in one 32-bit store.  Needs nx even.  Per cell
// the arithmetic is the one-cell kernel's non-compensated FP32 form, evaluated per lane.
template <int LAT, int ST, bool WALLS, bool REF>
__device__ __forceinline__ void stream_collide_pair(const typename Storage<ST>::T *__restrict__ src,
                                                    typename Storage<ST>::T *__restrict__ dst, const KParams<LAT> &kp,
                                                    int small_y)
{
    static_assert(Lattice<LAT>::D == 2 && ST != ST_FP32, "paired cells: 2-D lattice, 16-bit storage");
    constexpr int Q = Lattice<LAT>::Q;
    using T = typename Storage<ST>::T;
    const int x = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (x >= kp.nx) return;
    const int y = blockIdx.y + kp.y0;
    const long long o = cell_index<LAT>(kp, x, y + kp.gh, 0);
    // a block whose every source word (x - c_x - 1 .. x + 1 - c_x + 1, |c_x| <= R) lies inside
    // the row gathers at the fixed byte offsets
    const int xb = 2 * blockIdx.x * blockDim.x;
    constexpr int R = Lattice<LAT>::R;
    bool interior = xb >= R + 1 && xb + 2 * (int)blockDim.x + R + 1 <= kp.nx;
    if constexpr (!WALLS) interior = interior && y >= R && y + R < kp.ny;
    // every load of the cell is issued before any word is combined (the byte permutes
    // and shifts wait for their loads): raw words first, then a compiler barrier
    uint32_t rs[Q], rt[Q], xs[Q], xt[Q];
    if (interior) {
        const char *base = reinterpret_cast<const char *>(src + o);
        static_for<0, Q>([&](auto II) {
            constexpr int I = decltype(II)::value;
            constexpr int cx = cv<LAT, I, 0>();
            const char *ps = base + kp.goff[I], *pt = base + kp.goff[Q + I];
            if constexpr (cx % 2 == 0) {
                rs[I] = __ldg(reinterpret_cast<const unsigned int *>(ps));
                rt[I] = __ldg(reinterpret_cast<const unsigned int *>(pt));
            } else {
                // the aligned words before and after the odd element
                rs[I] = __ldg(reinterpret_cast<const unsigned int *>(ps - 2));
                xs[I] = __ldg(reinterpret_cast<const unsigned int *>(ps + 2));
                rt[I] = __ldg(reinterpret_cast<const unsigned int *>(pt - 2));
                xt[I] = __ldg(reinterpret_cast<const unsigned int *>(pt + 2));
            }
        });
        asm volatile("" ::: "memory");
        static_for<0, Q>([&](auto II) {
            constexpr int I = decltype(II)::value;
            if constexpr (cv<LAT, I, 0>() % 2 != 0) {
                rs[I] = __byte_perm(rs[I], xs[I], 0x5432);
                rt[I] = __byte_perm(rt[I], xt[I], 0x5432);
            }
        });
    } else {
        const unsigned short *sp = reinterpret_cast<const unsigned short *>(src);
        static_for<0, Q>([&](auto II) {
            constexpr int I = decltype(II)::value;
            constexpr int cx = cv<LAT, I, 0>(), cy = cv<LAT, I, 1>();
            // nx >= 2 is even here, so x - c_x and x + 1 - c_x wrap with one correction
            // each once |c_x| <= nx; smaller rows take the modulo path
            const bool sx = kp.nx < 4;
            const int x0 = wrap_sub<cx>(x, kp.nx, sx), x1 = wrap_sub<cx>(x + 1, kp.nx, sx);
            int ys;
            if constexpr (WALLS) ys = y - cy + kp.gh;
            else ys = wrap_sub<cy>(y, kp.ny, small_y);
            const long long row = (long long)ys * kp.nx;
            const long long ps = (long long)I * kp.plane + row, pt = (long long)(Q + I) * kp.plane + row;
            rs[I] = __ldg(sp + ps + x0);
            xs[I] = __ldg(sp + ps + x1);
            rt[I] = __ldg(sp + pt + x0);
            xt[I] = __ldg(sp + pt + x1);
        });
        asm volatile("" ::: "memory");
        static_for<0, Q>([&](auto II) {
            constexpr int I = decltype(II)::value;
            rs[I] |= xs[I] << 16;
            rt[I] |= xt[I] << 16;
        });
    }
    // the words also go to this thread's shared-memory column for the rolled relaxation
    __shared__ uint32_t park[2 * Q * 128];
    uint32_t *col = park + threadIdx.x;
    static_for<0, Q>([&](auto II) {
        constexpr int I = decltype(II)::value;
        col[I * 128] = rs[I];
        col[(Q + I) * 128] = rt[I];
    });
    collide_store_paired<LAT, ST, REF>(kp, rs, rt, col, dst, o);
}

template <int LAT, int ST, bool WALLS>
__global__ void __launch_bounds__(128, 3) k_stream_collide_pair(const typename Storage<ST>::T *__restrict__ src,
                                                               typename Storage<ST>::T *__restrict__ dst,
                                                               const KParams<LAT> kp, int small_y)
{
    stream_collide_pair<LAT, ST, WALLS, false>(src, dst, kp, small_y);
}

// With a reference state: kp is a grid constant, so the rolled relaxation reads each
// shell's shift at a computed constant-bank offset.
template <int LAT, int ST, bool WALLS>
__global__ void __launch_bounds__(128, 3) k_stream_collide_pair_ref(const typename Storage<ST>::T *__restrict__ src,
                                                                   typename Storage<ST>::T *__restrict__ dst,
                                                                   const __grid_constant__ KParams<LAT> kp,
                                                                   int small_y)
{
    stream_collide_pair<LAT, ST, WALLS, true>(src, dst, kp, small_y);
}

// One cell's populations as deviations from rho = T = 1 (the stored values plus the
// reference state's shift), and back.
template <int LAT, int ST>
__device__ __forceinline__ void load_cell(const typename Storage<ST>::T *__restrict__ buf, const KParamsOf<LAT, ST> &kp,
                                          long long o, typename Storage<ST>::R *s, typename Storage<ST>::R *t)
{
    constexpr int Q = Lattice<LAT>::Q;
    static_for<0, Q>([&](auto II) {
        constexpr int i = decltype(II)::value;
        constexpr int sh = Lattice<LAT>::T.shell[i];
        s[i] = Storage<ST>::ld(buf + (long long)i * kp.plane + o) + kp.ref_g[sh];
        t[i] = Storage<ST>::ld(buf + (long long)(Q + i) * kp.plane + o) + kp.ref_h[sh];
    });
}

template <int LAT, int ST>
__device__ __forceinline__ void store_cell(typename Storage<ST>::T *__restrict__ buf, const KParamsOf<LAT, ST> &kp,
                                           long long o, const typename Storage<ST>::R *s,
                                           const typename Storage<ST>::R *t)
{
    constexpr int Q = Lattice<LAT>::Q;
    static_for<0, Q>([&](auto II) {
        constexpr int i = decltype(II)::value;
        constexpr int sh = Lattice<LAT>::T.shell[i];
        Storage<ST>::st(buf + (long long)i * kp.plane + o, s[i] - kp.ref_g[sh]);
        Storage<ST>::st(buf + (long long)(Q + i) * kp.plane + o, t[i] - kp.ref_h[sh]);
    });
}

// Scaled equilibrium populations of (rho, u = r v, T) with Lambda = T delta into s[], t[].
template <int LAT, class S>
__device__ __forceinline__ void maxwell_pops(const KParams<LAT, S> &kp, S drho, const S (&v)[Lattice<LAT>::D], S th,
                                             S *s, S *t)
{
    constexpr int D = Lattice<LAT>::D;
    constexpr int Q = Lattice<LAT>::Q;
    EqState<D, S> e;
    maxwell_state<D>(drho, v, kp.r, kp.r_lo, kp.R2_hi, th, e);
    PolyCoef<D, S, Lattice<LAT>::ORDER> pc;
    poly_coeffs<true, true>(e, kp, pc);
    const EqScalT<S> z = eq_scalars<D>(e, kp.halfNf);
    s[0] = z.drho + pc.k[0];
    t[0] = vfma(z.hr, pc.k[0], z.hb);
    static_for<0, (Q - 1) / 2>([&](auto PP) {
        constexpr int I = 1 + 2 * decltype(PP)::value;
        S E, O;
        poly_eval_pair<LAT, I>(pc, E, O);
        s[I] = z.drho + (E + O);
        t[I] = vfma(z.hr, E + O, z.hb);
        s[I + 1] = z.drho + (E - O);
        t[I + 1] = vfma(z.hr, E - O, z.hb);
    });
}

// Initial populations (equilibrium of the fields, Lambda = T delta) for every stored
// cell; ghost rows take the nearest domain row's field.  Fields are FP64 device arrays.
// Optional non-equilibrium parts (warm start): Pi (D(D+1)/2 x n, rho sigma as
// lbm_moments reports it) adds the traceless part P of Pi - rho T delta to g through the
// second Hermite term, s_i += P : (xi xi - delta) / 2, which reproduces Pi and leaves
// mass, momentum and energy unchanged; q (D x n) adds a heat flux split by heat capacity:
// the translational share (D+2)/(D+2+N_f) to g through the third Hermite term
// s_i += (xi^2 - D - 2)(q_g . xi)/(D + 2), the internal share to h, t_i += q_h . xi.
template <int LAT, int ST>
__global__ void k_init(typename Storage<ST>::T *__restrict__ dst, const KParamsOf<LAT, ST> kp,
                       const double *__restrict__ rho, const double *__restrict__ u,
                       const double *__restrict__ T, const double *__restrict__ Pi, const double *__restrict__ q)
{
    constexpr int D = Lattice<LAT>::D;
    constexpr int Q = Lattice<LAT>::Q;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= kp.nx) return;
    const int ys = blockIdx.y, z = blockIdx.z;
    int y = ys - kp.gh;
    y = y < 0 ? 0 : (y > kp.ny - 1 ? kp.ny - 1 : y);
    const long long n = (long long)kp.nx * kp.ny * kp.nz;
    const long long f = ((long long)z * kp.ny + y) * kp.nx + x;
    using R = typename Storage<ST>::R;
    R vv[D];
#pragma unroll
    for (int a = 0; a < D; ++a) vv[a] = (R)(u[a * n + f] / (double)kp.r_d);
    R s[Q], t[Q];
    maxwell_pops<LAT>(kp, (R)(rho[f] - 1.0), vv, (R)(T[f] - 1.0), s, t);
    if (Pi || q) {
        R P[D][D], qg[D], qh[D];
        const double rT = rho[f] * T[f];
        int k = 0;
        for (int a = 0; a < D; ++a)
            for (int b = a; b < D; ++b) {
                const double v = Pi ? Pi[(k++) * n + f] - (a == b ? rT : 0.0) : 0.0;
                P[a][b] = P[b][a] = (R)v;
            }
        R tr = 0.f;
        for (int a = 0; a < D; ++a) tr += P[a][a];
        for (int a = 0; a < D; ++a) P[a][a] -= tr / D;
        const double share = (D + 2.0) / (D + 2.0 + kp.Nf);
        for (int a = 0; a < D; ++a) {
            const double qa = q ? q[a * n + f] : 0.0;
            qg[a] = (R)(qa * share);
            qh[a] = (R)(qa * (1.0 - share));
        }
        static_for<0, Q>([&](auto II) {
            constexpr int I = decltype(II)::value;
            R xi[D], x2 = 0.f, qgx = 0.f, qhx = 0.f, pxx = 0.f;
            static_for<0, D>([&](auto AA) {
                constexpr int a = decltype(AA)::value;
                xi[a] = kp.r * (R)cv<LAT, I, a>();
            });
            for (int a = 0; a < D; ++a) {
                x2 += xi[a] * xi[a];
                qgx += qg[a] * xi[a];
                qhx += qh[a] * xi[a];
                for (int b = 0; b < D; ++b) pxx += P[a][b] * xi[a] * xi[b];
            }
            s[I] += R(0.5) * pxx + (x2 - (R)(D + 2)) * qgx / (R)(D + 2);
            t[I] += qhx;
        });
    }
    const long long o = cell_index<LAT>(kp, x, ys, z);
    store_cell<LAT, ST>(dst, kp, o, s, t);
}


// Wall procedure (hybrid KBC + NEEP, Sec. VI A), one thread per (column x, wall b),
// run on the post-collision buffer after the fluid rows were updated.  Boundary row at
// distance k (k = 0 wall row, 1..gh ghost rows): state u_k = u_w - k(u_1 - u_w),
// T_k = T_w - k(T_1 - T_w) from the first fluid row's (u_1, T_1); populations
// rho_w G(1, u_k, T_k delta) + the first fluid row's non-equilibrium (populations minus
// their Maxwellian).  rho_w balances exactly the mass the fluid sends into these rows
// in the next streaming against the mass the rows send back.
template <class R = float> struct WallParamsT {
    R vw[2][3];  // wall velocity in lattice units, u_w / r
    R thw[2];    // T_w - 1
};
using WallParams = WallParamsT<float>;

// Moment sums of the auxiliary kernels (walls, moments, diagnostics): compensated in FP32,
// plain in FP64.
template <class R> constexpr bool aux_precise() { return std::is_same<R, float>::value; }

// The wall procedure for one column (x, z) of wall b (0 bottom, 1 top) of buffer `buf`
// (z = 0 in 2-D; in 3-D the walls are the planes y = 0 and y = ny - 1, periodic in x, z).
template <int LAT, int ST>
__device__ __forceinline__ void wall_column(typename Storage<ST>::T *__restrict__ buf, const KParamsOf<LAT, ST> &kp,
                                            const WallParamsT<typename Storage<ST>::R> &wp, int x, int b, int z = 0)
{
    constexpr int D = Lattice<LAT>::D;
    constexpr int Q = Lattice<LAT>::Q;
    using R = typename Storage<ST>::R;
    static_assert(Lattice<LAT>::R <= 3, "two ghost rows beyond each wall row cover a reach of 3");
    const int n = b == 0 ? 1 : -1;
    const int yw = b == 0 ? 0 : kp.ny - 1;
    const int small_x = kp.nx < 4, small_z = kp.nz < 4;
    R s1[Q], t1[Q];
    load_cell<LAT, ST>(buf, kp, cell_index<LAT>(kp, x, yw + n + kp.gh, z), s1, t1);
    RawMoments<D, R> m;
    raw_moments<LAT, aux_precise<R>()>(kp, ArrayPopT<R>{s1, t1}, m);
    CellState<D, R> c;
    cell_state<LAT, false, aux_precise<R>()>(kp, m, c);
    R ms[Q], mt[Q];
    maxwell_pops<LAT>(kp, c.drho, c.v, c.th_eq, ms, mt);
#pragma unroll
    for (int i = 0; i < Q; ++i) {  // non-equilibrium of the first fluid row
        s1[i] -= ms[i];
        t1[i] -= mt[i];
    }
    R uk[3][D], thk[3];   // lattice-unit velocities of the boundary rows
    for (int k = 0; k <= 2; ++k) {
#pragma unroll
        for (int a = 0; a < D; ++a) uk[k][a] = wp.vw[b][a] - k * (c.v[a] - wp.vw[b][a]);
        thk[k] = wp.thw[b] - k * (c.th_eq - wp.thw[b]);
    }
    // unit-density equilibria of the boundary rows (deviation / w): drho = 0
    R gk[3][Q], hk[3][Q];
    for (int k = 0; k <= 2; ++k) maxwell_pops<LAT>(kp, R(0), uk[k], thk[k], gk[k], hk[k]);
    // leaving - B - A, all in deviation form: the w parts of "leaving" and "A" cancel.
    R Ld = 0.f, Bd = 0.f, Ad = 0.f, W = 0.f;
    static_for<0, Q>([&](auto II) {
        constexpr int I = decltype(II)::value;
        constexpr int cx = cv<LAT, I, 0>(), cy = cv<LAT, I, 1>(), cz = cv<LAT, I, 2>();
        constexpr int shI = Lattice<LAT>::T.shell[I];
        if constexpr (cy != 0) {
            const int cn = cy * n;
            const R w = kp.w[I];
            if (cn < 0) {
                const int xs = wrap_sub<cx>(x, kp.nx, small_x);
                const int zs = D == 3 ? wrap_sub<cz>(z, kp.nz, small_z) : 0;
                for (int sdist = 1; sdist <= -cn; ++sdist)
                    Ld = vfma(w, Storage<ST>::ld(buf + (long long)I * kp.plane
                                                 + cell_index<LAT>(kp, xs, yw + n * sdist + kp.gh, zs))
                                     + kp.ref_g[shI], Ld);
            } else {
                W = vfma((R)cn, w, W);
                Bd = vfma((R)cn * w, s1[I], Bd);
                for (int k = 0; k < cn; ++k) Ad = vfma(w, gk[k][I], Ad);
            }
        }
    });
    const R drw = (Ld - Bd - Ad) / (W + Ad);   // rho_w - 1
    const R rw = 1.f + drw;
    for (int k = 0; k <= 2; ++k) {
        const long long o = cell_index<LAT>(kp, x, yw - n * k + kp.gh, z);
        // G(rho_w, u_k, T_k)/w - 1 = drw + rw * gk;   (N_f/2)(rho_w T_k G/w - 1) = drw' + rw * hk
        const R hb = kp.halfNf * drw;
        R sk[Q], tk[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            sk[i] = vfma(rw, gk[k][i], drw) + s1[i];
            tk[i] = vfma(rw, hk[k][i], hb) + t1[i];
        }
        store_cell<LAT, ST>(buf, kp, o, sk, tk);
    }
}

template <int LAT, int ST>
__global__ void k_walls(typename Storage<ST>::T *__restrict__ buf, const KParamsOf<LAT, ST> kp,
                        const WallParamsT<typename Storage<ST>::R> wp)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= kp.nx) return;
    wall_column<LAT, ST>(buf, kp, wp, x, blockIdx.y, blockIdx.z);
}

// Macroscopic fields of the stored populations (FP64 out, any pointer may be null).
template <int LAT, int ST>
__global__ void k_moments(const typename Storage<ST>::T *__restrict__ buf, const KParamsOf<LAT, ST> kp,
                          double *rho, double *u, double *T, double *Pi, double *q)
{
    constexpr int D = Lattice<LAT>::D;
    constexpr int Q = Lattice<LAT>::Q;
    using R = typename Storage<ST>::R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= kp.nx) return;
    const int y = blockIdx.y, z = blockIdx.z;
    R s[Q], t[Q];
    load_cell<LAT, ST>(buf, kp, cell_index<LAT>(kp, x, y + kp.gh, z), s, t);
    RawMoments<D, R> m;
    raw_moments<LAT, aux_precise<R>()>(kp, ArrayPopT<R>{s, t}, m);
    CellState<D, R> c;
    cell_state<LAT, false, aux_precise<R>()>(kp, m, c);
    const long long n = (long long)kp.nx * kp.ny * kp.nz;
    const long long f = ((long long)z * kp.ny + y) * kp.nx + x;
    if (rho) rho[f] = 1.0 + (double)c.drho;
    if (u)
        for (int a = 0; a < D; ++a) u[a * n + f] = c.u[a];
    if (T) T[f] = 1.0 + (double)c.th_eq;
    if (Pi) {
        int k = 0;
        for (int a = 0; a < D; ++a)
            for (int bb = a; bb < D; ++bb)
                Pi[(k++) * n + f] = (a == bb ? (double)c.rho : 0.0) + (double)c.rsdev[a][bb];
    }
    if (q) {
        // q_a = sum g |v|^2 v_a / 2 + sum h v_a, v = xi - u; the rest-state (w) part is
        // -u_a (D + 2 + u^2 + N_f)/2 in closed form (degree-3 moments of the lattice).
        R u2 = 0.f;
        for (int a = 0; a < D; ++a) u2 += c.u[a] * c.u[a];
        R qa[D];
        for (int a = 0; a < D; ++a) qa[a] = R(-0.5) * c.u[a] * (D + 2 + u2 + kp.Nf);
        static_for<0, Q>([&](auto II) {
            constexpr int I = decltype(II)::value;
            const R w = kp.w[I];
            R v[D], v2 = 0.f;
            static_for<0, D>([&](auto AA) {
                constexpr int a = decltype(AA)::value;
                v[a] = kp.r * (R)cv<LAT, I, a>() - c.u[a];
                v2 += v[a] * v[a];
            });
            const R gd = w * s[I], hd = w * t[I];
            for (int a = 0; a < D; ++a) qa[a] += (R(0.5) * v2 * gd + hd) * v[a];
        });
        for (int a = 0; a < D; ++a) q[a * n + f] = qa[a];
    }
}

template <typename Tv> __device__ __forceinline__ Tv warp_sum(Tv v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sums of kDiagNV doubles, written by thread 0 to out[0..kDiagNV).
__device__ __forceinline__ void block_sums(double (&acc)[kDiagNV], double *out)
{
    __shared__ double sh[kDiagThreads / 32][kDiagNV];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v < kDiagNV; ++v) {
        double x = warp_sum(acc[v]);
        if (lane == 0) sh[wid][v] = x;
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int v = 0; v < kDiagNV; ++v) {
            double x = lane < kDiagThreads / 32 ? sh[lane][v] : 0.0;
            x = warp_sum(x);
            if (lane == 0) out[v] = x;
        }
    }
}

// FP64 diagnostics, stage 1: a fixed grid strides over the domain cells, each block
// writes kDiagNV partial sums: {sum drho, sum rho u (3), sum (rho E - rho E_rest),
// sum du_x^2, sum u_x^2, sum dT^2, sum T^2, bad cells}.  Snapshots u_x, T - 1 for the
// next call's residual.
template <int LAT, int ST>
__global__ void __launch_bounds__(kDiagThreads) k_diag(const typename Storage<ST>::T *__restrict__ buf,
                                                        const KParamsOf<LAT, ST> kp, typename Storage<ST>::R *snap,
                                                        int have_snap, double *partials)
{
    constexpr int D = Lattice<LAT>::D;
    constexpr int Q = Lattice<LAT>::Q;
    using R = typename Storage<ST>::R;
    double acc[kDiagNV];
#pragma unroll
    for (int v = 0; v < kDiagNV; ++v) acc[v] = 0.0;
    const long long n = (long long)kp.nx * kp.ny * kp.nz;
    for (long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x; f < n;
         f += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(f % kp.nx);
        const long long yz = f / kp.nx;
        const int y = (int)(yz % kp.ny), z = (int)(yz / kp.ny);
        R s[Q], t[Q];
        load_cell<LAT, ST>(buf, kp, cell_index<LAT>(kp, x, y + kp.gh, z), s, t);
        RawMoments<D, R> m;
        raw_moments<LAT, aux_precise<R>()>(kp, ArrayPopT<R>{s, t}, m);
        CellState<D, R> c;
        cell_state<LAT, false, aux_precise<R>()>(kp, m, c);
        acc[0] += (double)m.drho;
        for (int a = 0; a < D; ++a) acc[1 + a] += (double)kp.r * (double)m.J[a];
        R trM = 0.f;
        for (int a = 0; a < D; ++a) trM += m.M[a][a];
        acc[4] += 0.5 * (double)kp.r * (double)kp.r * (double)trM + (double)m.H;
        const R ux = c.u[0], th = c.th_eq;
        bool ok = isfinite(c.rho) && isfinite(th) && c.rho > 0.f && 1.f + th > 0.f;
        for (int a = 0; a < D; ++a) ok = ok && isfinite(c.u[a]);
        acc[9] += ok ? 0.0 : 1.0;
        acc[6] += (double)ux * ux;
        acc[8] += (1.0 + th) * (1.0 + th);
        if (have_snap) {
            const double du = (double)ux - snap[f], dT = (double)th - snap[n + f];
            acc[5] += du * du;
            acc[7] += dT * dT;
        }
        snap[f] = ux;
        snap[n + f] = th;
    }
    block_sums(acc, partials + (long long)blockIdx.x * kDiagNV);
}

// Stage 2: one block sums the partials in a fixed order (deterministic).
__global__ void __launch_bounds__(kDiagThreads) k_diag_final(const double *__restrict__ partials, int nblk,
                                                              double *out);

// Domain populations to / from absolute FP64 [i][z][y][x].
template <int LAT, int ST>
__global__ void k_get_pops(const typename Storage<ST>::T *__restrict__ buf, const KParamsOf<LAT, ST> kp, double *g,
                           double *h)
{
    constexpr int Q = Lattice<LAT>::Q;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= kp.nx) return;
    const int y = blockIdx.y, z = blockIdx.z;
    const long long n = (long long)kp.nx * kp.ny * kp.nz;
    const long long f = ((long long)z * kp.ny + y) * kp.nx + x;
    const long long o = cell_index<LAT>(kp, x, y + kp.gh, z);
    static_for<0, Q>([&](auto II) {
        constexpr int i = decltype(II)::value;
        constexpr int sh = Lattice<LAT>::T.shell[i];
        const double w = kp.w[i];
        // the reference shift added in FP64
        if (g) g[i * n + f] = w * (1.0 + (double)kp.ref_g[sh] + (double)Storage<ST>::ld(buf + (long long)i * kp.plane + o));
        if (h)
            h[i * n + f] = w * ((double)kp.halfNf + (double)kp.ref_h[sh]
                                + (double)Storage<ST>::ld(buf + (long long)(Q + i) * kp.plane + o));
    });
}

template <int LAT, int ST>
__global__ void k_set_pops(typename Storage<ST>::T *__restrict__ buf, const KParamsOf<LAT, ST> kp, const double *g,
                           const double *h)
{
    constexpr int Q = Lattice<LAT>::Q;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= kp.nx) return;
    const int y = blockIdx.y, z = blockIdx.z;
    const long long n = (long long)kp.nx * kp.ny * kp.nz;
    const long long f = ((long long)z * kp.ny + y) * kp.nx + x;
    const long long o = cell_index<LAT>(kp, x, y + kp.gh, z);
    using R = typename Storage<ST>::R;
    static_for<0, Q>([&](auto II) {
        constexpr int i = decltype(II)::value;
        constexpr int sh = Lattice<LAT>::T.shell[i];
        const double w = kp.w[i];
        // the reference shift subtracted in FP64, before the rounding to the storage form
        Storage<ST>::st(buf + (long long)i * kp.plane + o, (R)(g[i * n + f] / w - 1.0 - (double)kp.ref_g[sh]));
        Storage<ST>::st(buf + (long long)(Q + i) * kp.plane + o,
                        (R)(h[i * n + f] / w - (double)kp.halfNf - (double)kp.ref_h[sh]));
    });
}

} // namespace lbm
