// Compile-time lattice tables for the CUDA path.
//
// D2Q37: the velocity shells of Table D2Q37 (Sec. VI A): (0,0), (1,0), (1,1), (2,0),
// (2,1), (3,0), (3,1), (3,3) and their signed permutations, xi_i = r c_i.
// D3Q103: a degree-9 3-D lattice at the same scale (the paper gives none): shells
// (0,0,0), (1,0,0), (1,1,1), (2,0,0), (2,1,0), (2,2,0), (2,2,2), (3,0,0), (3,1,1), (3,3,3).
// D2Q33: Shim's lattice of Table D2Q33 (Sec. VI B, the shock tube): shells (0,0), (1,0),
// (1,1), (2,0), (2,2), (3,0), (2,1), (4,4), at its own scale; reach 4.
// D2Q77: a degree-13 lattice for the sixth-order (Burnett) expansion of Sec. IV, which the
// paper names but gives no lattice for: shells (0,0), (1,0), (1,1), (2,0), (2,1), (2,2),
// (3,0), (3,1), (3,2), (3,3), (4,0), (4,1), (4,4), (5,0), (5,3) at its own scale; reach 5.
//
// The order is the library's own: index 0 is the rest velocity, then opposite pairs
// (2k+1, 2k+2) with c_{2k+2} = -c_{2k+1}, so a kernel evaluates the even and odd parts
// of the equilibrium polynomial once per pair.  The shell weights are not compile-time
// constants: the host derives them in FP64 (lattice_host.cpp) and uploads them.
#pragma once
#include <type_traits>
#include <utility>

#define LBM_HD __host__ __device__

namespace lbm {

enum : int { LAT_D2Q37 = 1, LAT_D3Q103 = 2, LAT_D2Q33 = 3, LAT_D2Q77 = 4 };

template <int LAT> struct LatticeDims;
template <> struct LatticeDims<LAT_D2Q37> { static constexpr int D = 2, Q = 37, NSHELL = 8; };
template <> struct LatticeDims<LAT_D3Q103> { static constexpr int D = 3, Q = 103, NSHELL = 10; };
template <> struct LatticeDims<LAT_D2Q33> { static constexpr int D = 2, Q = 33, NSHELL = 8; };
template <> struct LatticeDims<LAT_D2Q77> { static constexpr int D = 2, Q = 77, NSHELL = 15; };

// Order N of the equilibrium's Hermite expansion: 4 (Eq. GExpansion) on the degree-9
// lattices, 6 (the Burnett order, Sec. IV) on the degree-13 D2Q77.
template <int LAT> struct LatticeOrder { static constexpr int N = 4; };
template <> struct LatticeOrder<LAT_D2Q77> { static constexpr int N = 6; };

struct VelTable {
    int c[128][3];
    int shell[128];
    int Q;
};

// first nonzero component positive: one representative of each opposite pair
LBM_HD constexpr bool positive_rep(int x, int y, int z)
{
    return x > 0 || (x == 0 && (y > 0 || (y == 0 && z > 0)));
}

LBM_HD constexpr VelTable build_table(int lat)
{
    const int kShells2[8][3] = {{0, 0, 0}, {1, 0, 0}, {1, 1, 0}, {2, 0, 0},
                                {2, 1, 0}, {3, 0, 0}, {3, 1, 0}, {3, 3, 0}};
    const int kShells3[10][3] = {{0, 0, 0}, {1, 0, 0}, {1, 1, 1}, {2, 0, 0}, {2, 1, 0},
                                 {2, 2, 0}, {2, 2, 2}, {3, 0, 0}, {3, 1, 1}, {3, 3, 3}};
    const int kShells33[8][3] = {{0, 0, 0}, {1, 0, 0}, {1, 1, 0}, {2, 0, 0},
                                 {2, 2, 0}, {3, 0, 0}, {2, 1, 0}, {4, 4, 0}};
    const int kShells77[15][3] = {{0, 0, 0}, {1, 0, 0}, {1, 1, 0}, {2, 0, 0}, {2, 1, 0},
                                  {2, 2, 0}, {3, 0, 0}, {3, 1, 0}, {3, 2, 0}, {3, 3, 0},
                                  {4, 0, 0}, {4, 1, 0}, {4, 4, 0}, {5, 0, 0}, {5, 3, 0}};
    const int D = lat == LAT_D3Q103 ? 3 : 2;
    VelTable t{};
    t.Q = 1;
    t.c[0][0] = t.c[0][1] = t.c[0][2] = 0;
    t.shell[0] = 0;
    const int nsh = lat == LAT_D2Q77 ? 15 : (D == 2 ? 8 : 10);
    const int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    for (int s = 1; s < nsh; ++s) {
        int gen[3] = {0, 0, 0};
        for (int d = 0; d < 3; ++d)
            gen[d] = lat == LAT_D2Q33   ? kShells33[s][d]
                     : lat == LAT_D2Q77 ? kShells77[s][d]
                                        : (D == 2 ? kShells2[s][d] : kShells3[s][d]);
        const int np = D == 2 ? 2 : 6;
        for (int p = 0; p < np; ++p)
            for (int m = 0; m < (1 << D); ++m) {
                int v[3] = {0, 0, 0};
                for (int d = 0; d < D; ++d) {
                    int src = D == 2 ? (p == 0 ? d : 1 - d) : perms[p][d];
                    v[d] = gen[src] * (((m >> d) & 1) ? -1 : 1);
                }
                if (!positive_rep(v[0], v[1], v[2])) continue;
                bool dup = false;
                for (int q = 1; q < t.Q; ++q)
                    if (t.c[q][0] == v[0] && t.c[q][1] == v[1] && t.c[q][2] == v[2]) dup = true;
                if (dup) continue;
                for (int d = 0; d < 3; ++d) {
                    t.c[t.Q][d] = v[d];
                    t.c[t.Q + 1][d] = -v[d];
                }
                t.shell[t.Q] = t.shell[t.Q + 1] = s;
                t.Q += 2;
            }
    }
    return t;
}

LBM_HD constexpr int max_reach(const VelTable &t)
{
    int r = 0;
    for (int q = 0; q < t.Q; ++q)
        for (int d = 0; d < 3; ++d) r = t.c[q][d] > r ? t.c[q][d] : r;
    return r;
}

template <int LAT> struct Lattice {
    static constexpr int D = LatticeDims<LAT>::D;
    static constexpr int Q = LatticeDims<LAT>::Q;
    static constexpr int NSHELL = LatticeDims<LAT>::NSHELL;
    static constexpr int ORDER = LatticeOrder<LAT>::N;
    static constexpr VelTable T = build_table(LAT);
    static constexpr int R = max_reach(T);   // largest |c_i| component: the stencil's reach
    static_assert(T.Q == Q, "velocity count");
};
template <int LAT> constexpr VelTable Lattice<LAT>::T;

template <int LAT, int I, int DIM> LBM_HD constexpr int cv() { return Lattice<LAT>::T.c[I][DIM]; }

// Monomials c^alpha of total degree <= N in D variables, ordered by degree (and, within a
// degree, by falling exponent of c_x): the tables for N = 4 and N = 6 share their first
// entries.  Sized for D = 3, N = 4 (35) and D = 2, N = 6 (28).
struct MonoTable {
    int e[35][3];
    int deg[35];
    int K;
};

LBM_HD constexpr MonoTable build_monos(int D, int N)
{
    MonoTable m{};
    m.K = 0;
    for (int n = 0; n <= N; ++n)
        for (int a = n; a >= 0; --a)
            for (int b = n - a; b >= 0; --b) {
                int c = n - a - b;
                if (D == 2 && c != 0) continue;
                m.e[m.K][0] = a;
                m.e[m.K][1] = b;
                m.e[m.K][2] = c;
                m.deg[m.K] = n;
                m.K++;
            }
    return m;
}

template <int D, int N = 4> struct Monos {
    static_assert((D == 2 && N <= 6) || N <= 4, "monomial table size");
    static constexpr MonoTable M = build_monos(D, N);
    static constexpr int K = M.K;
};
template <int D, int N> constexpr MonoTable Monos<D, N>::M;

// Extents below this take the modulo wrap of x - c: one add or subtract reaches [0, n)
// only for n >= |c|, and |c| <= R.
template <int LAT> LBM_HD constexpr int wrap_threshold() { return Lattice<LAT>::R > 4 ? Lattice<LAT>::R : 4; }

// index of the 2-D monomial c_x^i c_y^j in the table
LBM_HD constexpr int mono_k2(int i, int j) { return (i + j) * (i + j + 1) / 2 + j; }

LBM_HD constexpr int ipow(int b, int e)
{
    int v = 1;
    for (int k = 0; k < e; ++k) v *= b;
    return v;
}

// value of monomial k at integer velocity I
template <int LAT, int I, int K> LBM_HD constexpr int mono_at()
{
    constexpr int D = Lattice<LAT>::D;
    using M = Monos<D, Lattice<LAT>::ORDER>;
    int v = 1;
    for (int d = 0; d < D; ++d) v *= ipow(Lattice<LAT>::T.c[I][d], M::M.e[K][d]);
    return v;
}

// d-th index (0-based, nondecreasing) of the index tuple of monomial K
template <int D, int K> LBM_HD constexpr int mono_index(int pos)
{
    int acc = 0;
    for (int d = 0; d < D; ++d) {
        acc += Monos<D>::M.e[K][d];
        if (pos < acc) return d;
    }
    return D - 1;
}

// 1 / alpha! for monomial K
template <int D, int K> LBM_HD constexpr double inv_alpha_factorial()
{
    double f = 1.0;
    for (int d = 0; d < D; ++d)
        for (int k = 2; k <= Monos<D>::M.e[K][d]; ++k) f *= k;
    return 1.0 / f;
}

// Compile-time loop: f(std::integral_constant<int, I>) for I = B .. E-1.
template <int B, int E, typename F> LBM_HD __forceinline__ void static_for(F &&f)
{
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        static_for<B + 1, E>(f);
    }
}

} // namespace lbm
