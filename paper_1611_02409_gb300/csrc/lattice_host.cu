// FP64 derivation of the lattice weights and scale (host code of the CUDA library).
//
// A lattice of shells {signed permutations of a generator} x r integrates the unit
// Gaussian exactly up to degree 9 when, for every even multi-index alpha with
// |alpha| <= 8, sum_i w_i (r c_i)^alpha = prod_d (alpha_d - 1)!!  (odd moments vanish by
// symmetry).  D2Q37 has 8 shell weights and 9 such conditions, so r is fixed too
// (Sec. VI A prints r = 1.19697977): it is the root of the determinant of the augmented
// 9 x 9 system [M(r) | b], found here by regula falsi (Illinois variant).  The weights
// then solve the normal equations M^T M w = M^T b in extended precision.  The 3-D
// lattice reuses that r (its 11 conditions in 10 shell weights are consistent there);
// D2Q33 (Table D2Q33, 8 shells, 9 conditions) has its own r, found the same way.  D2Q77
// (15 shells) integrates exactly up to degree 13: its 16 conditions run to |alpha| <= 12
// and fix its r the same way.  Every condition is divided by its right-hand side (a
// positive factor: the root and the solution stay, the conditioning improves).
#include <cmath>

#include "lattice.cuh"
#include "ops.h"

namespace lbm {
namespace {

typedef long double ld;

struct Conds {
    int n;
    int e[16][3];
    ld rhs[16];
};

Conds conditions(int D, int maxdeg)
{
    Conds c{};
    for (int deg = 0; deg <= maxdeg; deg += 2)
        for (int a = deg; a >= 0; a -= 2)
            for (int b = a; b >= 0; b -= 2) {
                int z = deg - a - b;
                if (z < 0 || z > b || (z & 1)) continue;
                if (D == 2 && z != 0) continue;
                c.e[c.n][0] = a;
                c.e[c.n][1] = b;
                c.e[c.n][2] = z;
                ld v = 1;
                for (int d = 0; d < 3; ++d)
                    for (int k = c.e[c.n][d] - 1; k > 0; k -= 2) v *= k;
                c.rhs[c.n] = v;
                c.n++;
            }
    return c;
}

// row k of the shell moment matrix at scale r, divided by the condition's rhs
void shell_row(const VelTable &t, int D, int nsh, ld r, const int *e, ld rhs, ld *row)
{
    for (int s = 0; s < nsh; ++s) row[s] = 0;
    for (int i = 0; i < t.Q; ++i) {
        ld v = 1;
        for (int d = 0; d < D; ++d) v *= std::pow(r * t.c[i][d], (ld)e[d]);
        row[t.shell[i]] += v;
    }
    for (int s = 0; s < nsh; ++s) row[s] /= rhs;
}

// Gaussian elimination with partial pivoting on an n x (n+1) augmented matrix; returns
// the determinant of the left block and, if x != nullptr, the solution.
ld eliminate(int n, ld (*M)[17], ld *x)
{
    ld det = 1;
    for (int col = 0; col < n; ++col) {
        int p = col;
        for (int k = col + 1; k < n; ++k)
            if (std::fabs(M[k][col]) > std::fabs(M[p][col])) p = k;
        if (M[p][col] == 0) return 0;
        if (p != col) {
            for (int j = 0; j <= n; ++j) std::swap(M[col][j], M[p][j]);
            det = -det;
        }
        det *= M[col][col];
        for (int k = col + 1; k < n; ++k) {
            ld f = M[k][col] / M[col][col];
            for (int j = col; j <= n; ++j) M[k][j] -= f * M[col][j];
        }
    }
    if (x)
        for (int k = n - 1; k >= 0; --k) {
            ld v = M[k][n];
            for (int j = k + 1; j < n; ++j) v -= M[k][j] * x[j];
            x[k] = v / M[k][k];
        }
    return det;
}

// determinant of [M(r) | b] for a system with exactly nsh + 1 conditions
ld augmented_det(const VelTable &t, int D, int nsh, const Conds &cd, ld r)
{
    ld A[16][17];
    for (int k = 0; k < cd.n; ++k) {
        shell_row(t, D, nsh, r, cd.e[k], cd.rhs[k], A[k]);
        A[k][nsh] = 1;
    }
    return eliminate(cd.n, A, nullptr);
}

bool normal_solve(const VelTable &t, int D, int nsh, const Conds &cd, ld r, ld *ws)
{
    ld M[16][16], N[16][17];
    for (int k = 0; k < cd.n; ++k) shell_row(t, D, nsh, r, cd.e[k], cd.rhs[k], M[k]);
    for (int a = 0; a < nsh; ++a) {
        for (int b = 0; b < nsh; ++b) {
            ld v = 0;
            for (int k = 0; k < cd.n; ++k) v += M[k][a] * M[k][b];
            N[a][b] = v;
        }
        ld v = 0;
        for (int k = 0; k < cd.n; ++k) v += M[k][a];
        N[a][nsh] = v;
    }
    return eliminate(nsh, N, ws) != 0;
}

ld residual(const VelTable &t, int D, int nsh, const Conds &cd, int k, ld r, const ld *ws)
{
    ld row[16];
    shell_row(t, D, nsh, r, cd.e[k], cd.rhs[k], row);
    ld v = -1;
    for (int s = 0; s < nsh; ++s) v += row[s] * ws[s];
    return v;  // relative to the condition's rhs
}

} // namespace

int derive_lattice(int lattice, int (*c)[3], double *w, double *r_out)
{
    if (lattice != LAT_D2Q37 && lattice != LAT_D3Q103 && lattice != LAT_D2Q33 && lattice != LAT_D2Q77) return -1;
    // scale r from the 2-D system: D2Q37's (reused by D3Q103), D2Q33's own (printed as
    // 0.819381 sqrt(2) = 1.15878, Table D2Q33) or D2Q77's (0.97000849874, the only root in
    // [0.8, 1.4])
    const bool q33 = lattice == LAT_D2Q33, q77 = lattice == LAT_D2Q77;
    const VelTable t2 = build_table(q33 ? LAT_D2Q33 : q77 ? LAT_D2Q77 : LAT_D2Q37);
    const int maxdeg = q77 ? 12 : 8, nsh2 = q77 ? 15 : 8;
    const Conds c2 = conditions(2, maxdeg);
    ld ra = q33 ? 1.15L : q77 ? 0.965L : 1.18L, rb = q33 ? 1.17L : q77 ? 0.975L : 1.21L;
    ld fa = augmented_det(t2, 2, nsh2, c2, ra), fb = augmented_det(t2, 2, nsh2, c2, rb);
    if (!(fa * fb < 0)) return -1;
    int side = 0;
    for (int it = 0; it < 400 && rb - ra > 1e-18L; ++it) {
        ld rc = (ra * fb - rb * fa) / (fb - fa);
        ld fc = augmented_det(t2, 2, nsh2, c2, rc);
        if (fc == 0) { ra = rb = rc; break; }
        if ((fc < 0) == (fb < 0)) {
            rb = rc; fb = fc;
            if (side == -1) fa *= 0.5L;
            side = -1;
        } else {
            ra = rc; fa = fc;
            if (side == 1) fb *= 0.5L;
            side = 1;
        }
    }
    const ld r = 0.5L * (ra + rb);
    const int D = lattice == LAT_D3Q103 ? 3 : 2;
    const VelTable t = build_table(lattice);
    const Conds cd = conditions(D, maxdeg);
    const int nsh = q77 ? 15 : D == 2 ? 8 : 10;
    ld ws[16];
    if (!normal_solve(t, D, nsh, cd, r, ws)) return -1;
    for (int k = 0; k < cd.n; ++k)
        if (std::fabs(residual(t, D, nsh, cd, k, r, ws)) > 1e-11L) return -1;
    for (int i = 0; i < t.Q; ++i) {
        for (int d = 0; d < 3; ++d) c[i][d] = t.c[i][d];
        w[i] = (double)ws[t.shell[i]];
    }
    *r_out = (double)r;
    return t.Q;
}

} // namespace lbm
