/*
 * FP64 CPU oracle for the polyatomic ES-BGK lattice Boltzmann scheme of
 * Hu, Zhang, Du, Jin, Kong (arXiv 1611.02409).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA path is checked against.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code, header,
 * table or generator with the CUDA library: the lattice weights, the Hermite
 * machinery, the parameter mapping and the boundary procedure are all written
 * out again here, in the paper's notation and order.
 *
 * Everything is double precision, populations are stored absolute (no shift),
 * cell-major ([cell][i]), and every step is written as the paper states it:
 *
 *   - discrete moments                      Sec. V, moment sums after Eq. DisReductionH
 *   - temperatures / corrected tensor Lambda Sec. II (T_rel), Sec. V (dimensionless Lambda)
 *   - Hermite polynomials H^(n)             Sec. IV, Grad's identities and the H^(0..6) list
 *   - Hermite coefficients a^(n)            Sec. IV, Eq. fESCoe (general term formula)
 *   - truncated Gaussian G^(4)              Sec. IV, Eq. GExpansion; discrete G_i of Sec. V
 *     (G^(6), the Burnett order of Sec. IV, on the degree-13 D2Q77)
 *   - stream + collide                      Sec. V, Eq. DiscreteReductionG / DiscreteReductionH
 *   - lattices                              Sec. VI, Table D2Q37 (weights re-solved in FP64)
 *   - walls (hybrid KBC + NEEP)             Sec. VI A (prose only; reading below)
 *
 * Readings of places where the paper is silent, garbled or inconsistent:
 *   R1  the energy populations relax toward (N_f/2) T_rel G_i (Eq. ReductionH); the
 *       discrete equations print T_eq / T, which conserves energy only for kappa = 1.
 *   R2  rho e_int = sum_i h_i (the printed 1/2 contradicts the definition of h).
 *   R3  parameter mapping: mode SHIFTED (default) sets tau_s = tau_f,
 *       tau_q = (tau_f - 1/2)/Pr + 1/2, omega = 1/tau_q, and the Gaussian's nu from
 *       1 - nu + kappa nu = tau_q / tau_s, so that the lattice transport coefficients
 *       carry the set Pr; mode LITERAL uses omega = Pr/tau_f and 1 - nu + kappa nu = 1/Pr.
 *   R4  D3Q103 (shells 000,100,111,200,210,220,222,300,311,333, same scale r) stands in
 *       for the 3-D lattice the paper does not give.
 *   R5  walls: rows y=0 and y=Ny-1 are wall nodes, two ghost rows lie beyond each;
 *       wall density from zero net mass exchange with the fluid (the kinetic boundary
 *       condition's flux balance, taken over the populations that cross in one step),
 *       equilibrium part G(rho_w, u, T delta) with u, T extrapolated linearly from the
 *       wall values through the first fluid row, non-equilibrium part copied from the
 *       first fluid row (populations minus their own Maxwellian).  In 3-D (D3Q103)
 *       the same per wall column (x, z), periodic in x and z.
 *   R6  initial populations are the equilibrium of the given fields with Lambda = T delta;
 *       with walls, the wall procedure (R5) then rebuilds the wall and ghost rows from the
 *       first fluid rows, as after every step.
 *   R16 the shock tube's open ends (Sec. VI B) are zero-gradient: a population that would
 *       stream in from outside the x range is the boundary cell's own of that velocity.
 *   R19 D2Q77 (shells 00,10,11,20,21,22,30,31,32,33,40,41,44,50,53; scale r the root of
 *       its augmented degree-13 moment system) stands in for the degree-13 lattice that
 *       the sixth-order expansion needs and the paper does not give; on it the
 *       equilibrium is expanded to order 6.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdio.h>

#define ORC_MAXQ 128
#define ORC_MAXN 8
#define ORC_MAXT 6561 /* 3^8: largest D^n tensor held */

enum { ORC_D2Q37 = 1, ORC_D3Q103 = 2, ORC_D2Q33 = 3, ORC_D2Q77 = 4 };
enum { ORC_PR_SHIFTED = 0, ORC_PR_LITERAL = 1 };

/* ------------------------------------------------------------------------- */
/* Small dense linear algebra (used only to re-solve the lattice weights).    */
/* ------------------------------------------------------------------------- */

/* Determinant of an n x n row-major matrix by Gaussian elimination with
 * partial pivoting. */
static double orc_det(int n, const double *Ain)
{
    double A[16 * 16];
    memcpy(A, Ain, sizeof(double) * n * n);
    double det = 1.0;
    for (int k = 0; k < n; ++k) {
        int p = k;
        for (int i = k + 1; i < n; ++i)
            if (fabs(A[i * n + k]) > fabs(A[p * n + k])) p = i;
        if (A[p * n + k] == 0.0) return 0.0;
        if (p != k) {
            for (int j = 0; j < n; ++j) {
                double t = A[k * n + j]; A[k * n + j] = A[p * n + j]; A[p * n + j] = t;
            }
            det = -det;
        }
        det *= A[k * n + k];
        for (int i = k + 1; i < n; ++i) {
            double f = A[i * n + k] / A[k * n + k];
            for (int j = k; j < n; ++j) A[i * n + j] -= f * A[k * n + j];
        }
    }
    return det;
}

/* Least squares min ||A x - b|| for an m x n (m >= n) row-major A by Householder QR. */
static void orc_lstsq(int m, int n, const double *Ain, const double *bin, double *x)
{
    double A[16 * 16], b[16];
    memcpy(A, Ain, sizeof(double) * m * n);
    memcpy(b, bin, sizeof(double) * m);
    for (int k = 0; k < n; ++k) {
        double nrm = 0.0;
        for (int i = k; i < m; ++i) nrm += A[i * n + k] * A[i * n + k];
        nrm = sqrt(nrm);
        double alpha = A[k * n + k] > 0 ? -nrm : nrm;
        double v[16];
        for (int i = 0; i < m; ++i) v[i] = 0.0;
        for (int i = k; i < m; ++i) v[i] = A[i * n + k];
        v[k] -= alpha;
        double vv = 0.0;
        for (int i = k; i < m; ++i) vv += v[i] * v[i];
        if (vv == 0.0) continue;
        for (int j = k; j < n; ++j) {
            double s = 0.0;
            for (int i = k; i < m; ++i) s += v[i] * A[i * n + j];
            s = 2.0 * s / vv;
            for (int i = k; i < m; ++i) A[i * n + j] -= s * v[i];
        }
        double s = 0.0;
        for (int i = k; i < m; ++i) s += v[i] * b[i];
        s = 2.0 * s / vv;
        for (int i = k; i < m; ++i) b[i] -= s * v[i];
    }
    for (int k = n - 1; k >= 0; --k) {
        double s = b[k];
        for (int j = k + 1; j < n; ++j) s -= A[k * n + j] * x[j];
        x[k] = s / A[k * n + k];
    }
}

/* ------------------------------------------------------------------------- */
/* Lattices (Sec. VI, Table D2Q37; 3-D lattice per reading R4).               */
/* ------------------------------------------------------------------------- */

typedef struct {
    int D, Q, nshell;
    double r;
    int c[ORC_MAXQ][3];   /* integer velocity, xi_i = r c_i */
    int shell[ORC_MAXQ];
    double w[ORC_MAXQ];
} orc_lattice;

/* Generators of the velocity shells: every signed permutation of these. */
static const int ORC_SHELLS_2D[8][3] = {
    {0, 0, 0}, {1, 0, 0}, {1, 1, 0}, {2, 0, 0}, {2, 1, 0}, {3, 0, 0}, {3, 1, 0}, {3, 3, 0}};
/* Table D2Q33 (Sec. VI B, Shim's lattice): (0,0), (1,0), (1,1), (2,0), (2,2), (3,0), (2,1),
 * (4,4); its scale r is printed as 0.819381 sqrt(2). */
static const int ORC_SHELLS_2D33[8][3] = {
    {0, 0, 0}, {1, 0, 0}, {1, 1, 0}, {2, 0, 0}, {2, 2, 0}, {3, 0, 0}, {2, 1, 0}, {4, 4, 0}};
/* D2Q77 (reading R19): the paper prints no lattice for its sixth-order (Burnett) expansion;
 * these 15 shells carry a positive-weight quadrature of degree 13 (even moments to 12). */
static const int ORC_SHELLS_2D77[15][3] = {
    {0, 0, 0}, {1, 0, 0}, {1, 1, 0}, {2, 0, 0}, {2, 1, 0}, {2, 2, 0}, {3, 0, 0}, {3, 1, 0},
    {3, 2, 0}, {3, 3, 0}, {4, 0, 0}, {4, 1, 0}, {4, 4, 0}, {5, 0, 0}, {5, 3, 0}};
static const int ORC_SHELLS_3D[10][3] = {
    {0, 0, 0}, {1, 0, 0}, {1, 1, 1}, {2, 0, 0}, {2, 1, 0}, {2, 2, 0}, {2, 2, 2}, {3, 0, 0}, {3, 1, 1}, {3, 3, 3}};

static int orc_add_shell(orc_lattice *L, const int *gen, int shell_id)
{
    static const int perm3[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    static const int perm2[2][3] = {{0, 1, 2}, {1, 0, 2}};
    int D = L->D, np = D == 3 ? 6 : 2;
    for (int p = 0; p < np; ++p)
        for (int s = 0; s < (1 << D); ++s) {
            int v[3] = {0, 0, 0};
            for (int d = 0; d < D; ++d) {
                int src = D == 3 ? perm3[p][d] : perm2[p][d];
                v[d] = gen[src] * ((s >> d) & 1 ? -1 : 1);
            }
            int dup = 0;
            for (int q = 0; q < L->Q; ++q)
                if (L->c[q][0] == v[0] && L->c[q][1] == v[1] && L->c[q][2] == v[2]) dup = 1;
            if (!dup) {
                if (L->Q >= ORC_MAXQ) return -1;
                L->c[L->Q][0] = v[0]; L->c[L->Q][1] = v[1]; L->c[L->Q][2] = v[2];
                L->shell[L->Q] = shell_id;
                L->Q++;
            }
        }
    return 0;
}

/* Even multi-indices (a_1 >= ... >= a_D, sum <= maxdeg) and (prod_d (a_d - 1)!!): the
 * moments E[xi^a] of the unit Gaussian that a quadrature of degree maxdeg + 1 must
 * reproduce; odd moments vanish by the lattice's symmetry. */
static int orc_moment_conditions(int D, int maxdeg, int (*a)[3], double *rhs)
{
    int m = 0;
    for (int a0 = 0; a0 <= maxdeg; a0 += 2)
        for (int a1 = 0; a1 <= a0; a1 += 2)
            for (int a2 = 0; a2 <= (D == 3 ? a1 : 0); a2 += 2) {
                if (a0 + a1 + a2 > maxdeg) continue;
                a[m][0] = a0; a[m][1] = a1; a[m][2] = a2;
                double v = 1.0;
                int e[3] = {a0, a1, a2};
                for (int d = 0; d < 3; ++d)
                    for (int k = e[d] - 1; k > 0; k -= 2) v *= k;
                rhs[m] = v;
                ++m;
            }
    return m;
}

static void orc_shell_matrix(const orc_lattice *L, double r, int m, int (*a)[3], double *M)
{
    for (int row = 0; row < m; ++row)
        for (int s = 0; s < L->nshell; ++s) {
            double acc = 0.0;
            for (int q = 0; q < L->Q; ++q) {
                if (L->shell[q] != s) continue;
                double t = 1.0;
                for (int d = 0; d < L->D; ++d) t *= pow(r * L->c[q][d], a[row][d]);
                acc += t;
            }
            M[row * L->nshell + s] = acc;
        }
}

/* Root in [lo, hi] of the determinant of the augmented moment system of a 2-D lattice
 * whose shells are one fewer than its moment conditions up to maxdeg (degree 9: 9
 * conditions, 8 shells; degree 13: 16 conditions, 15 shells), consistent only at that
 * scale r, by bisection.  Each condition is divided by its (positive) right-hand side. */
static double orc_solve_r(orc_lattice *L2, int maxdeg, double lo, double hi)
{
    int (*a)[3] = malloc(sizeof(int[32][3]));
    double rhs[32], M[32 * 16], Aug[16 * 16];
    int m2 = orc_moment_conditions(2, maxdeg, a, rhs);
    const int ns = L2->nshell, n = ns + 1;
    if (m2 != n) { free(a); return NAN; }
    for (int it = 0; it < 200; ++it) {
        double rr[2] = {lo, 0.5 * (lo + hi)}, f[2];
        for (int k = 0; k < 2; ++k) {
            orc_shell_matrix(L2, rr[k], m2, a, M);
            for (int i = 0; i < m2; ++i) {
                for (int j = 0; j < ns; ++j) Aug[i * n + j] = M[i * ns + j] / rhs[i];
                Aug[i * n + ns] = 1.0;
            }
            f[k] = orc_det(n, Aug);
        }
        if ((f[1] < 0) == (f[0] < 0)) lo = rr[1]; else hi = rr[1];
        if (hi - lo < 1e-15) break;
    }
    free(a);
    return 0.5 * (lo + hi);
}

/* Builds the lattice: velocities from the shell generators; the scale r of a 2-D lattice
 * is the root of the determinant of its augmented moment system (degree 9: D2Q37 in
 * [1.1, 1.3]; D2Q33 in [1.14, 1.18], around its printed 0.819381 sqrt(2) = 1.15878;
 * degree 13: D2Q77 in [0.96, 0.98], the only root in [0.8, 1.4]); the shell weights are
 * then the least-squares (= exact) solution of the row-normalised conditions.  D3Q103
 * reuses D2Q37's r. */
static int orc_build_lattice(int lattice, orc_lattice *L)
{
    memset(L, 0, sizeof(*L));
    double r;
    int maxdeg = 8;
    if (lattice == ORC_D2Q33) {
        L->D = 2;
        L->nshell = 8;
        for (int s = 0; s < 8; ++s) orc_add_shell(L, ORC_SHELLS_2D33[s], s);
        r = orc_solve_r(L, 8, 1.14, 1.18);
    } else if (lattice == ORC_D2Q77) {
        L->D = 2;
        L->nshell = 15;
        for (int s = 0; s < 15; ++s) orc_add_shell(L, ORC_SHELLS_2D77[s], s);
        maxdeg = 12;
        r = orc_solve_r(L, 12, 0.96, 0.98);
    } else {
        orc_lattice L2;
        memset(&L2, 0, sizeof(L2));
        L2.D = 2;
        L2.nshell = 8;
        for (int s = 0; s < 8; ++s) orc_add_shell(&L2, ORC_SHELLS_2D[s], s);
        r = orc_solve_r(&L2, 8, 1.1, 1.3);
        if (lattice == ORC_D2Q37) {
            *L = L2;
        } else if (lattice == ORC_D3Q103) {
            L->D = 3;
            L->nshell = 10;
            for (int s = 0; s < 10; ++s) orc_add_shell(L, ORC_SHELLS_3D[s], s);
        } else {
            return -1;
        }
    }
    L->r = r;
    int (*a)[3] = malloc(sizeof(int[32][3]));
    double rhs[32], M[32 * 16], ones[32], ws[16];
    int m = orc_moment_conditions(L->D, maxdeg, a, rhs);
    orc_shell_matrix(L, r, m, a, M);
    for (int i = 0; i < m; ++i) {
        for (int j = 0; j < L->nshell; ++j) M[i * L->nshell + j] /= rhs[i];
        ones[i] = 1.0;
    }
    orc_lstsq(m, L->nshell, M, ones, ws);
    for (int q = 0; q < L->Q; ++q) L->w[q] = ws[L->shell[q]];
    free(a);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Tensor Hermite machinery (Sec. IV).                                        */
/* ------------------------------------------------------------------------- */

/* Grad's symmetrised products are sums over the distinct placements of the
 * factors' indices.  A placement of pair-tensors and vectors over n index slots is
 * a partial pairing of the slots: a set of disjoint slot pairs (each carrying a
 * rank-2 factor) and the remaining single slots (each carrying the vector).
 * This routine enumerates all partial pairings of n slots once. */
typedef struct {
    int npairs;
    int pair[ORC_MAXN / 2][2];
    int nsingle;
    int single[ORC_MAXN];
} orc_pairing;

static int orc_enum_pairings(int n, int used, orc_pairing cur, orc_pairing *out, int count)
{
    int p = -1;
    for (int s = 0; s < n; ++s)
        if (!(used >> s & 1)) { p = s; break; }
    if (p < 0) { out[count] = cur; return count + 1; }
    orc_pairing a = cur; /* slot p is a single */
    a.single[a.nsingle++] = p;
    count = orc_enum_pairings(n, used | 1 << p, a, out, count);
    for (int q = p + 1; q < n; ++q) { /* slot p paired with slot q */
        if (used >> q & 1) continue;
        orc_pairing b = cur;
        b.pair[b.npairs][0] = p; b.pair[b.npairs][1] = q; b.npairs++;
        count = orc_enum_pairings(n, used | 1 << p | 1 << q, b, out, count);
    }
    return count;
}

static orc_pairing *orc_pairings[ORC_MAXN + 1];
static int orc_npairings[ORC_MAXN + 1];

static void orc_init_pairings(void)
{
    if (orc_pairings[0]) return;
    for (int n = 0; n <= ORC_MAXN; ++n) {
        orc_pairing *buf = malloc(sizeof(orc_pairing) * 800);
        orc_pairing z;
        memset(&z, 0, sizeof(z));
        orc_npairings[n] = orc_enum_pairings(n, 0, z, buf, 0);
        orc_pairings[n] = buf;
    }
}

static int orc_ipow(int b, int e) { int v = 1; while (e--) v *= b; return v; }

/* Slot indices of flat tensor index t (row-major over n slots of D values). */
static void orc_unflatten(int t, int n, int D, int *idx)
{
    for (int s = n - 1; s >= 0; --s) { idx[s] = t % D; t /= D; }
}

/* H^(n)(xi): Grad's formula H^(n) = xi^n - delta xi^(n-2) + delta^2 xi^(n-4) - ...
 * (Sec. IV), i.e. a sum over partial pairings with one delta per pair, xi on the
 * single slots and sign (-1)^(number of pairs). */
static void orc_hermite_tensor(int n, int D, const double *xi, double *H)
{
    orc_init_pairings();
    int nt = orc_ipow(D, n), idx[ORC_MAXN];
    for (int t = 0; t < nt; ++t) {
        orc_unflatten(t, n, D, idx);
        double acc = 0.0;
        for (int k = 0; k < orc_npairings[n]; ++k) {
            const orc_pairing *P = &orc_pairings[n][k];
            double term = (P->npairs & 1) ? -1.0 : 1.0;
            for (int j = 0; j < P->npairs && term != 0.0; ++j)
                term *= idx[P->pair[j][0]] == idx[P->pair[j][1]] ? 1.0 : 0.0;
            for (int j = 0; j < P->nsingle; ++j) term *= xi[idx[P->single[j]]];
            acc += term;
        }
        H[t] = acc;
    }
}

/* a^(n) by the general term formula Eq. fESCoe:
 *   a^(n) = sum_{alpha=0}^{[n/2]} sum_{beta=0}^{alpha} (-1)^(alpha-beta) Lambda^beta delta^(alpha-beta) u^(n-2 alpha)
 * with Grad's symmetrised products: for every partial pairing with alpha pairs, every
 * choice of beta of those pairs to carry Lambda (the rest carry delta) and u on the
 * single slots contributes one term. */
static void orc_hermite_coeff_tensor(int n, int D, const double *u, const double *Lam, double *a)
{
    orc_init_pairings();
    int nt = orc_ipow(D, n), idx[ORC_MAXN];
    for (int t = 0; t < nt; ++t) {
        orc_unflatten(t, n, D, idx);
        double acc = 0.0;
        for (int alpha = 0; alpha <= n / 2; ++alpha)
            for (int beta = 0; beta <= alpha; ++beta) {
                double sign = ((alpha - beta) & 1) ? -1.0 : 1.0;
                for (int k = 0; k < orc_npairings[n]; ++k) {
                    const orc_pairing *P = &orc_pairings[n][k];
                    if (P->npairs != alpha) continue;
                    double uprod = 1.0;
                    for (int j = 0; j < P->nsingle; ++j) uprod *= u[idx[P->single[j]]];
                    /* every subset of beta pairs that carries Lambda */
                    for (int mask = 0; mask < (1 << alpha); ++mask) {
                        if (__builtin_popcount(mask) != beta) continue;
                        double term = sign * uprod;
                        for (int j = 0; j < alpha; ++j) {
                            int i0 = idx[P->pair[j][0]], i1 = idx[P->pair[j][1]];
                            term *= (mask >> j & 1) ? Lam[i0 * D + i1] : (i0 == i1 ? 1.0 : 0.0);
                        }
                        acc += term;
                    }
                }
            }
        a[t] = acc;
    }
}

static double orc_factorial(int n) { double f = 1; for (int k = 2; k <= n; ++k) f *= k; return f; }

/* Per-lattice table of H^(n)(xi_i), n <= order, computed once. */
typedef struct {
    int order;
    double *H[ORC_MAXN + 1]; /* [Q][D^n] */
} orc_htab;

static void orc_build_htab(const orc_lattice *L, int order, orc_htab *T)
{
    T->order = order;
    for (int n = 0; n <= order; ++n) {
        int nt = orc_ipow(L->D, n);
        T->H[n] = malloc(sizeof(double) * nt * L->Q);
        for (int i = 0; i < L->Q; ++i) {
            double xi[3];
            for (int d = 0; d < L->D; ++d) xi[d] = L->r * L->c[i][d];
            orc_hermite_tensor(n, L->D, xi, T->H[n] + (size_t)i * nt);
        }
    }
}

static void orc_free_htab(orc_htab *T)
{
    for (int n = 0; n <= T->order; ++n) free(T->H[n]);
}

/* Discrete truncated Gaussian, Eq. GExpansion with G_i = w_i G(xi_i) / omega(xi_i):
 *   G_i = w_i rho sum_{n=0}^{order} (1/n!) a^(n) . H^(n)(xi_i)
 * with the full index contraction "." over all D^n index tuples. */
static void orc_equilibrium_tab(const orc_lattice *L, const orc_htab *T, double rho,
                                const double *u, const double *Lam, double *G)
{
    double a[7][729]; /* order <= 6, D <= 3 */
    for (int n = 0; n <= T->order; ++n) orc_hermite_coeff_tensor(n, L->D, u, Lam, a[n]);
    for (int i = 0; i < L->Q; ++i) {
        double s = 0.0;
        for (int n = 0; n <= T->order; ++n) {
            int nt = orc_ipow(L->D, n);
            const double *H = T->H[n] + (size_t)i * nt;
            double c = 0.0;
            for (int t = 0; t < nt; ++t) c += a[n][t] * H[t];
            s += c / orc_factorial(n);
        }
        G[i] = L->w[i] * rho * s;
    }
}

/* ------------------------------------------------------------------------- */
/* Parameter mapping (Sec. III Eq. Gamma, Eq. Pr; reading R3).                */
/* ------------------------------------------------------------------------- */

typedef struct {
    double Nf, omega, nuG, tau_s, tau_q, kappa;
} orc_coeffs;

static int orc_map_params(int D, double Pr, double gamma, double Nf_in, double kappa,
                          double tau, int mode, orc_coeffs *k)
{
    /* Eq. Gamma: gamma = (N_f + D + 2)/(N_f + D)  =>  N_f = 2/(gamma-1) - D */
    k->Nf = gamma > 0.0 ? 2.0 / (gamma - 1.0) - D : Nf_in;
    if (k->Nf < -1e-12) return -1;
    if (k->Nf < 0) k->Nf = 0.0;
    k->kappa = kappa;
    if (mode == ORC_PR_LITERAL) {
        /* collision rate Pr/tau_f (Eq. DiscreteReductionG), 1 - nu + kappa nu = 1/Pr (Eq. Pr) */
        k->omega = Pr / tau;
        k->nuG = kappa < 1.0 ? (1.0 - 1.0 / Pr) / (1.0 - kappa) : 0.0;
        k->tau_s = tau;
        k->tau_q = tau / Pr;
    } else {
        k->tau_s = tau;
        k->tau_q = (tau - 0.5) / Pr + 0.5;
        k->omega = 1.0 / k->tau_q;
        k->nuG = kappa < 1.0 ? (1.0 - k->tau_q / k->tau_s) / (1.0 - kappa) : 0.0;
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Moments and the corrected tensor (Sec. II, Sec. V).                        */
/* ------------------------------------------------------------------------- */

typedef struct {
    double rho, u[3], sigma[9], Ttr, Tint, Teq, Trel, Lam[9];
} orc_state;

static void orc_moments_of(const orc_lattice *L, const orc_coeffs *k, const double *g,
                           const double *h, orc_state *s)
{
    int D = L->D;
    double rho = 0.0, j[3] = {0, 0, 0}, ekin2 = 0.0, H = 0.0;
    for (int i = 0; i < L->Q; ++i) {
        rho += g[i];                                    /* rho   = sum g_i          */
        double x2 = 0.0;
        for (int d = 0; d < D; ++d) {
            double xi = L->r * L->c[i][d];
            j[d] += g[i] * xi;                          /* rho u = sum g_i xi_i     */
            x2 += xi * xi;
        }
        ekin2 += 0.5 * x2 * g[i];                       /* rho(u^2/2 + e_tr)        */
        H += h[i];                                      /* rho e_int (reading R2)   */
    }
    s->rho = rho;
    double u2 = 0.0;
    for (int d = 0; d < D; ++d) { s->u[d] = j[d] / rho; u2 += s->u[d] * s->u[d]; }
    double e_tr = ekin2 / rho - 0.5 * u2;
    s->Ttr = 2.0 * e_tr / D;                            /* e_tr = (D/2) T_tr        */
    /* sigma = (1/rho) sum (xi - u)(xi - u) g   (Eq. Lambda, discrete) */
    for (int a = 0; a < D; ++a)
        for (int b = 0; b < D; ++b) {
            double acc = 0.0;
            for (int i = 0; i < L->Q; ++i)
                acc += (L->r * L->c[i][a] - s->u[a]) * (L->r * L->c[i][b] - s->u[b]) * g[i];
            s->sigma[a * D + b] = acc / rho;
        }
    if (k->Nf > 0.0) {
        double e_int = H / rho;
        s->Tint = 2.0 * e_int / k->Nf;                  /* e_int = (N_f/2) T_int    */
        s->Teq = (D * s->Ttr + k->Nf * s->Tint) / (D + k->Nf); /* e = (D+N_f)/2 T_eq */
    } else {
        s->Tint = 0.0;
        s->Teq = s->Ttr;
    }
    s->Trel = k->kappa * s->Teq + (1.0 - k->kappa) * s->Tint; /* T_rel, Sec. II */
    if (k->Nf == 0.0) s->Trel = s->Teq;
    /* Lambda = (1-kappa)[(1-nu) T_tr delta + nu sigma] + kappa T_eq delta */
    for (int a = 0; a < D; ++a)
        for (int b = 0; b < D; ++b)
            s->Lam[a * D + b] = (1.0 - k->kappa) * ((a == b ? (1.0 - k->nuG) * s->Ttr : 0.0)
                                                   + k->nuG * s->sigma[a * D + b])
                              + (a == b ? k->kappa * s->Teq : 0.0);
}

/* ------------------------------------------------------------------------- */
/* Simulation state.                                                          */
/* ------------------------------------------------------------------------- */

typedef struct {
    orc_lattice L;
    orc_htab T;
    orc_coeffs k;
    int nx, ny, nz, walls, gh, nys; /* gh ghost rows beyond each wall row; nys stored rows */
    int open_x;                     /* zero-gradient open ends in x (reading R16) */
    double uw[2][3], Tw[2];
    double *g, *h, *g2, *h2;        /* [stored cell][i] */
    long steps;
} orc_sim;

static size_t orc_cell(const orc_sim *S, int x, int ys, int z)
{
    return ((size_t)z * S->nys + ys) * S->nx + x;
}

static int orc_mod(int a, int n) { int m = a % n; return m < 0 ? m + n : m; }

/* Equilibrium populations of state (rho, u, T delta): g part and h part (R6). */
static void orc_maxwell_pops(const orc_sim *S, double rho, const double *u, double T,
                             double *g, double *h)
{
    int D = S->L.D;
    double Lam[9] = {0};
    for (int d = 0; d < D; ++d) Lam[d * D + d] = T;
    orc_equilibrium_tab(&S->L, &S->T, rho, u, Lam, g);
    for (int i = 0; i < S->L.Q; ++i) h[i] = 0.5 * S->k.Nf * T * g[i];
}

void *orc_create(int lattice, int nx, int ny, int nz, int walls, double Pr, double gamma,
                 double Nf, double kappa, double tau, int mode, const double *wall_u,
                 const double *wall_T)
{
    orc_sim *S = calloc(1, sizeof(orc_sim));
    if (orc_build_lattice(lattice, &S->L)) { free(S); return NULL; }
    if (orc_map_params(S->L.D, Pr, gamma, Nf, kappa, tau, mode, &S->k)) { free(S); return NULL; }
    /* the Hermite expansion's order: 4 (Eq. GExpansion) on the degree-9 lattices, 6 (the
     * Burnett order, Sec. IV) on the degree-13 D2Q77 */
    orc_build_htab(&S->L, lattice == ORC_D2Q77 ? 6 : 4, &S->T);
    S->nx = nx; S->ny = ny; S->nz = S->L.D == 3 ? nz : 1;
    S->walls = walls;
    /* walls: D2Q37 or D3Q103 (reach 3: two ghost rows beyond each wall row suffice) */
    if (walls && (lattice == ORC_D2Q33 || lattice == ORC_D2Q77 || ny < 5)) { orc_free_htab(&S->T); free(S); return NULL; }
    S->gh = walls ? 2 : 0;
    S->nys = ny + 2 * S->gh;
    for (int b = 0; b < 2; ++b) {
        for (int d = 0; d < 3; ++d) S->uw[b][d] = wall_u ? wall_u[b * 3 + d] : 0.0;
        S->Tw[b] = wall_T ? wall_T[b] : 1.0;
    }
    size_t n = (size_t)S->nx * S->nys * S->nz * S->L.Q;
    S->g = calloc(n, sizeof(double)); S->h = calloc(n, sizeof(double));
    S->g2 = calloc(n, sizeof(double)); S->h2 = calloc(n, sizeof(double));
    return S;
}

int orc_set_open_x(void *p, int open)
{
    ((orc_sim *)p)->open_x = open ? 1 : 0;
    return 0;
}

void orc_destroy(void *p)
{
    orc_sim *S = p;
    if (!S) return;
    free(S->g); free(S->h); free(S->g2); free(S->h2);
    orc_free_htab(&S->T);
    free(S);
}

static void orc_walls(orc_sim *S, double *g, double *h);

/* Fields are SoA [component][z][y][x] over the Nx x Ny (x Nz) domain. */
int orc_init(void *p, const double *rho, const double *u, const double *T)
{
    orc_sim *S = p;
    int D = S->L.D, Q = S->L.Q;
    size_t ncell = (size_t)S->nx * S->ny * S->nz;
    #pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < S->nz; ++z)
        for (int ys = 0; ys < S->nys; ++ys) {
            int y = ys - S->gh;
            if (y < 0) y = 0;
            if (y > S->ny - 1) y = S->ny - 1; /* ghost rows take the nearest row's field */
            for (int x = 0; x < S->nx; ++x) {
                size_t f = ((size_t)z * S->ny + y) * S->nx + x;
                double uu[3] = {0, 0, 0};
                for (int d = 0; d < D; ++d) uu[d] = u[d * ncell + f];
                size_t c = orc_cell(S, x, ys, z);
                orc_maxwell_pops(S, rho[f], uu, T[f], S->g + c * Q, S->h + c * Q);
            }
        }
    /* reading R6: the wall procedure fills the wall and ghost rows from the initial fluid
     * rows, as after every step, so the first streaming exchanges mass with the walls in
     * balance too: the fluid rows keep exactly their initial mass from the start */
    if (S->walls) orc_walls(S, S->g, S->h);
    S->steps = 0;
    return 0;
}

/* One collision of a cell's (streamed) populations: Eq. DiscreteReductionG / H with the
 * h target (N_f/2) T_rel G_i (reading R1). */
static void orc_collide(const orc_sim *S, const double *g, const double *h, double *go, double *ho)
{
    orc_state st;
    double G[ORC_MAXQ];
    orc_moments_of(&S->L, &S->k, g, h, &st);
    orc_equilibrium_tab(&S->L, &S->T, st.rho, st.u, st.Lam, G);
    double om = S->k.omega;
    for (int i = 0; i < S->L.Q; ++i) {
        go[i] = g[i] - om * (g[i] - G[i]);
        ho[i] = h[i] - om * (h[i] - 0.5 * S->k.Nf * st.Trel * G[i]);
    }
}

/* Wall procedure (reading R5), applied to the post-collision buffer.  For each wall
 * and column x: the state of the boundary row at distance k from the wall (k = 0 is the
 * wall row, k = 1, 2 the ghost rows) is u_k = u_w - k (u_1 - u_w), T_k = T_w - k (T_1 - T_w)
 * with (u_1, T_1) the first fluid row's; its populations are rho_w G(1, u_k, T_k delta)
 * plus the first fluid row's non-equilibrium (its populations minus their Maxwellian).
 * rho_w balances, exactly, the mass that crosses into the boundary rows of column x in
 * the next streaming against the mass those rows send back into the fluid. */
static void orc_walls(orc_sim *S, double *g, double *h)
{
    int Q = S->L.Q, D = S->L.D;
    for (int b = 0; b < 2; ++b) {
        int n = b == 0 ? 1 : -1;               /* wall normal (y), into the fluid */
        int yw = b == 0 ? 0 : S->ny - 1;       /* wall row */
        int yn = yw + n;                       /* first fluid row */
        /* one wall column per (x, z) (z = 0 in 2-D) */
        #pragma omp parallel for collapse(2) schedule(static)
        for (int z = 0; z < S->nz; ++z)
        for (int x = 0; x < S->nx; ++x) {
            /* non-equilibrium of the first fluid row: populations minus their Maxwellian */
            size_t cn1 = orc_cell(S, x, yn + S->gh, z);
            const double *gn = g + cn1 * Q, *hn = h + cn1 * Q;
            orc_state st;
            orc_moments_of(&S->L, &S->k, gn, hn, &st);
            double Mg[ORC_MAXQ], Mh[ORC_MAXQ], neq_g[ORC_MAXQ], neq_h[ORC_MAXQ];
            orc_maxwell_pops(S, st.rho, st.u, st.Teq, Mg, Mh);
            for (int i = 0; i < Q; ++i) { neq_g[i] = gn[i] - Mg[i]; neq_h[i] = hn[i] - Mh[i]; }
            /* boundary-row states and their unit-density equilibria */
            double Tk[3], Gk[3][ORC_MAXQ], Hk[3][ORC_MAXQ];
            for (int kk = 0; kk <= S->gh; ++kk) {
                double uk[3] = {0, 0, 0};
                for (int d = 0; d < D; ++d) uk[d] = S->uw[b][d] - kk * (st.u[d] - S->uw[b][d]);
                Tk[kk] = S->Tw[b] - kk * (st.Teq - S->Tw[b]);
                orc_maxwell_pops(S, 1.0, uk, Tk[kk], Gk[kk], Hk[kk]);
            }
            /* mass leaving the fluid into column (x, z)'s boundary rows: population i
             * (moving toward the wall) from fluid rows 1..|c_iy| away from the wall */
            double leaving = 0.0, A = 0.0, B = 0.0;
            for (int i = 0; i < Q; ++i) {
                int cn = S->L.c[i][1] * n;
                int xs = orc_mod(x - S->L.c[i][0], S->nx);
                int zs = orc_mod(z - S->L.c[i][2], S->nz);
                if (cn < 0)
                    for (int s = 1; s <= -cn; ++s)
                        leaving += g[orc_cell(S, xs, yw + n * s + S->gh, zs) * Q + i];
                /* mass the boundary rows k = 0..c_n-1 send into the fluid */
                if (cn > 0)
                    for (int kk = 0; kk < cn; ++kk) { A += Gk[kk][i]; B += neq_g[i]; }
            }
            double rho_w = (leaving - B) / A;
            for (int kk = 0; kk <= S->gh; ++kk) {
                size_t c = orc_cell(S, x, yw - n * kk + S->gh, z);
                for (int i = 0; i < Q; ++i) {
                    g[c * Q + i] = rho_w * Gk[kk][i] + neq_g[i];
                    h[c * Q + i] = rho_w * Hk[kk][i] + neq_h[i];
                }
            }
        }
    }
}

/* nsteps of pull-stream + collide (Eq. DiscreteReductionG / H), then walls. */
int orc_step(void *p, int nsteps)
{
    orc_sim *S = p;
    int Q = S->L.Q;
    int y0 = S->walls ? 1 : 0, y1 = S->walls ? S->ny - 2 : S->ny - 1;
    for (int step = 0; step < nsteps; ++step) {
        #pragma omp parallel for collapse(2) schedule(static)
        for (int z = 0; z < S->nz; ++z)
            for (int y = y0; y <= y1; ++y) {
                double gs[ORC_MAXQ], hs[ORC_MAXQ];
                for (int x = 0; x < S->nx; ++x) {
                    for (int i = 0; i < Q; ++i) {
                        /* g_i(x + xi_i dt, t + dt) <- post-collision g_i(x, t): pull from x - c_i */
                        int xs = x - S->L.c[i][0];
                        /* open ends: a population entering from outside the domain is the
                         * boundary cell's own (zero-gradient) */
                        xs = S->open_x ? (xs < 0 ? 0 : (xs > S->nx - 1 ? S->nx - 1 : xs)) : orc_mod(xs, S->nx);
                        int ys = S->walls ? y - S->L.c[i][1] : orc_mod(y - S->L.c[i][1], S->ny);
                        int zs = orc_mod(z - S->L.c[i][2], S->nz);
                        size_t c = orc_cell(S, xs, ys + S->gh, zs);
                        gs[i] = S->g[c * Q + i];
                        hs[i] = S->h[c * Q + i];
                    }
                    size_t c = orc_cell(S, x, y + S->gh, z);
                    orc_collide(S, gs, hs, S->g2 + c * Q, S->h2 + c * Q);
                }
            }
        if (S->walls) orc_walls(S, S->g2, S->h2);
        double *t = S->g; S->g = S->g2; S->g2 = t;
        t = S->h; S->h = S->h2; S->h2 = t;
        S->steps++;
    }
    return 0;
}

/* Macroscopic fields of the stored populations over the domain, SoA [comp][z][y][x]:
 * rho, u (D), T = T_eq, Pi = rho sigma (D(D+1)/2: xx,xy,(xz),yy,(yz),(zz)) and the heat
 * flux q_a = sum g_i |xi_i-u|^2 (xi_i-u)_a / 2 + sum h_i (xi_i-u)_a.  Any output may be NULL. */
int orc_moments(void *p, double *rho, double *u, double *T, double *Pi, double *q)
{
    orc_sim *S = p;
    int D = S->L.D, Q = S->L.Q;
    size_t ncell = (size_t)S->nx * S->ny * S->nz;
    #pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < S->nz; ++z)
        for (int y = 0; y < S->ny; ++y)
            for (int x = 0; x < S->nx; ++x) {
                size_t f = ((size_t)z * S->ny + y) * S->nx + x;
                size_t c = orc_cell(S, x, y + S->gh, z);
                const double *g = S->g + c * Q, *h = S->h + c * Q;
                orc_state st;
                orc_moments_of(&S->L, &S->k, g, h, &st);
                if (rho) rho[f] = st.rho;
                if (u) for (int d = 0; d < D; ++d) u[d * ncell + f] = st.u[d];
                if (T) T[f] = st.Teq;
                if (Pi) {
                    int m = 0;
                    for (int a = 0; a < D; ++a)
                        for (int b = a; b < D; ++b) Pi[(m++) * ncell + f] = st.rho * st.sigma[a * D + b];
                }
                if (q) {
                    double qa[3] = {0, 0, 0};
                    for (int i = 0; i < Q; ++i) {
                        double v[3] = {0, 0, 0}, v2 = 0.0;
                        for (int d = 0; d < D; ++d) { v[d] = S->L.r * S->L.c[i][d] - st.u[d]; v2 += v[d] * v[d]; }
                        for (int d = 0; d < D; ++d) qa[d] += 0.5 * v2 * v[d] * g[i] + v[d] * h[i];
                    }
                    for (int d = 0; d < D; ++d) q[d * ncell + f] = qa[d];
                }
            }
    return 0;
}

/* Totals over the domain: out = {mass, momentum x, y, z, total energy sum(xi^2 g/2 + h)}. */
int orc_diagnostics(void *p, double *out)
{
    orc_sim *S = p;
    int D = S->L.D, Q = S->L.Q;
    double m = 0, j[3] = {0, 0, 0}, E = 0;
    for (int z = 0; z < S->nz; ++z)
        for (int y = 0; y < S->ny; ++y)
            for (int x = 0; x < S->nx; ++x) {
                size_t c = orc_cell(S, x, y + S->gh, z);
                for (int i = 0; i < Q; ++i) {
                    double g = S->g[c * Q + i], x2 = 0;
                    m += g;
                    for (int d = 0; d < D; ++d) {
                        double xi = S->L.r * S->L.c[i][d];
                        j[d] += g * xi;
                        x2 += xi * xi;
                    }
                    E += 0.5 * x2 * g + S->h[c * Q + i];
                }
            }
    out[0] = m; out[1] = j[0]; out[2] = j[1]; out[3] = j[2]; out[4] = E;
    return 0;
}

/* Populations over the domain rows, SoA [i][z][y][x] (no ghost rows). */
int orc_get_pops(void *p, double *g, double *h)
{
    orc_sim *S = p;
    int Q = S->L.Q;
    size_t ncell = (size_t)S->nx * S->ny * S->nz;
    for (int z = 0; z < S->nz; ++z)
        for (int y = 0; y < S->ny; ++y)
            for (int x = 0; x < S->nx; ++x) {
                size_t f = ((size_t)z * S->ny + y) * S->nx + x, c = orc_cell(S, x, y + S->gh, z);
                for (int i = 0; i < Q; ++i) {
                    if (g) g[i * ncell + f] = S->g[c * Q + i];
                    if (h) h[i * ncell + f] = S->h[c * Q + i];
                }
            }
    return 0;
}

/* Sets the domain populations from SoA [i][z][y][x]; wall ghost rows are rebuilt by the
 * wall procedure. */
int orc_set_pops(void *p, const double *g, const double *h)
{
    orc_sim *S = p;
    int Q = S->L.Q;
    size_t ncell = (size_t)S->nx * S->ny * S->nz;
    for (int z = 0; z < S->nz; ++z)
        for (int y = 0; y < S->ny; ++y)
            for (int x = 0; x < S->nx; ++x) {
                size_t f = ((size_t)z * S->ny + y) * S->nx + x, c = orc_cell(S, x, y + S->gh, z);
                for (int i = 0; i < Q; ++i) {
                    S->g[c * Q + i] = g[i * ncell + f];
                    S->h[c * Q + i] = h[i * ncell + f];
                }
            }
    if (S->walls) orc_walls(S, S->g, S->h);
    return 0;
}

long orc_steps(void *p) { return ((orc_sim *)p)->steps; }

/* ------------------------------------------------------------------------- */
/* Entry points for the pin tests.                                            */
/* ------------------------------------------------------------------------- */

/* Lattice: D, Q, r, integer velocities c[Q][3], weights w[Q].  Returns Q or -1. */
int orc_lattice_info(int lattice, int *D, int *Q, double *r, int *c, double *w)
{
    orc_lattice L;
    if (orc_build_lattice(lattice, &L)) return -1;
    if (D) *D = L.D;
    if (Q) *Q = L.Q;
    if (r) *r = L.r;
    for (int i = 0; i < L.Q; ++i) {
        if (c) for (int d = 0; d < 3; ++d) c[i * 3 + d] = L.c[i][d];
        if (w) w[i] = L.w[i];
    }
    return L.Q;
}

int orc_hermite_poly(int n, int D, const double *xi, double *out)
{
    if (n < 0 || n > ORC_MAXN || D < 1 || D > 3) return -1;
    orc_hermite_tensor(n, D, xi, out);
    return 0;
}

int orc_hermite_coeff(int n, int D, const double *u, const double *Lam, double *out)
{
    if (n < 0 || n > ORC_MAXN || D < 1 || D > 3) return -1;
    orc_hermite_coeff_tensor(n, D, u, Lam, out);
    return 0;
}

/* Discrete equilibrium G_i of (rho, u, Lambda) truncated at `order` (<= 6). */
int orc_equilibrium(int lattice, int order, double rho, const double *u, const double *Lam, double *G)
{
    orc_lattice L;
    orc_htab T;
    if (order < 0 || order > 6 || orc_build_lattice(lattice, &L)) return -1;
    orc_build_htab(&L, order, &T);
    orc_equilibrium_tab(&L, &T, rho, u, Lam, G);
    orc_free_htab(&T);
    return 0;
}

/* Mapped coefficients: out = {N_f, omega, nu_G, tau_s, tau_q}. */
int orc_params(int D, double Pr, double gamma, double Nf, double kappa, double tau, int mode, double *out)
{
    orc_coeffs k;
    if (orc_map_params(D, Pr, gamma, Nf, kappa, tau, mode, &k)) return -1;
    out[0] = k.Nf; out[1] = k.omega; out[2] = k.nuG; out[3] = k.tau_s; out[4] = k.tau_q;
    return 0;
}

/* One collision of a single cell's populations (for the invariant pins). */
int orc_collide_cell(void *p, const double *g, const double *h, double *go, double *ho)
{
    orc_collide((orc_sim *)p, g, h, go, ho);
    return 0;
}

/* Moments of a single cell's populations: out = {rho, u[3], Ttr, Tint, Teq, Trel, Lambda[9]}. */
int orc_cell_state(void *p, const double *g, const double *h, double *out)
{
    orc_sim *S = p;
    orc_state st;
    orc_moments_of(&S->L, &S->k, g, h, &st);
    out[0] = st.rho;
    for (int d = 0; d < 3; ++d) out[1 + d] = d < S->L.D ? st.u[d] : 0.0;
    out[4] = st.Ttr; out[5] = st.Tint; out[6] = st.Teq; out[7] = st.Trel;
    for (int a = 0; a < 9; ++a) out[8 + a] = 0.0;
    for (int a = 0; a < S->L.D; ++a)
        for (int b = 0; b < S->L.D; ++b) out[8 + a * 3 + b] = st.Lam[a * S->L.D + b];
    return 0;
}
