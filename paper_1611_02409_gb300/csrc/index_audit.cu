// Host-side audit of the stream-collide kernels' addressing (lbm_debug_index_audit).
//
// compute-sanitizer is not available where these kernels run, so every gather and store
// is checked here on the host instead: for each computed cell of a configuration, the
// element indices a kernel variant reads and writes are formed with the kernels' own index
// helpers (wrap_sub, src_x, cell_index, the byte offsets make_kparams tabulates, the wrap
// threshold the launch uses), following each kernel's choice between its fixed-offset
// interior gather and its wrapped seam gather.  An access counts as bad when it falls
// outside the 2 Q planes of a population buffer, when a 32-bit access of the paired kernel
// is off a 4-byte boundary, or when it is not the element the pull-stream definition
// names: population i of the cell at (x, y, z) - c_i, periodic by plain modulo, clamped at
// open x ends, in the ghost rows beyond walls (and the cell's own element for a store).
// With walls, the wall kernel's reads (first fluid row, the leaving populations' cells)
// and writes (wall and ghost rows) are audited too; LBM_AUDIT_BATCH audits one instance
// of the batched step (32-bit offsets).  No device work.
#include "../../include/lbm.h"
#include "dispatch.cuh"

namespace lbm {
namespace {

struct Tally {
    long long total = 0;   // elements in one population buffer
    long long bad = 0;
    void check(long long e)
    {
        if (e < 0 || e >= total) ++bad;
    }
    // in range and equal to the element the definition names
    void check(long long e, long long want)
    {
        check(e);
        if (e != want) ++bad;
    }
    // a 32-bit access at element e of 16-bit storage: both halves in range, word-aligned
    void check_word(long long e)
    {
        check(e);
        check(e + 1);
        if (e % 2 != 0) ++bad;
    }
};

int mod(int a, int n) { return ((a % n) + n) % n; }

// The element that population p (set * Q + i) of the cell (x, y, z) pulls from, from the
// definition alone: the source cell (x, y, z) - c_i, periodic in x, y, z by modulo, x
// clamped at open ends, y into the ghost rows when there are walls.
template <int LAT>
long long want_src(const KParams<LAT> &kp, int set, int i, int x, int y, int z)
{
    constexpr int D = Lattice<LAT>::D, Q = Lattice<LAT>::Q;
    const int cx = Lattice<LAT>::T.c[i][0], cy = Lattice<LAT>::T.c[i][1], cz = Lattice<LAT>::T.c[i][2];
    int xs = x - cx;
    xs = kp.open_x ? (xs < 0 ? 0 : (xs >= kp.nx ? kp.nx - 1 : xs)) : mod(xs, kp.nx);
    const int ys = kp.gh ? y - cy + kp.gh : mod(y - cy, kp.ny);
    const int zs = D == 3 ? mod(z - cz, kp.nz) : 0;
    return (long long)(set * Q + i) * kp.plane + ((long long)zs * kp.nys + ys) * kp.nx + xs;
}

// ... and the element of population p of the cell (x, y, z) itself (stores, own-cell reads).
template <int LAT> long long own_elem(const KParams<LAT> &kp, int p, int x, int y, int z)
{
    return (long long)p * kp.plane + ((long long)z * kp.nys + y + kp.gh) * kp.nx + x;
}

// k_stream_collide (direct): fixed byte offsets away from the seams, wrapped indices near them.
template <int LAT, bool WALLS>
void audit_direct(const KParams<LAT> &kp, long long elem, bool sx, bool sy, bool sz, int x, int y, int z, Tally &t)
{
    constexpr int D = Lattice<LAT>::D, Q = Lattice<LAT>::Q, R = Lattice<LAT>::R;
    const long long o = cell_index<LAT>(kp, x, y + kp.gh, z);
    bool interior = x >= R && x + R < kp.nx;
    if (!WALLS) interior = interior && y >= R && y + R < kp.ny;
    if (D == 3) interior = interior && z >= R && z + R < kp.nz;
    if (interior) {
        for (int p = 0; p < 2 * Q; ++p) t.check(o + kp.goff[p] / elem, want_src(kp, p / Q, p % Q, x, y, z));
    } else {
        static_for<0, Q>([&](auto II) {
            constexpr int I = decltype(II)::value;
            constexpr int cx = cv<LAT, I, 0>(), cy = cv<LAT, I, 1>(), cz = cv<LAT, I, 2>();
            const int xs = src_x<cx>(x, kp.nx, sx, kp.open_x);
            const int ys = WALLS ? y - cy + kp.gh : wrap_sub<cy>(y, kp.ny, sy);
            const int zs = D == 3 ? wrap_sub<cz>(z, kp.nz, sz) : z;
            const long long idx = cell_index<LAT>(kp, xs, ys, zs);
            t.check((long long)I * kp.plane + idx, want_src(kp, 0, I, x, y, z));
            t.check((long long)(Q + I) * kp.plane + idx, want_src(kp, 1, I, x, y, z));
        });
    }
    for (int p = 0; p < 2 * Q; ++p) t.check(o + kp.soff[p] / elem, own_elem(kp, p, x, y, z));
}

// k_stream_collide_2p (two-pass): tabulated wrapped columns, rows and planes for -R..R.
template <int LAT, bool WALLS>
void audit_twopass(const KParams<LAT> &kp, long long elem, bool sx, bool sy, bool sz, int x, int y, int z, Tally &t)
{
    constexpr int D = Lattice<LAT>::D, Q = Lattice<LAT>::Q, R = Lattice<LAT>::R;
    long long col[2 * R + 1], row[2 * R + 1], pln[2 * R + 1];
    static_for<0, 2 * R + 1>([&](auto KK) {
        constexpr int C = decltype(KK)::value - R;
        col[KK] = src_x<C>(x, kp.nx, sx, kp.open_x);
        const int ys = WALLS ? y - C + kp.gh : wrap_sub<C>(y, kp.ny, sy);
        row[KK] = (long long)ys * kp.nx;
        pln[KK] = D == 3 ? (long long)wrap_sub<C>(z, kp.nz, sz) * kp.nys * kp.nx : 0;
    });
    static_for<0, Q>([&](auto II) {
        constexpr int I = decltype(II)::value;
        const long long at = pln[cv<LAT, I, 2>() + R] + row[cv<LAT, I, 1>() + R] + col[cv<LAT, I, 0>() + R];
        t.check((long long)I * kp.plane + at, want_src(kp, 0, I, x, y, z));
        t.check((long long)(Q + I) * kp.plane + at, want_src(kp, 1, I, x, y, z));
    });
    const long long o = cell_index<LAT>(kp, x, y + kp.gh, z);
    for (int p = 0; p < 2 * Q; ++p) t.check(o + kp.soff[p] / elem, own_elem(kp, p, x, y, z));
}

// k_stream_collide_pair (two cells x, x + 1 per thread, 16-bit storage, 128-thread blocks).
template <int LAT, bool WALLS>
void audit_paired(const KParams<LAT> &kp, long long elem, bool sy, int x, int y, Tally &t)
{
    constexpr int Q = Lattice<LAT>::Q, R = Lattice<LAT>::R;
    const long long o = cell_index<LAT>(kp, x, y + kp.gh, 0);
    const int xb = 2 * 128 * (x / 256);
    bool interior = xb >= R + 1 && xb + 2 * 128 + R + 1 <= kp.nx;
    if (!WALLS) interior = interior && y >= R && y + R < kp.ny;
    if (interior) {
        static_for<0, Q>([&](auto II) {
            constexpr int I = decltype(II)::value;
            constexpr int cx = cv<LAT, I, 0>();
            for (int set = 0; set < 2; ++set) {
                // the (merged) word holds the sources of the cells x and x + 1 at e and e + 1
                const long long e = o + kp.goff[set * Q + I] / elem;
                if (cx % 2 == 0) {
                    t.check_word(e);
                } else {
                    t.check_word(e - 1);
                    t.check_word(e + 1);
                }
                t.check(e, want_src(kp, set, I, x, y, 0));
                t.check(e + 1, want_src(kp, set, I, x + 1, y, 0));
            }
        });
    } else {
        const bool sx = kp.nx < 4;   // the paired kernel's own seam threshold (reach 3)
        static_for<0, Q>([&](auto II) {
            constexpr int I = decltype(II)::value;
            constexpr int cx = cv<LAT, I, 0>(), cy = cv<LAT, I, 1>();
            const int x0 = wrap_sub<cx>(x, kp.nx, sx), x1 = wrap_sub<cx>(x + 1, kp.nx, sx);
            const int ys = WALLS ? y - cy + kp.gh : wrap_sub<cy>(y, kp.ny, sy);
            const long long row = (long long)ys * kp.nx;
            for (int set = 0; set < 2; ++set) {
                const long long ps = (long long)(set * Q + I) * kp.plane + row;
                t.check(ps + x0, want_src(kp, set, I, x, y, 0));
                t.check(ps + x1, want_src(kp, set, I, x + 1, y, 0));
            }
        });
    }
    for (int p = 0; p < 2 * Q; ++p) {
        t.check_word(o + kp.soff[p] / elem);
        t.check(o + kp.soff[p] / elem, own_elem(kp, p, x, y, 0));
    }
}

// k_walls (one thread per column x, wall b, plane z): reads the first fluid row's cell and,
// for each population leaving the fluid toward the wall, the cells 1 .. |c_y| rows inside
// displaced by -c_x (-c_z); writes the wall row and the two ghost rows beyond it.
template <int LAT> void audit_walls(const KParams<LAT> &kp, int x, int b, int z, Tally &t)
{
    constexpr int D = Lattice<LAT>::D, Q = Lattice<LAT>::Q;
    const int n = b == 0 ? 1 : -1;
    const int yw = b == 0 ? 0 : kp.ny - 1;
    const int small_x = kp.nx < 4, small_z = kp.nz < 4;   // the wall kernel's own (reach 3)
    const long long o1 = cell_index<LAT>(kp, x, yw + n + kp.gh, z);
    for (int p = 0; p < 2 * Q; ++p) t.check((long long)p * kp.plane + o1, own_elem(kp, p, x, yw + n, z));
    static_for<0, Q>([&](auto II) {
        constexpr int I = decltype(II)::value;
        constexpr int cx = cv<LAT, I, 0>(), cy = cv<LAT, I, 1>(), cz = cv<LAT, I, 2>();
        const int cn = cy * n;
        if (cy != 0 && cn < 0) {
            const int xs = wrap_sub<cx>(x, kp.nx, small_x);
            const int zs = D == 3 ? wrap_sub<cz>(z, kp.nz, small_z) : 0;
            for (int sdist = 1; sdist <= -cn; ++sdist) {
                const int yf = yw + n * sdist;   // a fluid row
                if (yf < 1 || yf > kp.ny - 2) ++t.bad;
                const long long want = (long long)I * kp.plane +
                    (((long long)(D == 3 ? mod(z - cz, kp.nz) : 0) * kp.nys + yf + kp.gh) * kp.nx + mod(x - cx, kp.nx));
                t.check((long long)I * kp.plane + cell_index<LAT>(kp, xs, yf + kp.gh, zs), want);
            }
        }
    });
    for (int k = 0; k <= 2; ++k) {
        const int yr = yw - n * k;            // the wall row, then the ghost rows beyond it
        const long long o = cell_index<LAT>(kp, x, yr + kp.gh, z);
        for (int p = 0; p < 2 * Q; ++p) t.check((long long)p * kp.plane + o, own_elem(kp, p, x, yr, z));
    }
}

// k_bstep (batched instances, D2Q37 FP32): per instance, 32-bit element offsets from the
// instance's buffer, stencil rows and columns tabulated for -3..3 with the batch's own
// wrap threshold (4); every product and sum must also fit a 32-bit int.
void audit_batch(const KParams<LAT_D2Q37> &kp, int walls, int x, int y, Tally &t)
{
    constexpr int LAT = LAT_D2Q37, Q = Lattice<LAT>::Q;
    const long long kMax = 2147483647LL;
    const int nx = kp.nx, ny = kp.ny, gh = kp.gh;
    const long long pl = kp.plane;
    if (pl > kMax) ++t.bad;
    const bool sx = nx < 4, sy = ny < 4;
    long long rowo[7], col[7];
    static_for<0, 7>([&](auto KK) {
        constexpr int C = decltype(KK)::value - 3;
        const int ys = walls ? y - C + gh : wrap_sub<C>(y, ny, sy);
        rowo[KK] = (long long)ys * nx;
        col[KK] = wrap_sub<C>(x, nx, sx);
    });
    static_for<0, Q>([&](auto II) {
        constexpr int I = decltype(II)::value;
        const long long idx = rowo[cv<LAT, I, 1>() + 3] + col[cv<LAT, I, 0>() + 3];
        for (int set = 0; set < 2; ++set) {
            const long long e = (long long)(set * Q + I) * pl + idx;
            if (e > kMax || (long long)(set * Q + I) * pl > kMax) ++t.bad;
            t.check(e, want_src(kp, set, I, x, y, 0));
        }
    });
    const long long o = (long long)(y + gh) * nx + x;
    for (int p = 0; p < 2 * Q; ++p) {
        if ((long long)p * pl > kMax) ++t.bad;
        t.check((long long)p * pl + o, own_elem(kp, p, x, y, 0));
    }
}

// k_stream_collide_tma (staged, D2Q37): per tile of TW cells (x0, y, z) and plane p, the
// bulk copies of the source row segment [x0 - H, x0 + TW + H) (three pieces at a periodic
// seam) into the stage row; each copy must lie in the buffer, start 16-byte aligned at
// both ends and move a multiple of 16 bytes; then each cell's read stage[p][H + tx - c_x]
// must hold the element the definition names.
template <int ST, bool WALLS> void audit_staged(const KParams<LAT_D2Q37> &kp, int x0, int y, int z, Tally &t)
{
    constexpr int LAT = LAT_D2Q37, Q = Lattice<LAT>::Q;
    using G = TileGeom<ST>;
    constexpr long long sz = sizeof(typename G::T);
    const bool small_y = kp.ny < 4;
    const bool interior = x0 >= G::H && x0 + G::TW + G::H <= kp.nx;
    for (int p = 0; p < 2 * Q; ++p) {
        const int i = p < Q ? p : p - Q;
        const int cx = Lattice<LAT>::T.c[i][0], cy = Lattice<LAT>::T.c[i][1];
        int ys;
        if (WALLS) {
            ys = y - cy + kp.gh;
        } else {
            ys = y - cy;
            if (small_y) ys = ((ys % kp.ny) + kp.ny) % kp.ny;
            else ys += ys < 0 ? kp.ny : (ys >= kp.ny ? -kp.ny : 0);
        }
        const long long row = (long long)p * kp.plane + ((long long)z * kp.nys + ys) * kp.nx;
        // stage index j -> global element, from the copies issued
        long long src_of[G::L];
        auto copy = [&](int j0, long long e0, int n) {
            t.check(e0);
            t.check(e0 + n - 1);
            if ((e0 * sz) % 16 != 0 || ((long long)n * sz) % 16 != 0 ||
                ((long long)(p * G::L + j0) * sz) % 16 != 0)
                ++t.bad;
            for (int j = 0; j < n; ++j) src_of[j0 + j] = e0 + j;
        };
        if (interior) {
            copy(0, row + (x0 - G::H), G::L);
        } else {
            const int xl = x0 == 0 ? kp.nx - G::H : x0 - G::H;
            const int xr = x0 + G::TW == kp.nx ? 0 : x0 + G::TW;
            copy(0, row + xl, G::H);
            copy(G::H, row + x0, G::TW);
            copy(G::H + G::TW, row + xr, G::H);
        }
        for (int tx = 0; tx < G::TW; ++tx) {
            const int j = G::H + tx - cx;
            if (j < 0 || j >= G::L) {
                ++t.bad;
                continue;
            }
            t.check(src_of[j], want_src(kp, p / Q, i, x0 + tx, y, z));
        }
    }
    for (int tx = 0; tx < G::TW; ++tx) {
        const long long o = cell_index<LAT>(kp, x0 + tx, y + kp.gh, z);
        for (int p = 0; p < 2 * Q; ++p) t.check(o + kp.soff[p] / sz, own_elem(kp, p, x0 + tx, y, z));
    }
}

template <int LAT, bool WALLS> long long audit(const Ctx &c, int variant, int wrap)
{
    constexpr int D = Lattice<LAT>::D, Q = Lattice<LAT>::Q;
    const KParams<LAT> kp = make_kparams<LAT>(c);
    const long long elem = storage_bytes(c.storage);
    Tally t;
    t.total = 2LL * Q * c.plane;
    const int kWrap = wrap > 0 ? wrap : wrap_threshold<LAT>();
    const bool sx = c.nx < kWrap, sy = c.ny < kWrap, sz = c.nz < kWrap;
    const int y0 = c.walls ? 1 : 0, ncomp = c.walls ? c.ny - 2 : c.ny;
    if constexpr (LAT == LAT_D2Q37) {
        if (variant == LBM_KERNEL_STAGED) {
            // the tiles the launch enumerates: (nx / TW) per row, ncomp rows
            const int TW = c.storage == 0 ? TileGeom<ST_FP32>::TW : TileGeom<ST_FP16>::TW;
            for (int tile = 0; tile < (c.nx / TW) * ncomp; ++tile) {
                const int x0 = (tile % (c.nx / TW)) * TW, y = y0 + (tile / (c.nx / TW)) % ncomp;
                if (c.storage == 0) audit_staged<ST_FP32, WALLS>(kp, x0, y, 0, t);
                else audit_staged<ST_FP16, WALLS>(kp, x0, y, 0, t);   // FP16 and BF16: 2-byte values
            }
            if constexpr (WALLS)
                for (int b = 0; b < 2; ++b)
                    for (int x = 0; x < c.nx; ++x) audit_walls<LAT>(kp, x, b, 0, t);
            return t.bad;
        }
    }
    for (int z = 0; z < (D == 3 ? c.nz : 1); ++z)
        for (int yy = 0; yy < ncomp; ++yy)
            for (int x = 0; x < c.nx; ++x) {
                const int y = y0 + yy;
                if (variant == LBM_AUDIT_BATCH) {
                    if constexpr (LAT == LAT_D2Q37) audit_batch(kp, c.walls, x, y, t);
                } else if (variant == LBM_KERNEL_TWOPASS) audit_twopass<LAT, WALLS>(kp, elem, sx, sy, sz, x, y, z, t);
                else if (variant == LBM_KERNEL_DIRECT) audit_direct<LAT, WALLS>(kp, elem, sx, sy, sz, x, y, z, t);
                else if constexpr (LAT == LAT_D2Q37)
                    if (x % 2 == 0) audit_paired<LAT, WALLS>(kp, elem, c.ny < 4, x, y, t);
            }
    // the wall kernel runs after every step whichever variant streamed
    if constexpr (WALLS)
        for (int z = 0; z < (D == 3 ? c.nz : 1); ++z)
            for (int b = 0; b < 2; ++b)
                for (int x = 0; x < c.nx; ++x) audit_walls<LAT>(kp, x, b, z, t);
    return t.bad;
}

template <int LAT> long long audit_lattice(const Ctx &c, int variant, int wrap)
{
    if constexpr (LAT == LAT_D2Q37 || LAT == LAT_D3Q103)
        if (c.walls) return audit<LAT, true>(c, variant, wrap);
    return audit<LAT, false>(c, variant, wrap);
}

} // namespace
} // namespace lbm

extern "C" long long lbm_debug_index_audit(const lbm_params *p, int variant, int wrap_threshold)
{
    using namespace lbm;
    if (!p) return -LBM_ERR_ARG;
    Ctx c;
    int D = 0, Q = 0;
    double r = 0.0;
    const int rc = make_ctx(*p, c, &D, &Q, &r);
    if (rc != LBM_OK && rc != LBM_WARN_PR_RANGE) return -rc;
    const bool d2q37_16 = p->lattice == LBM_D2Q37 && (p->storage == LBM_FP16 || p->storage == LBM_BF16);
    if (p->storage == LBM_FP64 && variant != LBM_KERNEL_TWOPASS) return -LBM_ERR_ARG;   // two-pass only
    if (variant == LBM_KERNEL_PAIRED && !(d2q37_16 && !c.open_x && c.nx % 2 == 0)) return -LBM_ERR_ARG;
    if (variant == LBM_KERNEL_STAGED && !(p->lattice == LBM_D2Q37 && !c.open_x && c.nx % 128 == 0))
        return -LBM_ERR_ARG;   // what the staged launch admits
    if (variant == LBM_AUDIT_BATCH &&
        !(p->lattice == LBM_D2Q37 && p->storage == LBM_FP32 && !c.open_x && 2LL * Q * c.plane < (1LL << 31)))
        return -LBM_ERR_ARG;   // what lbm_batch_create admits
    if (variant != LBM_KERNEL_DIRECT && variant != LBM_KERNEL_TWOPASS && variant != LBM_KERNEL_PAIRED &&
        variant != LBM_KERNEL_STAGED && variant != LBM_AUDIT_BATCH)
        return -LBM_ERR_ARG;
    if (wrap_threshold < 0) return -LBM_ERR_ARG;
    switch (p->lattice) {
    case LBM_D2Q37: return audit_lattice<LAT_D2Q37>(c, variant, wrap_threshold);
    case LBM_D3Q103: return audit_lattice<LAT_D3Q103>(c, variant, wrap_threshold);
    case LBM_D2Q33: return audit_lattice<LAT_D2Q33>(c, variant, wrap_threshold);
    case LBM_D2Q77: return audit_lattice<LAT_D2Q77>(c, variant, wrap_threshold);
    default: return -LBM_ERR_ARG;
    }
}

// The shifts exactly as make_kparams hands them to the kernels (FP32 launch parameters,
// widened).
namespace {
template <int LAT> int reference_state(const lbm::Ctx &c, double *dg, double *dh, double *share)
{
    using namespace lbm;
    const KParams<LAT> kp = make_kparams<LAT>(c);
    for (int i = 0; i < Lattice<LAT>::Q; ++i) {
        const int sh = Lattice<LAT>::T.shell[i];
        if (dg) dg[i] = kp.ref_g[sh];
        if (dh) dh[i] = kp.ref_h[sh];
    }
    if (share)
        for (int k = 0; k < 5; ++k) share[k] = (double)kp.ref_hi[k] + (double)kp.ref_lo[k];
    return Lattice<LAT>::Q;
}
} // namespace

extern "C" int lbm_debug_reference_state(const lbm_params *p, double *dg, double *dh, double *share)
{
    using namespace lbm;
    if (!p) return -LBM_ERR_ARG;
    Ctx c;
    int D = 0, Q = 0;
    double r = 0.0;
    const int rc = make_ctx(*p, c, &D, &Q, &r);
    if (rc != LBM_OK && rc != LBM_WARN_PR_RANGE) return -rc;
    switch (p->lattice) {
    case LBM_D2Q37: return reference_state<LAT_D2Q37>(c, dg, dh, share);
    case LBM_D3Q103: return reference_state<LAT_D3Q103>(c, dg, dh, share);
    case LBM_D2Q33: return reference_state<LAT_D2Q33>(c, dg, dh, share);
    case LBM_D2Q77: return reference_state<LAT_D2Q77>(c, dg, dh, share);
    default: return -LBM_ERR_ARG;
    }
}
