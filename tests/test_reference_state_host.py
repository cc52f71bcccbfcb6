"""The reference state's shifts as the kernels receive them (lbm_debug_reference_state,
host only, no GPU) against the FP64 oracle's rest equilibrium.

A handle with reference state (rho0, T0) stores g_i/w_i - 1 - dg_i and
h_i/w_i - N_f/2 - dh_i, with dg, dh the rest equilibrium at (rho0, u = 0, T0) over the
weight, less rho = T = 1.  The library computes them per shell from a closed form (the
isotropic Hermite terms of a Maxwellian at rest as Laguerre polynomials); the oracle builds
the same equilibrium from the paper's tensor contraction.  The moment shares must be the
lattice sums of the rounded shifts, which for the exact equilibrium are its mass rho0 - 1,
internal energy (N_f/2)(rho0 T0 - 1) and second moment (rho0 T0 - 1)/r^2 per axis."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1611_02409_gb300 import lbm as L

CASES = [(L.LBM_D2Q37, O.D2Q37, 1.25, 0.8), (L.LBM_D2Q37, O.D2Q37, 1.0, 1.2), (L.LBM_D2Q37, O.D2Q37, 0.9, 1.0),
         (L.LBM_D3Q103, O.D3Q103, 1.25, 0.85), (L.LBM_D3Q103, O.D3Q103, 1.0, 1.15),
         (L.LBM_D2Q33, O.D2Q33, 1.1, 0.9), (L.LBM_D2Q77, O.D2Q77, 1.2, 1.1)]


def oracle_rest(olat, D, rho0, T0, gamma):
    shape = (2,) * D
    nz, ny, nx = (1,) * (3 - D) + shape
    o = O.Sim(olat, nx=nx, ny=ny, nz=nz, Pr=0.71, gamma=gamma, kappa=0.2, tau=0.8)
    o.init(np.full(shape, rho0), np.zeros((D,) + shape), np.full(shape, T0))
    g, h = o.populations()
    c = np.array(o.c)
    o.close()
    return g.reshape(len(c), -1)[:, 0], h.reshape(len(c), -1)[:, 0], c


@pytest.mark.parametrize("lat,olat,rho0,T0", CASES)
def test_shifts_are_the_oracle_rest_equilibrium(lat, olat, rho0, T0):
    gamma = 1.4
    D, r, c, w = L.lbm_lattice_table(lat)
    p = L.make_params(lattice=lat, nx=8, ny=8, nz=8 if D == 3 else 1, gamma=gamma, tau=0.8, rho0=rho0, T0=T0)
    dg, dh, share = L.lbm_debug_reference_state(p)
    Nf = 2.0 / (gamma - 1.0) - D
    go, ho, co = oracle_rest(olat, D, rho0, T0, gamma)
    idx = [next(j for j in range(len(co)) if tuple(co[j]) == tuple(v)) for v in c]
    want_g = go[idx] / w - 1.0
    want_h = ho[idx] / w - 0.5 * Nf
    # the shifts reach the kernels as FP32 launch parameters
    assert np.abs(dg - want_g).max() <= 1e-7 * max(1.0, np.abs(want_g).max())
    assert np.abs(dh - want_h).max() <= 1e-7 * max(1.0, np.abs(want_h).max())
    # shares: the lattice sums of the rounded shifts (hi + lo, to ~1e-15) ...
    c2 = c[:, :3].astype(float) ** 2
    sums = [np.sum(w * dg), np.sum(w * dh)] + [np.sum(w * dg * c2[:, a]) for a in range(3)]
    assert np.allclose(share, sums, rtol=0, atol=1e-14)
    # ... and, the equilibrium being exact to second order, its mass, internal energy and
    # second moment
    assert share[0] == pytest.approx(rho0 - 1.0, abs=1e-7)
    assert share[1] == pytest.approx(0.5 * Nf * (rho0 * T0 - 1.0), abs=2e-7)
    for a in range(D):
        assert share[2 + a] == pytest.approx((rho0 * T0 - 1.0) / r ** 2, abs=1e-7)


def test_unit_reference_has_no_shift():
    for lat in (L.LBM_D2Q37, L.LBM_D3Q103, L.LBM_D2Q33, L.LBM_D2Q77):
        for ref in (dict(rho0=1.0, T0=1.0), dict(rho0=0.0, T0=0.0)):
            p = L.make_params(lattice=lat, nx=8, ny=8, nz=8 if lat == L.LBM_D3Q103 else 1, tau=0.8, **ref)
            dg, dh, share = L.lbm_debug_reference_state(p)
            assert not dg.any() and not dh.any() and not share.any()


def test_invalid_reference_is_refused():
    with pytest.raises(L.LbmError):
        L.lbm_debug_reference_state(L.make_params(T0=-1.0))
