"""Pins of the oracle's discrete equilibrium and collision (Secs. IV-V).

* G_i (Eq. GExpansion, full tensor contraction) against the same truncated expansion
  built independently in the 1-D product basis: G/omega projected on He_alpha(xi) =
  prod_d He_{alpha_d}(xi_d), |alpha| <= 4, with the projections E[He_alpha] of the exact
  Gaussian computed by Gauss-Hermite quadrature.
* Lattice moments of G_i up to order 4 equal the Gaussian's moments (rho, rho u,
  rho(Lambda + uu), ...), which a degree-9 lattice integrates exactly.  On the degree-13
  D2Q77 the sixth-order expansion (a^(5), a^(6) of Sec. IV) reproduces them up to order 6
  and the fourth-order one does not.
* Collision invariants: mass, momentum and total energy (reading R1, T_rel in the h
  target); equilibrium is a fixed point; the stress deviator and the translational-
  internal temperature gap relax at the rates the parameter mapping (reading R3) sets.
"""
import itertools
from math import factorial

import numpy as np
import pytest
from numpy.polynomial import hermite_e as He

from oracle import oracle as O

rng = np.random.default_rng(77)


def he(k, x):
    c = np.zeros(k + 1)
    c[k] = 1.0
    return He.hermeval(x, c)


def gauss_expect(D, u, Lam, f, m=8):
    z, wz = He.hermegauss(m)
    wz = wz / np.sqrt(2 * np.pi)
    Lc = np.linalg.cholesky(Lam)
    acc = 0.0
    for nodes in itertools.product(range(m), repeat=D):
        acc = acc + np.prod(wz[list(nodes)]) * f(u + Lc @ z[list(nodes)])
    return acc


def product_basis_equilibrium(which, rho, u, Lam, order=4):
    D, r, c, w = O.lattice(which)
    xi = r * c[:, :D].astype(float)
    P = np.zeros(len(c))
    for alpha in itertools.product(range(order + 1), repeat=D):
        if sum(alpha) > order:
            continue
        coef = gauss_expect(D, u, Lam, lambda x: np.prod([he(alpha[d], x[d]) for d in range(D)]))
        coef /= np.prod([factorial(a) for a in alpha])
        P += coef * np.prod([he(alpha[d], xi[:, d]) for d in range(D)], axis=0)
    return w * rho * P


def spd(D, s=0.15):
    A = rng.normal(size=(D, D)) * s
    return (0.9 + 0.2 * rng.random()) * np.eye(D) + 0.5 * (A + A.T)


@pytest.mark.parametrize("which", [O.D2Q37, O.D3Q103])
def test_equilibrium_vs_product_basis(which):
    D = 2 if which == O.D2Q37 else 3
    for _ in range(2):
        rho, u, Lam = 0.8 + 0.4 * rng.random(), rng.normal(size=D) * 0.2, spd(D)
        G = O.equilibrium(which, rho, u, Lam)
        ref = product_basis_equilibrium(which, rho, u, Lam)
        assert np.allclose(G, ref, rtol=1e-11, atol=1e-15)


@pytest.mark.parametrize("which", [O.D2Q37, O.D3Q103])
def test_equilibrium_moments_to_order4(which):
    D, r, c, w = O.lattice(which)
    xi = r * c[:, :D].astype(float)
    rho, u, Lam = 1.1, rng.normal(size=D) * 0.2, spd(D)
    G = O.equilibrium(which, rho, u, Lam)
    for deg in range(5):
        for alpha in itertools.product(range(deg + 1), repeat=D):
            if sum(alpha) != deg:
                continue
            lat = np.sum(G * np.prod(xi ** np.array(alpha), axis=1))
            ref = rho * gauss_expect(D, u, Lam, lambda x: np.prod(x ** np.array(alpha)))
            assert abs(lat - ref) < 1e-12 * max(1, abs(ref)), (alpha, lat, ref)


def _moment_errors(which, order, maxdeg, rho, u, Lam):
    D, r, c, w = O.lattice(which)
    xi = r * c[:, :D].astype(float)
    G = O.equilibrium(which, rho, u, Lam, order=order)
    out = {}
    for deg in range(maxdeg + 1):
        for a in range(deg + 1):
            alpha = np.array((a, deg - a))
            lat = np.sum(G * np.prod(xi ** alpha, axis=1))
            ref = rho * gauss_expect(D, u, Lam, lambda x: np.prod(x ** alpha))
            out[(a, deg - a)] = abs(lat - ref) / max(1, abs(ref))
    return out


def test_d2q77_sixth_order_moments():
    # Sec. IV: the sixth-order expansion reproduces the Gaussian's moments up to order 6
    # on a degree-13 lattice (6 + 6 <= 13); order 7 is beyond the truncation
    rho, u, Lam = 0.93, np.array([0.35, -0.2]), spd(2, 0.2)
    e6 = _moment_errors(O.D2Q77, 6, 7, rho, u, Lam)
    assert max(v for k, v in e6.items() if sum(k) <= 6) < 1e-12, e6
    assert max(v for k, v in e6.items() if sum(k) == 7) > 1e-6
    # the fourth-order expansion on the same lattice misses orders 5 and 6
    e4 = _moment_errors(O.D2Q77, 4, 6, rho, u, Lam)
    assert max(v for k, v in e4.items() if sum(k) <= 4) < 1e-12
    assert min(max(v for k, v in e4.items() if sum(k) == d) for d in (5, 6)) > 1e-5, e4


def test_d2q77_equilibrium_vs_product_basis():
    rho, u, Lam = 1.07, np.array([-0.25, 0.15]), spd(2)
    G = O.equilibrium(O.D2Q77, rho, u, Lam, order=6)
    ref = product_basis_equilibrium(O.D2Q77, rho, u, Lam, order=6)
    assert np.allclose(G, ref, rtol=1e-11, atol=1e-16)


def test_equilibrium_order4_truncation_differs_from_order6():
    # the fifth and sixth Hermite terms are dropped (Eq. GExpansion), so orders differ
    u, Lam = np.array([0.3, 0.1]), np.array([[1.1, 0.05], [0.05, 0.95]])
    G4 = O.equilibrium(O.D2Q37, 1.0, u, Lam, order=4)
    G6 = O.equilibrium(O.D2Q37, 1.0, u, Lam, order=6)
    assert np.abs(G4 - G6).max() > 1e-6


def _perturbed_state(sim, rho=1.05, u=(0.05, -0.03, 0.02), T=1.02, amp=2e-3, which=None):
    D = sim.D
    u = np.array(u[:D], float)
    which = which or (O.D2Q37 if D == 2 else O.D3Q103)
    G = O.equilibrium(which, rho, u, T * np.eye(D), order=6 if which == O.D2Q77 else 4)
    g = G * (1 + amp * rng.normal(size=G.size))
    h = 0.5 * sim.coeffs["Nf"] * T * G * (1 + amp * rng.normal(size=G.size))
    return g, h


def _invariants(sim, g, h):
    xi = sim.r * sim.c[:, :sim.D].astype(float)
    return np.concatenate([[g.sum()], g @ xi, [np.sum(0.5 * (xi ** 2).sum(1) * g) + h.sum()]])


@pytest.mark.parametrize("which", [O.D2Q37, O.D3Q103, O.D2Q77])
@pytest.mark.parametrize("Pr,gamma,kappa,mode", [(0.71, 1.4, 0.2, O.PR_SHIFTED), (2.0, 1.3, 0.5, O.PR_SHIFTED),
                                                 (0.71, 1.4, 0.2, O.PR_LITERAL), (1.0, 1.1, 0.9, O.PR_SHIFTED)])
def test_collision_conserves_mass_momentum_energy(which, Pr, gamma, kappa, mode):
    sim = O.Sim(which, nx=4, ny=4, nz=4, Pr=Pr, gamma=gamma, kappa=kappa, tau=0.8, mode=mode)
    for _ in range(3):
        g, h = _perturbed_state(sim, which=which)
        go, ho = sim.collide_cell(g, h)
        # FP64 sums of 2Q terms of size <= ~3: roundoff <= 2Q * 2^-53 * 3 (~7e-14 for Q = 103)
        tol = 2 * len(g) * 2.0 ** -53 * 3
        dev = np.abs(_invariants(sim, go, ho) - _invariants(sim, g, h))
        assert np.all(dev <= tol), (dev, tol, sim.coeffs)
        assert np.abs(go - g).max() > 1e-6  # something did relax


def test_equilibrium_is_fixed_point():
    sim = O.Sim(O.D2Q37, nx=4, ny=4, Pr=0.71, gamma=1.4, kappa=0.2, tau=0.7)
    rho, u, T = 0.97, np.array([0.04, 0.01]), 1.03
    G = O.equilibrium(O.D2Q37, rho, u, T * np.eye(2))
    h = 0.5 * sim.coeffs["Nf"] * T * G
    go, ho = sim.collide_cell(G, h)
    assert np.allclose(go, G, atol=1e-15) and np.allclose(ho, h, atol=1e-15)


@pytest.mark.parametrize("mode", [O.PR_SHIFTED, O.PR_LITERAL])
@pytest.mark.parametrize("Pr", [0.5, 0.71, 2.0])
def test_relaxation_rates_match_mapping(mode, Pr):
    # traceless stress relaxes at omega (1 - nu + kappa nu); T_tr - T_eq at omega kappa.
    # In SHIFTED mode the first must be 1/tau_s exactly and omega = 1/tau_q.
    tau, kappa = 0.9, 0.2
    sim = O.Sim(O.D2Q37, nx=4, ny=4, Pr=Pr, gamma=1.4, kappa=kappa, tau=tau, mode=mode)
    k = sim.coeffs
    g, h = _perturbed_state(sim, amp=5e-3)
    s0, s1 = sim.cell_state(g, h), None
    go, ho = sim.collide_cell(g, h)
    s1 = sim.cell_state(go, ho)
    xi = sim.r * sim.c[:, :2].astype(float)

    def dev_stress(gg, st):
        v = xi - st["u"]
        P = (gg[:, None, None] * v[:, :, None] * v[:, None, :]).sum(0)
        return P - np.trace(P) / 2 * np.eye(2)

    rate = 1 - dev_stress(go, s1)[0, 1] / dev_stress(g, s0)[0, 1]
    expect = k["omega"] * (1 - k["nuG"] + kappa * k["nuG"])
    assert rate == pytest.approx(expect, rel=1e-9)
    if mode == O.PR_SHIFTED:
        assert rate == pytest.approx(1 / tau, rel=1e-12)
        assert k["omega"] == pytest.approx(1 / ((tau - 0.5) / Pr + 0.5), rel=1e-14)
    else:
        assert k["omega"] == pytest.approx(Pr / tau, rel=1e-14)
        assert 1 - k["nuG"] + kappa * k["nuG"] == pytest.approx(1 / Pr, rel=1e-12)
    gap0, gap1 = s0["Ttr"] - s0["Teq"], s1["Ttr"] - s1["Teq"]
    assert 1 - gap1 / gap0 == pytest.approx(k["omega"] * kappa, rel=1e-8)


def test_gamma_maps_to_Nf():
    # Eq. Gamma: gamma = (N_f + D + 2)/(N_f + D)
    for D, gamma in [(2, 1.4), (3, 1.4), (2, 1.3), (2, 1.67)]:
        Nf = O.params(D, 0.71, gamma)["Nf"]
        assert (Nf + D + 2) / (Nf + D) == pytest.approx(gamma, rel=1e-13)
