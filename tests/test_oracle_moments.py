"""Pins of the oracle's reported moments (Sec. V moment sums; reading C-10 for the heat
flux) and of its FP64 totals, each against a fact fixed by the mathematics rather than
by the oracle's own formulas:

* The heat flux q = sum g |xi - u|^2 (xi - u)/2 + sum h (xi - u) is the central third
  moment of g plus the internal-energy flux.  Any Gaussian has a vanishing central third
  moment, and an h proportional to G carries no flux relative to u, so q = 0 (to
  roundoff) for the discrete equilibrium G(rho, u, Lambda) of a degree-9 lattice, with
  Lambda = T delta or Lambda != T delta (the ES Gaussian), at any u.
* Adding a third-order Hermite term  w rho b:H^(3)(xi)/6  (b symmetric) to g and
  w rho c.xi to h changes neither rho, u nor sigma (Hermite orthogonality), and by the same
  orthogonality q_a = (rho/2) sum_e b_eea + rho c_a, at any u: only the cubic part of
  |xi - u|^2 (xi - u) projects on H^(3).
* The pressure tensor reported for G(rho, u, Lambda) is rho Lambda.
* The totals: sum_i (xi^2 g_i/2 + h_i) over the domain equals
  sum rho (u^2/2 + (D + N_f) T_eq / 2), since rho E = rho u^2/2 + (D/2) rho T_tr +
  (N_f/2) rho T_int and (D + N_f) T_eq = D T_tr + N_f T_int (Sec. II); mass and
  momentum are the sums of rho and rho u.
"""
import numpy as np
import pytest

from oracle import oracle as O

rng = np.random.default_rng(2024)


def he3(xi):
    """H^(3)_{abc}(xi) = xi_a xi_b xi_c - (delta_ab xi_c + delta_ac xi_b + delta_bc xi_a)."""
    D = xi.size
    d = np.eye(D)
    return (np.einsum("a,b,c->abc", xi, xi, xi) - np.einsum("ab,c->abc", d, xi)
            - np.einsum("ac,b->abc", d, xi) - np.einsum("bc,a->abc", d, xi))


def sym3(D, s):
    b = rng.normal(size=(D, D, D)) * s
    return sum(np.transpose(b, p) for p in [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]) / 6


def es_lambda(D, T):
    A = rng.normal(size=(D, D)) * 0.05
    return T * np.eye(D) + 0.5 * (A + A.T)


def cell_states(which, ncell):
    D = O.lattice(which)[0]
    out = []
    for k in range(ncell):
        rho = 1.0 + 0.1 * rng.uniform(-1, 1)
        u = 0.15 * rng.uniform(-1, 1, D)
        T = 1.0 + 0.1 * rng.uniform(-1, 1)
        Lam = T * np.eye(D) if k % 2 == 0 else es_lambda(D, T)   # Maxwellian and ES Gaussians
        out.append((rho, u, T, Lam))
    return out


def sim_with(which, g, h, shape):
    D = O.lattice(which)[0]
    if D == 2:
        S = O.Sim(which, nx=shape[1], ny=shape[0], Pr=0.71, gamma=1.4, kappa=0.2, tau=0.8)
    else:
        S = O.Sim(which, nx=shape[2], ny=shape[1], nz=shape[0], Pr=0.71, gamma=1.4, kappa=0.2, tau=0.8)
    S.set_populations(g, h)
    return S


def build(which, shape, perturb):
    """Populations of per-cell Gaussians (optionally with the third-order perturbation)
    and the perturbation's expected heat flux per cell."""
    D, r, c, w = O.lattice(which)
    xi = r * c[:, :D].astype(float)
    Q, n = len(c), int(np.prod(shape))
    g, h = np.zeros((Q, n)), np.zeros((Q, n))
    states = cell_states(which, n)
    q_expect = np.zeros((D, n))
    for f, (rho, u, T, Lam) in enumerate(states):
        G = O.equilibrium(which, rho, u, Lam)
        g[:, f] = G
        h[:, f] = (1.5 + 0.5 * rng.random()) * T * G       # proportional to G: no relative flux
        if perturb:
            b = sym3(D, 0.02)
            ch = 0.01 * rng.normal(size=D)
            g[:, f] += w * rho * np.array([np.einsum("abc,abc->", b, he3(x)) for x in xi]) / 6.0
            h[:, f] += w * rho * (xi @ ch)
            q_expect[:, f] = 0.5 * rho * np.einsum("eea->a", b) + rho * ch
    return states, g.reshape((Q,) + shape), h.reshape((Q,) + shape), q_expect


@pytest.mark.parametrize("which,shape", [(O.D2Q37, (3, 4)), (O.D3Q103, (2, 2, 3))])
def test_heat_flux_vanishes_for_gaussians_and_pressure_is_rho_lambda(which, shape):
    D = O.lattice(which)[0]
    states, g, h, _ = build(which, shape, perturb=False)
    S = sim_with(which, g, h, shape)
    m = S.moments()
    n = int(np.prod(shape))
    q = m["q"].reshape(D, n)
    assert np.abs(q).max() < 1e-13, np.abs(q).max()
    Pi = m["Pi"].reshape(-1, n)
    u = m["u"].reshape(D, n)
    for f, (rho, u0, T, Lam) in enumerate(states):
        assert m["rho"].reshape(n)[f] == pytest.approx(rho, abs=1e-13)
        assert np.abs(u[:, f] - u0).max() < 1e-13
        k = 0
        for a in range(D):
            for b in range(a, D):
                assert Pi[k, f] == pytest.approx(rho * Lam[a, b], abs=1e-13)
                k += 1
    S.close()


@pytest.mark.parametrize("which,shape", [(O.D2Q37, (3, 4)), (O.D3Q103, (2, 2, 3)), (O.D2Q77, (2, 3))])
def test_heat_flux_of_a_third_order_hermite_term(which, shape):
    D = O.lattice(which)[0]
    states, g, h, q_expect = build(which, shape, perturb=True)
    S = sim_with(which, g, h, shape)
    m = S.moments()
    n = int(np.prod(shape))
    q = m["q"].reshape(D, n)
    assert np.abs(q_expect).max() > 1e-3                     # the case is not vacuous
    assert np.abs(q - q_expect).max() < 1e-13, np.abs(q - q_expect).max()
    # rho and u are those of the unperturbed Gaussians (orthogonality)
    u = m["u"].reshape(D, n)
    for f, (rho, u0, T, Lam) in enumerate(states):
        assert m["rho"].reshape(n)[f] == pytest.approx(rho, abs=1e-13)
        assert np.abs(u[:, f] - u0).max() < 1e-13
    S.close()


@pytest.mark.parametrize("which,shape", [(O.D2Q37, (4, 5)), (O.D3Q103, (2, 3, 2))])
def test_totals_equal_sums_of_the_moment_fields(which, shape):
    D, r, c, w = O.lattice(which)
    _, g, h, _ = build(which, shape, perturb=True)
    # a generic non-equilibrium state: positive random multiplicative noise on every population
    g = g * (1.0 + 0.05 * rng.uniform(-1, 1, g.shape))
    h = h * (1.0 + 0.05 * rng.uniform(-1, 1, h.shape))
    S = sim_with(which, g, h, shape)
    m = S.moments()
    d = S.diagnostics()
    Nf = S.coeffs["Nf"]
    rho, T = m["rho"], m["T"]
    u2 = (m["u"] ** 2).sum(axis=0)
    assert d["mass"] == pytest.approx(rho.sum(), rel=1e-14)
    for a in range(D):
        assert d["momentum"][a] == pytest.approx((rho * m["u"][a]).sum(), abs=1e-13)
    E = (rho * (0.5 * u2 + 0.5 * (D + Nf) * T)).sum()
    assert d["energy"] == pytest.approx(E, rel=1e-13)
    # and the total energy is not just the translational part: the h populations count
    assert abs(d["energy"] - (rho * (0.5 * u2 + 0.5 * D * T)).sum()) > 0.1 * abs(E)
    S.close()
