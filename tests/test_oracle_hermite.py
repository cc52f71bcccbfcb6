"""Pins of the oracle's Hermite machinery (Sec. IV).

* H^(n) (Grad's formula) against products of numpy's 1-D probabilists' Hermite
  polynomials: a component with k_d indices equal to d is prod_d He_{k_d}(xi_d).
* a^(n) (general term formula, Eq. fESCoe) against brute-force tensor Gauss-Hermite
  quadrature of E_{xi ~ N(u, Lambda)}[H^(n)(xi)] (Eq. HermiteCo), with the integrand
  built from numpy's He_k, not from the oracle.
"""
import itertools

import numpy as np
import pytest
from numpy.polynomial import hermite_e as He

from oracle import oracle as O

rng = np.random.default_rng(1234)


def he(k, x):
    c = np.zeros(k + 1)
    c[k] = 1.0
    return He.hermeval(x, c)


def he_tensor_component(idx, xi):
    D = len(xi)
    return np.prod([he(list(idx).count(d), xi[d]) for d in range(D)], axis=0)


@pytest.mark.parametrize("D", [1, 2, 3])
@pytest.mark.parametrize("n", range(0, 7))
def test_hermite_poly_vs_numpy(D, n):
    for _ in range(3):
        xi = rng.normal(size=D) * 1.5
        H = O.hermite_poly(n, xi)
        for idx in itertools.product(range(D), repeat=n):
            ref = he_tensor_component(idx, xi)
            assert abs(H[idx] - ref) < 1e-11 * max(1.0, abs(ref)), (idx, H[idx], ref)


def gauss_expect(D, u, Lam, f, m=8):
    """E[f(xi)], xi ~ N(u, Lam), by an m^D-point tensor Gauss-Hermite rule (exact for
    polynomials of degree <= 2m-1 in each variable)."""
    z, wz = He.hermegauss(m)
    wz = wz / np.sqrt(2 * np.pi)
    Lc = np.linalg.cholesky(Lam)
    acc = 0.0
    for nodes in itertools.product(range(m), repeat=D):
        eta = z[list(nodes)]
        wt = np.prod(wz[list(nodes)])
        acc = acc + wt * f(u + Lc @ eta)
    return acc


def random_spd(D, scale=0.3):
    A = rng.normal(size=(D, D)) * scale
    return np.eye(D) + 0.5 * (A + A.T) + D * scale * np.eye(D) * 0.5


@pytest.mark.parametrize("D", [2, 3])
@pytest.mark.parametrize("n", range(0, 7))
def test_hermite_coeff_vs_quadrature(D, n):
    u = rng.normal(size=D) * 0.4
    Lam = random_spd(D)
    a = O.hermite_coeff(n, u, Lam)
    for idx in itertools.product(range(D), repeat=n):
        ref = gauss_expect(D, u, Lam, lambda xi: he_tensor_component(idx, xi))
        assert abs(a[idx] - ref) < 1e-10 * max(1.0, abs(ref)), (idx, a[idx], ref)


def test_hermite_coeff_low_orders_explicit():
    # the first orders printed after Eq. fESCoe, evaluated by hand for D = 2
    u = np.array([0.3, -0.2])
    Lam = np.array([[1.2, 0.1], [0.1, 0.8]])
    A = Lam - np.eye(2)
    assert O.hermite_coeff(0, u, Lam) == pytest.approx(1.0)
    assert np.allclose(O.hermite_coeff(1, u, Lam), u)
    assert np.allclose(O.hermite_coeff(2, u, Lam), A + np.outer(u, u))
    a3 = O.hermite_coeff(3, u, Lam)
    assert a3[0, 0, 0] == pytest.approx(3 * A[0, 0] * u[0] + u[0] ** 3)
    assert a3[0, 0, 1] == pytest.approx(A[0, 0] * u[1] + 2 * A[0, 1] * u[0] + u[0] ** 2 * u[1])
    a4 = O.hermite_coeff(4, u, Lam)
    assert a4[0, 0, 0, 0] == pytest.approx(3 * A[0, 0] ** 2 + 6 * A[0, 0] * u[0] ** 2 + u[0] ** 4)
    assert a4[0, 0, 1, 1] == pytest.approx(A[0, 0] * A[1, 1] + 2 * A[0, 1] ** 2 + A[0, 0] * u[1] ** 2
                                           + A[1, 1] * u[0] ** 2 + 4 * A[0, 1] * u[0] * u[1]
                                           + u[0] ** 2 * u[1] ** 2)


def test_hermite_coeff_maxwellian_special_case():
    # kappa = 1 (or nu = 0) gives Lambda = T delta: the polyatomic BGK Maxwellian, whose
    # 1-D coefficients are E[He_n(u + sqrt(T) z)] = sum_k n!/(k!(n-2k)! 2^k) (T-1)^k u^(n-2k)
    from math import factorial
    u, T = np.array([0.25, -0.1]), 1.3
    for n in range(7):
        a = O.hermite_coeff(n, u, T * np.eye(2))
        ref = sum(factorial(n) / (factorial(k) * factorial(n - 2 * k) * 2 ** k) * (T - 1) ** k
                  * u[0] ** (n - 2 * k) for k in range(n // 2 + 1))
        assert a[(0,) * n] == pytest.approx(ref, rel=1e-12, abs=1e-14)


def test_hermite_coeff_is_symmetric():
    u = rng.normal(size=3) * 0.3
    Lam = random_spd(3)
    a = O.hermite_coeff(5, u, Lam)
    for p in itertools.permutations(range(5)):
        assert np.allclose(a, np.transpose(a, p), atol=1e-14)
