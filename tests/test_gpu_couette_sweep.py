"""Thermal Couette grid on the GPU (Sec. VI A): 4 x 256 channels, top wall moving at
U = 0.05 with T_top = 1.02, bottom wall at rest with T_bottom = 1, swept over
Pr in {0.5, 0.71, 1, 2} x gamma in {1.3, 1.4, 1.67}, FP32, all in one batch.

Steady compressible Couette flow with this scheme's transport has a constant dynamic
viscosity (mu = p (tau - 1/2) dt with uniform pressure) and conductivity, so u is
linear and T follows Eq. CouetteDi3 with unequal walls:
    T(eta) = T_b + (T_t - T_b) eta + Pr U^2 / (D + N_f + 2) eta (1 - eta),  eta = y/H.
Each case first runs to residual 1e-8 (per-step relative change of u_x and T); then all
continue for nine decay times of the slowest thermal mode, H^2 / (pi^2 nu / Pr), which
leaves far less than the FP32 rounding of the profile from the steady state.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

NU = 0.02  # lattice units at tau = 0.528655 on D2Q37


@pytest.fixture(scope="module")
def L():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_1611_02409_gb300 import build
    build.build()
    from paper_1611_02409_gb300 import lbm
    return lbm


def analytic(case, ny):
    Pr, gamma, U, _, dT = case["inputs"]
    Nf = 2.0 / (gamma - 1.0) - 2.0
    eta = np.arange(ny) / (ny - 1)
    heat = Pr * U ** 2 / (2 + Nf + 2)
    return U * eta, 1.0 + dT * eta + heat * eta * (1 - eta), heat


def test_couette_grid_matches_analytic_profile(L):
    from paper_1611_02409_gb300 import sweep
    cases = sweep.couette_grid()
    H = cases[0]["params"]["ny"]
    t_slow = (H - 1) ** 2 / (np.pi ** 2 * NU / max(sweep.COUETTE_PR))
    out = sweep.run_couette(L, cases, tol=1e-8, settle_steps=int(9 * t_slow), check_every=1000)
    assert out["converged"].all(), out["residual"]
    errs = []
    for i, c in enumerate(cases):
        u_an, T_an, heat = analytic(c, H)
        u, T = out["profiles_settled"][i]
        U = c["inputs"][2]
        eu = np.abs(u - u_an).max() / U
        eT = np.abs(T - T_an).max() / (heat / 4)   # relative to the peak viscous heating
        errs.append((eu, eT))
        assert eu < 2e-3, (i, eu)
        assert eT < 0.1, (i, eT)
    # from rest the velocity mode (decay time H^2 / (pi^2 nu), the same for every case)
    # sets the steps to 1e-8: several of its decay times
    t_u = (H - 1) ** 2 / (np.pi ** 2 * NU)
    assert (out["steps_to_tol"] > 2 * t_u).all() and (out["steps_to_tol"] < 12 * t_u).all(), out["steps_to_tol"]
