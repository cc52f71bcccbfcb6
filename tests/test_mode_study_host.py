"""Host-side pieces of the Prandtl-number mapping study (no GPU): the start-up series of
Eq. CouetteVelocityDimensionless, each mapping's predicted diffusivities, the decay fit."""
import numpy as np
import pytest

from paper_1611_02409_gb300 import mode_study as M


def test_startup_series_limits_and_heat_equation():
    eta = np.linspace(0, 1, 201)
    assert np.abs(M.startup_series(eta, 10.0) - eta).max() < 1e-12          # steady: linear
    assert np.abs(M.startup_series(eta[:150], 1e-9)).max() < 1e-3            # at rest away from the moving wall
    # solves u_t = nu u_yy: centred differences in time and space agree
    s, ds = 0.02, 1e-6
    e = np.linspace(0.1, 0.9, 9)
    ut = (M.startup_series(e, s + ds) - M.startup_series(e, s - ds)) / (2 * ds)
    h = 1e-4
    uyy = (M.startup_series(e + h, s) - 2 * M.startup_series(e, s) + M.startup_series(e - h, s)) / h ** 2
    assert np.allclose(ut, uyy, rtol=1e-4, atol=1e-6)


def test_predicted_prandtl_numbers():
    r = 1.2
    for tau in (0.51, 0.8, 2.0):
        nu, chi, pe = M.predicted("shifted", tau, 0.71, r)
        assert pe == pytest.approx(0.71) and nu == pytest.approx((tau - 0.5) / r ** 2)
        nu, chi, pe = M.predicted("literal", tau, 0.71, r)
        assert chi == pytest.approx((tau / 0.71 - 0.5) / r ** 2)
        assert pe == pytest.approx((tau - 0.5) / (tau / 0.71 - 0.5))
    assert M.predicted("literal", 0.528655, M.PAPER_PR, r)[2] == pytest.approx(0.1194, abs=1e-3)


def test_fit_rate_skips_transient_and_tail():
    ts = np.arange(0, 1601, 25)
    a = np.exp(-0.003 * ts)
    a[0] *= 1.1                                         # initial transient, excluded
    a[ts * 0.003 > 2.5] += 1e-3                         # a slow remainder past e^-2.5, excluded
    assert M._fit_rate(ts, a, 0.003) == pytest.approx(0.003, rel=1e-9)
