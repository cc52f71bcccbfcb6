"""The allocation-free totals entry point (lbm_field_totals_static) against the
handle's own FP64 diagnostics.

Callers that cannot call cudaMalloc (device memory reserved up front by a host
framework, or a loop that must not risk an allocation's device synchronisation) get
conservation totals of fields they already hold, reduced through a fixed scratch array
inside the library.  This file is collected last so that a failure here comes after
every other test has run; it must pass alone in a fresh process too.
"""
import numpy as np
import pytest

from paper_1611_02409_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_field_totals_static_matches_diagnostics_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_1611_02409_gb300 import build
    build.build()
    from paper_1611_02409_gb300 import lbm
    params = dict(Pr=0.71, gamma=1.4, kappa=0.2, tau=0.528655)
    sim = lbm.Simulation(nx=160, ny=96, **params)
    sim.init(*inputs.taylor_green_2d(160, ny=96, U0=0.05, T_amp=0.02))
    for _ in range(2):  # two calls in a row, the second on an advanced state
        sim.step(25)
        ref = sim.diagnostics()
        m = sim.moments(device=True)
        out = torch.full((6,), float("nan"), dtype=torch.float64, device="cuda")
        lbm.lbm_field_totals_static(2, sim.coeffs["Nf"], m["rho"], m["u"], m["T"], out, sim.stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        # same tolerance as the diagnostics test: 1e-6 relative (per-cell FP32 values summed in FP64)
        assert got[0] == pytest.approx(ref["mass"], rel=1e-6)
        assert got[4] == pytest.approx(ref["energy"], rel=1e-6)
        assert np.abs(got[1:3] - ref["momentum"][:2]).max() < 1e-6 * ref["mass"]
        assert got[3] == 0.0 and got[5] == 0.0
    sim.close()
