"""The allocation-free totals entry point (lbm_field_totals_static) against the
handle's own FP64 diagnostics and against FP64 sums of the same fields on the host.

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


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_1611_02409_gb300 import build
    build.build()
    from paper_1611_02409_gb300 import lbm
    return torch, lbm


def host_totals(D, Nf, m):
    rho, u, T = (m[k].double().cpu().numpy() for k in ("rho", "u", "T"))
    u2 = (u ** 2).sum(axis=0)
    mom = [(rho * u[a]).sum() for a in range(D)] + [0.0] * (3 - D)
    return np.array([rho.sum(), *mom, (rho * (0.5 * u2 + 0.5 * (D + Nf) * T)).sum()])


def totals(torch, lbm, D, Nf, m, stream):
    out = torch.full((6,), float("nan"), dtype=torch.float64, device="cuda")
    lbm.lbm_field_totals_static(D, Nf, m["rho"], m["u"], m["T"], out, stream)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def check_against(got, ref, host, D):
    # diagnostics sum the per-cell FP32 values in FP64: 1e-6 relative; the host sums of
    # the very same FP64 fields differ only by the order of the additions
    assert got[0] == pytest.approx(ref["mass"], rel=1e-6)
    assert got[4] == pytest.approx(ref["energy"], rel=1e-6)
    assert np.abs(got[1:1 + D] - ref["momentum"][:D]).max() < 1e-6 * ref["mass"]
    assert np.abs(got[:5] - host).max() <= 1e-11 * np.abs(host).max()
    assert got[5] == 0.0


def test_field_totals_static_matches_diagnostics_twice(env):
    torch, lbm = env
    params = dict(Pr=0.71, gamma=1.4, kappa=0.2, tau=0.528655)
    sim = lbm.Simulation(nx=160, ny=96, **params)
    sim.init(*inputs.taylor_green_2d(160, ny=96, U0=0.05, T_amp=0.02))
    for _ in range(2):  # two calls in a row, the second on an advanced state
        sim.step(25)
        ref = sim.diagnostics()
        m = sim.moments(device=True)
        got = totals(torch, lbm, 2, sim.coeffs["Nf"], m, sim.stream)
        check_against(got, ref, host_totals(2, sim.coeffs["Nf"], m), 2)
        assert got[3] == 0.0
    sim.close()


def test_field_totals_static_many_blocks_ragged(env):
    # 520 x 512 = 266,240 cells: 16 full blocks of 16,384 cells and a ragged 17th, so the
    # fixed-order final sum runs over several scratch rows
    torch, lbm = env
    sim = lbm.Simulation(nx=520, ny=512, Pr=0.71, gamma=1.4, kappa=0.2, tau=0.6)
    sim.init(*inputs.taylor_green_2d(520, ny=512, U0=0.05, T_amp=0.02, noise=1e-3, seed=5))
    sim.step(10)
    ref = sim.diagnostics()
    m = sim.moments(device=True)
    got = totals(torch, lbm, 2, sim.coeffs["Nf"], m, sim.stream)
    check_against(got, ref, host_totals(2, sim.coeffs["Nf"], m), 2)
    # a smaller call after the larger one: rows of the earlier call stay in the scratch
    # but are not part of this sum
    small = {k: v[..., :64, :].contiguous() for k, v in m.items()}
    got2 = totals(torch, lbm, 2, sim.coeffs["Nf"], small, sim.stream)
    h2 = host_totals(2, sim.coeffs["Nf"], small)
    assert np.abs(got2[:5] - h2).max() <= 1e-11 * np.abs(h2).max()
    sim.close()


def test_field_totals_static_3d(env):
    # 48^3 = 110,592 cells of a D3Q103 handle: momentum z and D = 3 in the energy
    torch, lbm = env
    sim = lbm.Simulation(lattice=lbm.LBM_D3Q103, nx=48, ny=48, nz=48, Pr=0.71, gamma=1.4, kappa=0.2, tau=0.6)
    sim.init(*inputs.taylor_green_3d(48, U0=0.05, T_amp=0.02, noise=1e-3, seed=6))
    sim.step(5)
    ref = sim.diagnostics()
    m = sim.moments(device=True)
    got = totals(torch, lbm, 3, sim.coeffs["Nf"], m, sim.stream)
    check_against(got, ref, host_totals(3, sim.coeffs["Nf"], m), 3)
    assert abs(got[3]) > 0.0
    sim.close()


def test_field_totals_static_counts_bad_cells(env):
    torch, lbm = env
    sim = lbm.Simulation(nx=200, ny=100, Pr=0.71, gamma=1.4, kappa=0.2, tau=0.6)
    sim.init(*inputs.taylor_green_2d(200, ny=100, U0=0.05, T_amp=0.02))
    m = sim.moments(device=True)
    Nf = sim.coeffs["Nf"]
    m["rho"][37, 11] = float("nan")
    assert totals(torch, lbm, 2, Nf, m, sim.stream)[5] == 1.0
    m["rho"][37, 11] = -0.5
    m["T"][99, 199] = 0.0
    assert totals(torch, lbm, 2, Nf, m, sim.stream)[5] == 2.0
    sim.close()
