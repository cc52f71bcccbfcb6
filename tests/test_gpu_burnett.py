"""D2Q77 with the sixth-order (Burnett) equilibrium of Sec. IV (reading R19) on the GPU.

* Cell-by-cell parity with the FP64 oracle after 1 and 9 steps, direct and two-pass
  kernels, FP32 and FP16 storage, periodic and open x ends, extents narrower than the
  stencil's reach (the modulo wrap) and ragged rows.  Tolerances as for D2Q37: FP32
  storage 2e-6 on the scaled deviations, FP16 a few storage roundings per step.
* The equilibrium itself at a strong state (u = (0.3, -0.2), T = 1.1, where the fifth- and
  sixth-order terms move the outer populations by several per cent): the initial
  populations against the oracle's G^(6) within 1.5e-6 of the scaled value (FP32
  evaluation of a degree-6 polynomial at |c| <= 5), and a fixed point of the collision.
* A thermal Taylor-Green field over 100 steps against the oracle (relative L2 of u, T).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1611_02409_gb300 import inputs

pytestmark = pytest.mark.gpu

PRM = dict(Pr=0.71, gamma=1.4, kappa=0.2, tau=0.8)
# BF16: about twice the measured element-wise error (1.6e-3 after one step)
TOL = {"fp32": 2e-6, "fp16": 2e-3, "bf16": 4e-3}


@pytest.fixture(scope="module")
def L():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_1611_02409_gb300 import build
    build.build()
    from paper_1611_02409_gb300 import lbm
    return lbm


def _index(sim, o):
    return [next(j for j in range(len(o.c)) if tuple(o.c[j]) == tuple(v)) for v in sim.c]


@pytest.mark.parametrize("storage", ["fp32", "fp16", "bf16"])
@pytest.mark.parametrize("kernel", [1, 4])            # direct, two-pass
@pytest.mark.parametrize("nx,ny,open_x", [(37, 23, False), (130, 9, True), (4, 6, False), (11, 3, True),
                                          (5, 5, False)])
def test_d2q77_elementwise(L, storage, kernel, nx, ny, open_x):
    fields = inputs.random_fields((ny, nx), seed=3 * nx + ny, drho=0.01, du=0.02, dT=0.02)
    sim = L.Simulation(lattice=L.LBM_D2Q77, nx=nx, ny=ny, storage=storage, kernel=kernel,
                       bc_x=L.LBM_OPEN if open_x else L.LBM_PERIODIC, **PRM)
    sim.init(*fields)
    o = O.Sim(O.D2Q77, nx=nx, ny=ny, open_x=open_x, **PRM)
    o.init(*fields)
    assert len(sim.c) == 77 and np.abs(sim.c).max() == 5
    idx = _index(sim, o)
    w = sim.w[:, None, None]
    for steps in (1, 9):
        sim.step(steps)
        o.step(steps)
        gg, hg = sim.populations()
        go, ho = o.populations()
        eg, eh = np.abs((gg - go[idx]) / w).max(), np.abs((hg - ho[idx]) / w).max()
        assert eg < TOL[storage] and eh < 3 * TOL[storage], (steps, eg, eh)
    sim.close()
    o.close()


def test_d2q77_sixth_order_equilibrium_at_strong_state(L):
    rho, u, T = 1.05, np.array([0.3, -0.2]), 1.1
    n = 8
    sim = L.Simulation(lattice=L.LBM_D2Q77, nx=n, ny=n, **PRM)
    sim.init(np.full((n, n), rho), u[:, None, None] * np.ones((2, n, n)), np.full((n, n), T))
    g, h = sim.populations()
    o = O.Sim(O.D2Q77, nx=4, ny=4, **PRM)
    idx = _index(sim, o)
    o.close()
    # compared as G_i / w_i = rho P(xi_i), each side with its own weights: the two FP64
    # derivations of the 2e-7 smallest weights differ by ~3e-7 relative (1e-13 absolute)
    wo = O.lattice(O.D2Q77)[3][idx]
    P6 = O.equilibrium(O.D2Q77, rho, u, T * np.eye(2), order=6)[idx] / wo
    P4 = O.equilibrium(O.D2Q77, rho, u, T * np.eye(2), order=4)[idx] / wo
    w = sim.w
    assert np.abs(P6 - P4).max() > 1e-2                     # the terms under test are not small
    # FP32 evaluation of the degree-6 polynomial at |c| up to 5 (monomials up to 5^6 that
    # largely cancel): ~1e-6 of the scaled value (up to 22 here, 36 for h), four orders
    # below the fifth- and sixth-order terms checked above
    rel = lambda x, ref: np.abs(x / w - ref) / (1 + np.abs(ref))
    assert rel(g[:, 0, 0], P6).max() < 1.5e-6
    assert np.abs(g - g[:, :1, :1]).max() == 0.0            # uniform
    Nf = 2 / (1.4 - 1) - 2
    assert rel(h[:, 0, 0], 0.5 * Nf * T * P6).max() < 1.5e-6
    # the equilibrium is a fixed point of the collision (and of streaming, the state being uniform)
    sim.step(3)
    g3, h3 = sim.populations()
    s0, s3 = g / w[:, None, None], g3 / w[:, None, None]
    assert (np.abs(s3 - s0) / (1 + np.abs(s0))).max() < 1.5e-6
    sim.close()


@pytest.mark.parametrize("storage,tol", [("fp32", 1e-5), ("fp16", 2e-3)])
def test_d2q77_taylor_green_100_steps(L, storage, tol):
    n = 48
    fields = inputs.taylor_green_2d(n, U0=0.05, T_amp=0.02)
    sim = L.Simulation(lattice=L.LBM_D2Q77, nx=n, ny=n, storage=storage, **PRM)
    sim.init(*fields)
    sim.step(100)
    m = sim.moments()
    sim.close()
    o = O.Sim(O.D2Q77, nx=n, ny=n, **PRM)
    o.init(*fields)
    o.step(100)
    mo = o.moments()
    o.close()
    du = np.linalg.norm(m["u"] - mo["u"]) / np.linalg.norm(mo["u"])
    dT = np.linalg.norm(m["T"] - mo["T"]) / np.linalg.norm(mo["T"] - 1)
    assert du < tol and dT < 10 * tol, (du, dT)


def _moving_thermal_rate_gpu(L, lattice, U, amp=1e-2, n=32, steps=300, every=30):
    # isobaric thermal wave carried by a uniform flow u_x = U (as the oracle's pin, at a
    # larger amplitude): the decay rate of its Fourier amplitude
    sim = L.Simulation(lattice=lattice, nx=n, ny=4, **PRM)
    x = np.arange(n)[None, :] * np.ones((4, 1))
    T = 1 + amp * np.sin(2 * np.pi * x / n)
    sim.init(1 / T, np.stack([U * np.ones((4, n)), np.zeros((4, n))]), T)
    ts, amps = [], []
    for t in range(0, steps + 1, every):
        if t:
            sim.step(every)
        m = sim.moments()
        ts.append(t)
        amps.append(2 * abs(np.mean((m["T"] - m["T"].mean()) * np.exp(-2j * np.pi * x / n))))
    sim.close()
    return -np.polyfit(ts[1:], np.log(amps[1:]), 1)[0]


def test_d2q77_galilean_invariance(L):
    # The sixth-order equilibrium keeps the thermal diffusivity of a wave carried at Mach
    # 0.42 at its rest value; the fourth-order one on D2Q37 moves it by 2.4e-4 (oracle:
    # 2e-6 against 2.3e-4).  In FP32 the temperature of the moving wave is the difference
    # of second moments ~1.1 and rho u^2 = 0.25, which resolves a 1e-3 wave to ~1e-4 per
    # step: the wave here is 1e-2 (measured: 3.7e-5 on D2Q77, 2.43e-4 on D2Q37).
    d77 = abs(_moving_thermal_rate_gpu(L, L.LBM_D2Q77, 0.5) / _moving_thermal_rate_gpu(L, L.LBM_D2Q77, 0.0) - 1)
    d37 = abs(_moving_thermal_rate_gpu(L, L.LBM_D2Q37, 0.5) / _moving_thermal_rate_gpu(L, L.LBM_D2Q37, 0.0) - 1)
    assert d77 < 1e-4 and d37 > 1.5e-4 and d37 > 3 * d77, (d77, d37)
