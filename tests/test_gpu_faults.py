"""Failure detection on the GPU, without faulting, trapping or hanging it.

* A NaN written into one population (through lbm_set_populations) is reported by the
  FP64 diagnostics as LBM_ERR_UNSTABLE, and the handle keeps working after re-init.
* A wait that nothing will satisfy (lbm_debug_inject_stall: the staged kernel announces
  its copies but issues none) runs out after its short limit; the next synchronising call
  returns LBM_ERR_TIMEOUT, and the same handle then steps correctly again.
* In a batch, an instance whose state turns NaN is deactivated at its residual check,
  and the other instances keep stepping.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1611_02409_gb300 import inputs

pytestmark = pytest.mark.gpu

CFG0 = dict(Pr=0.71, gamma=1.4, kappa=0.2, tau=0.528655)


@pytest.fixture(scope="module")
def L():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_1611_02409_gb300 import build
    build.build()
    from paper_1611_02409_gb300 import lbm
    return lbm


def test_nan_population_is_reported_unstable(L):
    fields = inputs.taylor_green_2d(32, ny=16)
    sim = L.Simulation(nx=32, ny=16, **CFG0)
    sim.init(*fields)
    g, h = sim.populations()
    g[5, 3, 7] = np.nan
    sim.set_populations(g, h)
    sim.step(3)
    d = L.lbm_diagnostics(sim.h, check=False)
    assert d["code"] == L.LBM_ERR_UNSTABLE and d["bad"] > 0, d
    sim.init(*fields)
    sim.step(3)
    d = sim.diagnostics()
    assert d["bad"] == 0
    sim.close()


def test_stalled_waits_time_out_and_the_handle_recovers(L):
    n, ny = 256, 12
    fields = inputs.taylor_green_2d(n, ny=ny)
    sim = L.Simulation(nx=n, ny=ny, kernel=L.LBM_KERNEL_STAGED, **CFG0)
    sim.init(*fields)
    L._check(L.lib().lbm_debug_inject_stall(sim.h, 1))
    sim.step(2)
    d = L.lbm_diagnostics(sim.h, check=False)
    assert d["code"] == L.LBM_ERR_TIMEOUT, d
    L._check(L.lib().lbm_debug_inject_stall(sim.h, 0))
    sim.init(*fields)
    sim.step(20)
    m = sim.moments()
    sim.close()
    o = O.Sim(O.D2Q37, nx=n, ny=ny, **CFG0)
    o.init(*fields)
    o.step(20)
    mo = o.moments()
    for k in ("rho", "u", "T"):
        assert np.linalg.norm(m[k] - mo[k]) <= 1e-5 * np.linalg.norm(mo[k]), k


def test_batch_deactivates_a_diverged_instance(L):
    params = [dict(nx=n, ny=n, **CFG0) for n in (32, 48, 40)]
    bt = L.Batch(params)
    for i, p in enumerate(params):
        rho, u, T = inputs.taylor_green_2d(p["nx"])
        if i == 1:
            rho = rho.copy()
            rho[4, 5] = np.nan
        bt.init(i, rho, u, T)
    done = bt.run(300, tol=0.0, check_every=100)
    steps, res, act = bt.status()
    bt.close()
    assert done == 300
    # the first check (step 100) already sees the NaN sums
    assert act[1] == 0 and np.isnan(res[1]) and steps[1] == 100
    assert act[0] == 1 and act[2] == 1 and steps[0] == 300 and steps[2] == 300
    assert np.isfinite(res[0]) and np.isfinite(res[2])
