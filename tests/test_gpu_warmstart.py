"""Warm start: the non-equilibrium initialisation reproduces the stress and heat flux
it is given, and a surrogate-initialised channel reaches the converged state of the
plain scheme from rest in fewer steps."""
import numpy as np
import pytest

from paper_1611_02409_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_1611_02409_gb300 import build
    build.build()
    from paper_1611_02409_gb300 import lbm
    return lbm


def test_init_neq_reproduces_stress_and_heat_flux(L):
    rng = np.random.default_rng(4)
    n = 12
    sim = L.Simulation(nx=n, ny=n, Pr=0.71, gamma=1.4, kappa=0.2, tau=0.8)
    rho = 1.0 + 0.02 * rng.uniform(-1, 1, (n, n))
    T = 1.0 + 0.02 * rng.uniform(-1, 1, (n, n))
    u = np.zeros((2, n, n))
    dev = 1e-3 * rng.uniform(-1, 1, (2, n, n))
    Pi = np.stack([rho * T + dev[0], 1e-3 * rng.uniform(-1, 1, (n, n)), rho * T - dev[0]])
    q = 1e-3 * rng.uniform(-1, 1, (2, n, n))
    L.lbm_init_fields_neq(sim.h, rho, u, T, Pi, q)
    m = sim.moments()
    assert np.abs(m["rho"] - rho).max() < 1e-6 and np.abs(m["T"] - T).max() < 1e-6
    assert np.abs(m["Pi"] - Pi).max() < 1e-6
    assert np.abs(m["q"] - q).max() < 1e-6
    sim.close()


def test_surrogate_warm_start_saves_steps(L):
    # Steps to residual 1e-8 (per-step relative change of u_x and T) from rest and from
    # the surrogate; then both are run well past convergence and must end in the same
    # steady state.  In FP32 the per-step change of these channels bottoms out at
    # 0.5-2e-9 (measured every 200 steps up to 12000 steps from rest), so a 1e-9 stop is
    # reached at random times once the fields have settled; 1e-8 lies above that floor.
    # The FP32 dynamics come to rest at fixed points that depend on the path by some
    # tens of ulps of the stored deviations (measured 1-3e-6 relative on u for these
    # channels), so the bar is 1e-5.
    from paper_1611_02409_gb300 import surrogate as S
    from paper_1611_02409_gb300 import sweep
    ts = S.training_set(L, n=24, seed=3, H_range=(13, 21), tol=1e-8, max_steps=400000, check_every=100)
    assert ts["converged"].all()
    sur = S.Surrogate(L, seed=0, max_batch=64, sizes=[5, 128, 128, 4 * S.NPTS])
    losses = sur.fit(ts["X"], ts["Y"], iters=800, lr=2e-3, log_every=200)
    assert losses[-1][1] < 0.2 * losses[0][1]
    test = S.draw_channels(6, seed=77, H=17)
    pred = sur.predict(np.array([c["inputs"] for c in test]))
    tol = 1e-8
    rest, _, br = S.run_channels(L, test, lambda i, bt: bt.init(i, *sweep.initial_fields(test[i])), tol, 400000,
                                 100)
    warm, _, bw = S.run_channels(L, test, lambda i, bt: bt.init_neq(i, *S.warm_fields(test[i], pred[i])), tol,
                                 400000, 100)
    assert rest["converged"].all() and warm["converged"].all()
    assert np.median(warm["steps"]) < 0.8 * np.median(rest["steps"]), (warm["steps"], rest["steps"])
    # continue both batches (lbm_batch_activate) well past convergence: tol 0 never stops
    n_long = int(2 * max(rest["steps"]))
    r2, fr = S.continue_channels(br, len(test), 0.0, n_long, 100)
    w2, fw = S.continue_channels(bw, len(test), 0.0, n_long, 100)
    br.close()
    bw.close()
    assert (r2["steps"] - rest["steps"] >= n_long).all() and (w2["steps"] - warm["steps"] >= n_long).all()
    for i in range(len(test)):
        for k in ("u", "T"):
            assert np.linalg.norm(fw[i][k] - fr[i][k]) <= 1e-5 * np.linalg.norm(fr[i][k]), (i, k)
