"""The warm start's converged state against the FP64 oracle (the final-field gate of the
learned warm start: error <= 1e-6).

Six held-out thermal Couette channels (tests/golden/couette_steady_oracle.txt: heights 33
to 65, parameters drawn from the training sweep's distribution) were settled by the FP64
oracle alone to within 1e-11 of their steady state.  Here each is run on the GPU with
FP64 storage twice, from rest and from a surrogate prediction, until the per-step change
times the slowest decay time bounds the distance to the steady state by 1e-8; both final
states must match the oracle's within 1e-6 (relative L2 per field: rho, u as a vector
field, T).  FP64 storage is what makes this possible: the FP32 iteration comes to rest at
fixed points that wander by a few 1e-6 of u with the path taken to them."""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
from make_couette_steady import load  # noqa: E402

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


def field_errors(f, prof):
    """Relative L2 errors of GPU fields [ny, nx] against oracle profiles [ny] (the steady
    channel is uniform in x)."""
    col = lambda v: np.repeat(v[:, None], f["rho"].shape[1], axis=1)
    rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
    uo = np.stack([col(prof[:, 1]), col(prof[:, 2])])
    return dict(rho=rel(f["rho"], col(prof[:, 0])), u=rel(f["u"], uo), T=rel(f["T"], col(prof[:, 3])))


def test_warm_and_rest_starts_reach_the_oracle_steady_state(L):
    from paper_1611_02409_gb300 import surrogate as S
    from paper_1611_02409_gb300 import sweep
    gold = load()
    cases = [sweep.channel_case(c["Pr"], c["gamma"], c["Ma"], c["tau"], c["dT"], c["H"]) for c, _ in gold]
    for (c, _), case in zip(gold, cases):
        assert case["params"]["wall_u"][1][0] == c["U"]          # same set-up as the oracle's
    # a small surrogate trained on FP32 channels of the same distribution (other draws)
    ts = S.training_set(L, n=48, seed=11, H_range=(33, 65), tol=1e-8, max_steps=400000, check_every=100)
    sur = S.Surrogate(L, seed=0, max_batch=64, sizes=[5, 256, 256, 4 * S.NPTS])
    sur.fit(ts["X"], ts["Y"], iters=1500, lr=2e-3, log_every=500)
    pred = sur.predict(np.array([c["inputs"] for c in cases]))
    res = S.gate_study(L, cases, pred, bound=1e-8)
    worst = {}
    for (c, prof), r in zip(gold, res):
        for start in ("rest", "warm"):
            assert r[start]["distance_bound"] <= 1e-8
            e = field_errors(r[start]["fields"], prof)
            worst[(c["H"], start)] = max(e.values())
            assert max(e.values()) <= 1e-6, (c["H"], start, e)
    steps = {s: np.array([r[s]["steps"] for r in res]) for s in ("rest", "warm")}
    assert np.median(steps["warm"]) < np.median(steps["rest"]), (steps, worst)
