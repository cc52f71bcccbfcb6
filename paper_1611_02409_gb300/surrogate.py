"""Learned warm start of thermal Couette channels.

A multilayer perceptron (5 -> 4 x 512 -> 4 x 256, GELU, bfloat16 products with FP32
accumulation, trained on the GPU by the library's own kernels, lbm_mlp_*) maps the
channel parameters (Pr, gamma, wall Mach number, tau, wall temperature difference) to
the steady profiles of u_x, T, Pi_xy and q_y at 256 points of y/H.  Pi_xy and q_y are
learned times (ny - 1), since in steady Couette flow they scale as 1/H.  The training
profiles are steady channels the scheme itself computes (one batch, run to residual
`tol`).  A prediction initialises a channel with its equilibrium plus the predicted
non-equilibrium stress and heat flux (lbm_batch_init_fields_neq).  The plain scheme
from rest remains the reference for the converged state.

    python -m paper_1611_02409_gb300.surrogate --out study.json
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import sweep

NPTS = 256
SIZES = [5, 512, 512, 512, 512, 4 * NPTS]
X_LO = np.array([0.5, 1.1, 0.01, 0.6, -0.05])
X_HI = np.array([2.0, 1.67, 0.1, 1.0, 0.05])


def draw_channels(n, seed, H=None, H_range=(64, 512)):
    """n channel cases with the sweep's parameter distribution; fixed height H if given."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(n):
        x = rng.uniform(X_LO, X_HI)
        h = H if H is not None else int(rng.integers(H_range[0], H_range[1] + 1))
        out.append(sweep.channel_case(*x, h))
    return out


def glorot(sizes, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    params = []
    for k, n in zip(sizes[:-1], sizes[1:]):
        a = np.sqrt(6.0 / (k + n))
        params.append([rng.uniform(-a, a, size=(k, n)), np.zeros(n)])
    return params


class Surrogate:
    """The profile network plus its input/output normalisation."""

    def __init__(self, lbm, seed=0, max_batch=512, sizes=SIZES):
        import torch
        self.torch = torch
        self.sizes = list(sizes)
        self.net = lbm.MLP(self.sizes, max_batch=max_batch)
        self.net.set_params(glorot(self.sizes, seed))
        self.y_mean = None
        self.y_std = None

    def _x(self, X):
        return self.torch.tensor(2.0 * (X - X_LO) / (X_HI - X_LO) - 1.0, dtype=self.torch.float32, device="cuda")

    def fit(self, X, Y, iters=3000, lr=1e-3, log_every=500):
        """X [n, 5] channel inputs, Y [n, 4, NPTS] profiles; full-batch Adam."""
        t = self.torch
        Yf = Y.reshape(len(Y), -1)
        self.y_mean = Yf.mean(0)
        self.y_std = np.maximum(Yf.std(0), 1e-6 * max(Yf.std(0).max(), 1e-30))
        xt = self._x(X)
        yt = t.tensor((Yf - self.y_mean) / self.y_std, dtype=t.float32, device="cuda")
        losses = []
        for it in range(iters):
            self.net.forward(xt)
            want = it % log_every == 0 or it == iters - 1
            loss = self.net.backward(yt, want_loss=want)
            if want:
                losses.append((it, loss))
            step_lr = lr if it < 0.7 * iters else lr * 0.2
            self.net.adam(lr=step_lr)
        return losses

    def predict(self, X):
        y = self.net.forward(self._x(X)).cpu().numpy().astype(np.float64)
        return (y * self.y_std + self.y_mean).reshape(len(X), 4, -1)


def training_set(lbm, n=256, seed=0, H_range=(64, 128), tol=1e-8, max_steps=2_000_000, check_every=200):
    """Steady channel profiles computed by the scheme in one batch."""
    cases = draw_channels(n, seed, H_range=H_range)
    status, prof, xin, conv, secs = sweep.run_sweep(lbm, cases, max_steps=max_steps, tol=tol,
                                                    check_every=check_every, autotune=False)
    return dict(X=xin, Y=prof, converged=conv, seconds=secs, batch_steps=status["batch_steps"],
                steps=status["steps"])


def warm_fields(case, prof):
    """(rho, u, T, Pi, q) of a channel from predicted profiles (u_x, T, Pi_xy (ny-1), q_y (ny-1))."""
    p = case["params"]
    nx, ny = p["nx"], p["ny"]
    yq = np.linspace(0.0, 1.0, prof.shape[1])
    y = np.arange(ny) / (ny - 1)
    ux = np.interp(y, yq, prof[0])
    T = np.interp(y, yq, prof[1])
    Pxy = np.interp(y, yq, prof[2]) / (ny - 1)
    qy = np.interp(y, yq, prof[3]) / (ny - 1)
    T = np.maximum(T, 0.5)
    # uniform pressure; the fluid rows (1..ny-2) carry the rest state's mass, the invariant
    # that (with the walls) selects the steady state
    rho = (1.0 / T) * (ny - 2) / np.sum(1.0 / T[1:-1])
    col = lambda v: np.repeat(v[:, None], nx, axis=1)
    R, Tt = col(rho), col(T)
    u = np.stack([col(ux), np.zeros((ny, nx))])
    Pi = np.stack([R * Tt, col(Pxy), R * Tt])
    q = np.stack([np.zeros((ny, nx)), col(qy)])
    return R, u, Tt, Pi, q


def _finish(bt, t0, done, n):
    secs = time.perf_counter() - t0
    steps, res, act = bt.status()
    fields = [bt.moments(i) for i in range(n)]
    return dict(steps=steps.copy(), residual=res, converged=act == 0, seconds=secs, batch_steps=done), fields


def run_channels(lbm, cases, init, tol, max_steps, check_every):
    """Runs the cases in one batch from `init(i, batch)` to residual `tol`; returns the
    per-instance result, the fields, and the still open batch."""
    bt = lbm.Batch([c["params"] for c in cases])
    for i in range(len(cases)):
        init(i, bt)
    t0 = time.perf_counter()
    done = bt.run(max_steps, tol=tol, check_every=check_every)
    res, fields = _finish(bt, t0, done, len(cases))
    return res, fields, bt


def continue_channels(bt, n, tol, max_steps, check_every):
    """Continues every instance of an open batch to the tighter residual `tol`."""
    bt.activate()
    t0 = time.perf_counter()
    done = bt.run(max_steps, tol=tol, check_every=check_every)
    return _finish(bt, t0, done, n)


def state_diff(fa, fb, idx):
    """Relative L2 differences of u and T between two sets of converged fields."""
    rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
    du = np.array([rel(fa[i]["u"], fb[i]["u"]) for i in idx])
    dT = np.array([rel(fa[i]["T"], fb[i]["T"]) for i in idx])
    return du, dT


def channel_tau_slow(case, r):
    """Slowest decay time, in steps, of a thermal Couette channel 4 x H near its steady
    state: the lowest shear mode decays in (H-1)^2 / (pi^2 nu) steps, the lowest thermal
    mode in Pr times that (chi = nu / Pr under the shifted mapping), with the lattice
    viscosity nu = (tau - 1/2) / r^2 at T = 1."""
    p = case["params"]
    nu = (p["tau"] - 0.5) / r ** 2
    return (p["ny"] - 1) ** 2 * max(1.0, p["Pr"]) / (np.pi ** 2 * nu)


def run_to_steady(sim, tau_slow, bound=1e-8, chunk=200, max_steps=5_000_000):
    """Steps one handle until its distance to the steady state is bounded by `bound`
    (relative, u_x and T).  Near a steady state the fields approach it as exp(-n / tau)
    with tau the slowest decay time, so the per-step change r (lbm_diagnostics' residual,
    taken over `chunk` steps) and the distance d satisfy d <= r tau; tau is the larger of
    tau_slow and the decay time measured from successive residuals.  Returns (steps,
    residual, distance bound)."""
    sim.diagnostics()
    steps, prev, res = 0, None, float("inf")
    while steps < max_steps:
        sim.step(chunk)
        steps += chunk
        res = sim.diagnostics()["residual"]
        tau_est = chunk / np.log(prev / res) if prev and 0.0 < res < prev else 0.0
        dist = res * max(tau_slow, tau_est)
        if steps >= 2 * chunk and dist <= bound:
            return steps, res, dist
        prev = res
    return steps, res, res * tau_slow


def gate_study(lbm, cases, pred, bound=1e-8, storage="fp64", chunk=200, max_decay_times=60):
    """Rest start and warm start (from the predicted profiles `pred`) of each channel on
    its own handle, each run to a distance `bound` from the steady state (or at most
    `max_decay_times` slowest decay times): steps, wall time and the final fields (rho, u,
    T) of both."""
    out = []
    for case, pr in zip(cases, pred):
        p = case["params"]
        row = {}
        for start in ("rest", "warm"):
            sim = lbm.Simulation(storage=storage, **p)
            if start == "rest":
                sim.init(*sweep.initial_fields(case))
            else:
                lbm.lbm_init_fields_neq(sim.h, *warm_fields(case, pr))
            tau_slow = channel_tau_slow(case, sim.r)
            t0 = time.perf_counter()
            steps, res, dist = run_to_steady(sim, tau_slow, bound, chunk, int(max_decay_times * tau_slow))
            secs = time.perf_counter() - t0
            m = sim.moments()
            sim.close()
            row[start] = dict(steps=steps, seconds=secs, residual=res, distance_bound=dist,
                              fields={k: m[k] for k in ("rho", "u", "T")})
        out.append(row)
    return out


def _summary(v):
    return dict(median=float(np.median(v)), p90=float(np.percentile(v, 90)), max=float(np.max(v))) if len(v) else None


def study(lbm, n_train=256, n_test=256, H=256, seed=0, tol=1e-8, tol_fine=1e-9, max_steps=6_000_000,
          check_every=200, train_H=(64, 128), iters=3000, refine=True, keep_model=False):
    """Trains on steady channels, then compares warm start and rest start on held-out
    4 x H channels: steps and batch wall time to residual `tol`, and the difference of
    the two converged states at `tol` and after both continue to `tol_fine`.  The
    residual is a per-step relative change, so a run that stops at it is still about
    tol x (slowest decay time) away from the steady state, from its own side; the
    difference must shrink with the tolerance if both reach the same state.  With
    keep_model the trained Surrogate is returned as res["model"]."""
    t0 = time.perf_counter()
    ts = training_set(lbm, n_train, seed, H_range=train_H, tol=tol)
    sur = Surrogate(lbm, seed=seed)
    losses = sur.fit(ts["X"], ts["Y"], iters=iters)
    t_train = time.perf_counter() - t0
    test = draw_channels(n_test, seed + 1000, H=H)
    X = np.array([c["inputs"] for c in test])
    t0 = time.perf_counter()
    pred = sur.predict(X)
    t_pred = time.perf_counter() - t0
    rest, f_rest, b_rest = run_channels(lbm, test, lambda i, bt: bt.init(i, *sweep.initial_fields(test[i])), tol,
                                        max_steps, check_every)
    warm, f_warm, b_warm = run_channels(lbm, test, lambda i, bt: bt.init_neq(i, *warm_fields(test[i], pred[i])),
                                        tol, max_steps, check_every)
    both = np.nonzero(rest["converged"] & warm["converged"])[0]
    du8, dT8 = state_diff(f_warm, f_rest, both)
    if not refine:   # steps and wall time to tol only
        b_rest.close()
        b_warm.close()
        rest9, f_rest9, warm9, f_warm9 = rest, f_rest, warm, f_warm
    else:
        rest9, f_rest9 = continue_channels(b_rest, n_test, tol_fine, max_steps, check_every)
        warm9, f_warm9 = continue_channels(b_warm, n_test, tol_fine, max_steps, check_every)
        b_rest.close()
        b_warm.close()
    both9 = np.nonzero(rest9["converged"] & warm9["converged"])[0]
    du9, dT9 = state_diff(f_warm9, f_rest9, both9)
    # how far each tol-state still was from the tol_fine state of the same run
    dr8, _ = state_diff(f_rest, f_rest9, both9)
    perr = []
    for i in range(n_test):
        ref = sweep.profiles(f_rest9[i])
        perr.append(np.linalg.norm(pred[i][0] - ref[0]) / max(np.linalg.norm(ref[0]), 1e-30))
    sr, sw = rest["steps"][both], warm["steps"][both]
    arrays = dict(X=X, steps_rest=rest["steps"], steps_warm=warm["steps"], steps_rest_fine=rest9["steps"],
                  steps_warm_fine=warm9["steps"], du_tol=du8, dT_tol=dT8, du_fine=du9, dT_fine=dT9)
    return dict(
        train=dict(n=n_train, H_range=list(train_H), converged=int(ts["converged"].sum()),
                   sweep_seconds=ts["seconds"], batch_steps=ts["batch_steps"], losses=losses,
                   seconds_total=t_train),
        test=dict(n=n_test, H=H, tol=tol, tol_fine=tol_fine, both_converged=int(len(both)),
                  rest_converged=int(rest["converged"].sum()), warm_converged=int(warm["converged"].sum()),
                  predict_seconds=t_pred,
                  steps_rest_median=float(np.median(sr)) if len(sr) else None,
                  steps_warm_median=float(np.median(sw)) if len(sw) else None,
                  steps_rest_mean=float(np.mean(sr)) if len(sr) else None,
                  steps_warm_mean=float(np.mean(sw)) if len(sw) else None,
                  step_ratio_median=float(np.median(sw / sr)) if len(sr) else None,
                  batch_seconds_rest=rest["seconds"], batch_seconds_warm=warm["seconds"],
                  batch_steps_rest=rest["batch_steps"], batch_steps_warm=warm["batch_steps"],
                  state_diff_at_tol=dict(u=_summary(du8), T=_summary(dT8)),
                  refined=bool(refine), both_converged_fine=int(len(both9)),
                  extra_steps_fine_median=dict(rest=float(np.median(rest9["steps"] - rest["steps"])),
                                               warm=float(np.median(warm9["steps"] - warm["steps"]))),
                  state_diff_at_tol_fine=dict(u=_summary(du9), T=_summary(dT9)),
                  rest_tol_state_vs_fine_u=_summary(dr8),
                  initial_u_profile_err_median=float(np.median(perr))),
        **({"model": sur} if keep_model else {})), arrays


def time_training(lbm, batch=256, iters=50, sizes=SIZES, seed=0):
    """Milliseconds per training iteration (forward, backward with the loss, Adam) of the
    network on random data, for each matrix-product form (tcgen05, mma.sync)."""
    import torch
    rng = np.random.Generator(np.random.PCG64(seed))
    x = torch.tensor(rng.uniform(-1, 1, (batch, sizes[0])), dtype=torch.float32, device="cuda")
    y = torch.tensor(rng.normal(size=(batch, sizes[-1])), dtype=torch.float32, device="cuda")
    out = {}
    for name, kind in (("tcgen05", lbm.LBM_MLP_GEMM_TCGEN05), ("mma_sync", lbm.LBM_MLP_GEMM_MMA_SYNC)):
        net = lbm.MLP(sizes, max_batch=batch, gemm=kind)
        net.set_params(glorot(sizes, seed))
        for _ in range(3):
            net.forward(x)
            net.backward(y, want_loss=False)
            net.adam(lr=1e-3)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(net.stream)
        for _ in range(iters):
            net.forward(x)
            net.backward(y, want_loss=False)
            net.adam(lr=1e-3)
        e1.record(net.stream)
        torch.cuda.synchronize()
        out[name] = e0.elapsed_time(e1) / iters
        net.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n-train", type=int, default=256)
    ap.add_argument("--n-test", type=int, default=256)
    ap.add_argument("--H", type=int, default=256)
    ap.add_argument("--iters", type=int, default=3000)
    ap.add_argument("--max-steps", type=int, default=6_000_000)
    ap.add_argument("--out", default=None)
    ap.add_argument("--npz", default=None, help="per-channel steps and state differences")
    ap.add_argument("--time-training", action="store_true",
                    help="only time training iterations of the network (batch 256, random data)")
    a = ap.parse_args()
    from . import build, lbm
    build.build()
    if a.time_training:
        print(json.dumps({"ms_per_iteration": time_training(lbm), "batch": 256, "sizes": SIZES}))
        return
    res, arrays = study(lbm, a.n_train, a.n_test, a.H, iters=a.iters, max_steps=a.max_steps)
    s = json.dumps(res, indent=1, default=float)
    print(s)
    if a.out:
        with open(a.out, "w") as f:
            f.write(s)
    if a.npz:
        np.savez_compressed(a.npz, **arrays)


if __name__ == "__main__":
    main()
