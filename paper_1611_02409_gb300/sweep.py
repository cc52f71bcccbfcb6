"""Batched parameter sweep: many uneven 2-D instances in one batch (lbm_batch_*).

The sweep mixes periodic thermal Taylor-Green squares (side drawn from 64..512 in steps
of 8) with thermal Couette channels 4 x H (H drawn from 64..512), each with its own
seeded Pr in [0.5, 2], gamma in [1.1, 1.67], tau in [0.6, 1.0], wall Mach number <= 0.1
and wall temperature ratio within 5 %.  Every instance stops at residual `tol` or the
step cap.  The channels' steady profiles -- u_x, T, Pi_xy and q_y averaged along x and
resampled to `npts` points of the normalised height y/H -- are the surrogate's training
set; Pi_xy and q_y scale as 1/H in steady Couette flow and are stored times (ny - 1).
"""
from __future__ import annotations

import numpy as np

from . import inputs


def draw_instances(n_square=256, n_channel=256, seed=0):
    """Parameter dicts (lbm.make_params keywords) plus the channel inputs
    (Pr, gamma, Ma, tau, dT) of every instance; seeded and reproducible."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(n_square):
        n = int(rng.choice(np.arange(64, 513, 8)))
        out.append(dict(kind="square", params=dict(nx=n, ny=n, Pr=float(rng.uniform(0.5, 2.0)),
                                                    gamma=float(rng.uniform(1.1, 1.67)), kappa=0.2,
                                                    tau=float(rng.uniform(0.6, 1.0)))))
    for _ in range(n_channel):
        H = int(rng.integers(64, 513))
        out.append(channel_case(float(rng.uniform(0.5, 2.0)), float(rng.uniform(1.1, 1.67)),
                                float(rng.uniform(0.01, 0.1)), float(rng.uniform(0.6, 1.0)),
                                float(rng.uniform(-0.05, 0.05)), H))
    return out


def channel_case(Pr, gamma, Ma, tau, dT, H, nx=4):
    """A 4 x H thermal Couette channel: bottom wall at rest with T = 1, top wall moving at
    Mach number Ma (of the bottom temperature) with T = 1 + dT."""
    U = Ma * np.sqrt(gamma * 1.0)
    return dict(kind="channel", inputs=np.array([Pr, gamma, Ma, tau, dT]),
                params=dict(nx=nx, ny=H, Pr=Pr, gamma=gamma, kappa=0.2, tau=tau, bc_y=1,
                            wall_u=[[0, 0, 0], [U, 0, 0]], wall_T=[1.0, 1.0 + dT]))


def initial_fields(case):
    p = case["params"]
    if case["kind"] == "square":
        return inputs.taylor_green_2d(p["nx"], U0=0.02, T_amp=0.01)
    return inputs.rest_channel(p["nx"], p["ny"])


def profiles(m, npts=256):
    """x-averaged u_x, T, Pi_xy, q_y of a channel, resampled to npts points of y/(ny-1);
    Pi_xy and q_y multiplied by (ny - 1)."""
    ny = m["T"].shape[0]
    y = np.arange(ny) / (ny - 1)
    yq = np.linspace(0.0, 1.0, npts)
    cols = [m["u"][0].mean(1), m["T"].mean(1), m["Pi"][1].mean(1) * (ny - 1), m["q"][1].mean(1) * (ny - 1)]
    return np.stack([np.interp(yq, y, c) for c in cols])


def run_sweep(lbm, cases, max_steps=20000, tol=1e-8, check_every=100, autotune=True):
    """Runs every case in one batch; returns (status dict, channel profiles, channel
    inputs, converged flags, seconds)."""
    import time
    bt = lbm.Batch([c["params"] for c in cases])
    tile = bt.autotune(20) if autotune else 128
    for i, c in enumerate(cases):
        bt.init(i, *initial_fields(c))
    t0 = time.perf_counter()
    done = bt.run(max_steps, tol=tol, check_every=check_every)
    secs = time.perf_counter() - t0
    steps, res, act = bt.status()
    prof, xin, conv = [], [], []
    for i, c in enumerate(cases):
        if c["kind"] != "channel":
            continue
        prof.append(profiles(bt.moments(i)))
        xin.append(c["inputs"])
        conv.append(act[i] == 0)
    bt.close()
    status = dict(batch_steps=done, steps=steps, residual=res, active=act, tile=tile)
    return status, np.array(prof), np.array(xin), np.array(conv), secs


COUETTE_PR = (0.5, 0.71, 1.0, 2.0)
COUETTE_GAMMA = (1.3, 1.4, 1.67)


def couette_grid(H=256, U=0.05, T_bottom=1.0, T_top=1.02, tau=0.528655, nx=4, kappa=0.2):
    """The Pr x gamma grid of thermal Couette channels nx x H: bottom wall at rest at
    T_bottom, top wall moving at U (paper units, sqrt(theta_0) = 1) at T_top; tau gives
    nu = 0.02 lattice units on D2Q37."""
    return [dict(kind="channel", inputs=np.array([Pr, g, U, tau, T_top - T_bottom]),
                 params=dict(nx=nx, ny=H, Pr=Pr, gamma=g, kappa=kappa, tau=tau, bc_y=1,
                             wall_u=[[0, 0, 0], [U, 0, 0]], wall_T=[T_bottom, T_top]))
            for Pr in COUETTE_PR for g in COUETTE_GAMMA]


def run_couette(lbm, cases, tol=1e-8, settle_steps=0, check_every=1000, max_steps=5_000_000):
    """All cases in one batch from rest: steps to residual `tol`, then (if settle_steps)
    every case continues `settle_steps` more steps.  Returns per-case steps to tol,
    x-averaged u_x and T profiles at tol and after settling, and seconds."""
    import time
    bt = lbm.Batch([c["params"] for c in cases])
    for i, c in enumerate(cases):
        bt.init(i, *initial_fields(c))
    t0 = time.perf_counter()
    bt.run(max_steps, tol=tol, check_every=check_every)
    secs = time.perf_counter() - t0
    steps, res, act = bt.status()
    prof = lambda m: np.stack([m["u"][0].mean(1), m["T"].mean(1)])
    at_tol = [prof(bt.moments(i)) for i in range(len(cases))]
    out = dict(steps_to_tol=steps.copy(), converged=act == 0, residual=res.copy(), seconds_to_tol=secs,
               profiles_at_tol=np.array(at_tol))
    if settle_steps:
        bt.activate()
        t0 = time.perf_counter()
        bt.run(settle_steps, tol=0.0, check_every=check_every)
        out["seconds_settle"] = time.perf_counter() - t0
        out["steps_total"] = bt.status()[0]
        out["profiles_settled"] = np.array([prof(bt.moments(i)) for i in range(len(cases))])
    bt.close()
    return out


def main():
    """The sweep (default 256 squares + 256 channels), one batch, residual 1e-8 or 20k steps."""
    import argparse
    import json
    ap = argparse.ArgumentParser()
    ap.add_argument("--max-steps", type=int, default=20000)
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--check-every", type=int, default=100)
    ap.add_argument("--out", default=None)
    ap.add_argument("--squares", type=int, default=256)
    ap.add_argument("--channels", type=int, default=256)
    a = ap.parse_args()
    from . import build, lbm
    build.build()
    cases = draw_instances(a.squares, a.channels)
    ncomp = np.array([c["params"]["nx"] * (c["params"]["ny"] - (2 if c["kind"] == "channel" else 0))
                      for c in cases], dtype=np.float64)
    status, prof, xin, conv, secs = run_sweep(lbm, cases, max_steps=a.max_steps, tol=a.tol,
                                              check_every=a.check_every, autotune=True)
    updates = float(np.sum(ncomp * status["steps"]))
    kinds = np.array([c["kind"] for c in cases])
    res = dict(instances=len(cases), cells_total=float(ncomp.sum()), batch_steps=int(status["batch_steps"]),
               tile=int(status["tile"]), seconds=secs, cell_updates=updates, mlups=updates / secs / 1e6,
               converged_channels=int(conv.sum()), channels=int((kinds == "channel").sum()),
               converged_squares=int(((status["active"] == 0) & (kinds == "square")).sum()),
               channel_heights_converged=[int(c["params"]["ny"]) for c, k in zip(cases, status["active"])
                                          if c["kind"] == "channel" and k == 0])
    print(json.dumps(res))
    if a.out:
        np.savez_compressed(a.out, X=xin, Y=prof, converged=conv)


if __name__ == "__main__":
    main()
