"""Prandtl-number mapping study (Sec. III, Eqs. Gamma and Pr; Sec. VI A) on the GPU.

The paper relaxes g and h at the rate Pr/tau and fixes the Gaussian's nu through
1 - nu + kappa nu = 1/Pr.  In the discrete update the traceless stress relaxes at
omega (1 - nu + kappa nu) and the heat flux at omega; with tau_s and tau_q the reciprocals
of those two rates, the lattice kinematic viscosity is nu_kin = (T/r^2)(tau_s - 1/2) and
the thermal diffusivity chi = (T/r^2)(tau_q - 1/2) (lattice units, c_s^2 = T/r^2).  The
library's two mappings:

  LBM_PR_SHIFTED  tau_s = tau, tau_q = 1/2 + (tau - 1/2)/Pr, so nu_kin/chi = Pr at every tau;
  LBM_PR_LITERAL  omega = Pr/tau and 1 - nu + kappa nu = 1/Pr as printed: tau_s = tau,
                  tau_q = tau/Pr, so nu_kin/chi = (tau - 1/2)/(tau/Pr - 1/2), which reaches
                  Pr only as tau grows (0.12 at tau = 0.528655, Pr = 1/1.4).

`transport_vs_tau` measures both diffusivities for every (mode, tau) as the instances of
one batch: shear waves decay at nu_kin k^2, isobaric thermal waves at chi k^2.

`paper_couette` runs the paper's thermal Couette set-up (Sec. VI A): X x Y = 50 x 400
D2Q37, rho = T = 1 at rest, the top wall moving at u0 = 1, both walls at T = 1,
kappa = 0.2, N_f = 3 (gamma = 1.4) and Pr = 1/1.4: the printed nu = 0.5 read as -0.5, the
sign for which 1 - nu + kappa nu = 1.4 gives the stated Pr = 0.71.  The paper gives no tau;
tau = 1 here.  The paper's time is t = steps / (r (Y - 1)): Delta x = r in its units and
the walls sit on rows 0 and Y - 1, as t = steps / (X r) in the shock tube (Sec. VI B).
The start-up velocity at t = 5, 10, 20, 60 is compared with Eq.
CouetteVelocityDimensionless written with nu_kin, and the steady temperature with
Eq. CouetteDi3, T = 1 + Pr_eff u0^2 / (D + N_f + 2) eta (1 - eta), eta = y / (Y - 1), for
each mapping's own Pr_eff.
"""
from __future__ import annotations

import time

import numpy as np

from . import inputs

PAPER_PR = 1.0 / 1.4
TAUS = (0.51, 0.528655, 0.55, 0.6, 0.7, 0.8, 1.0, 1.5, 2.0)
PAPER_TIMES = (5.0, 10.0, 20.0, 60.0)


def modes(lbm):
    return {"shifted": lbm.LBM_PR_SHIFTED, "literal": lbm.LBM_PR_LITERAL}


def predicted(mode_name, tau, Pr, r):
    """(nu_kin, chi, Pr_eff) of a mapping at temperature 1, lattice units."""
    tau_q = 0.5 + (tau - 0.5) / Pr if mode_name == "shifted" else tau / Pr
    nu, chi = (tau - 0.5) / r ** 2, (tau_q - 0.5) / r ** 2
    return nu, chi, nu / chi


def _fit_rate(ts, amps, pred_rate, max_decay=2.5, skip=1):
    """Exponential decay rate from amplitude samples: a log-linear fit over the samples
    after the first `skip` (the initial kinetic transient) and before the predicted decay
    reaches e^-max_decay (beyond it the slower non-hydrodynamic remainder dominates)."""
    ts, amps = np.asarray(ts, float), np.asarray(amps, float)
    sel = (ts * pred_rate <= max_decay) & (np.arange(len(ts)) >= skip)
    sel[skip:skip + 3] = True
    return -np.polyfit(ts[sel], np.log(amps[sel]), 1)[0]


def transport_vs_tau(lbm, taus=TAUS, Pr=PAPER_PR, gamma=1.4, kappa=0.2, n=128, steps=1600, every=25):
    """Measured nu_kin and chi for every mapping and tau (one batch, FP32).  Returns a list
    of rows: mode, tau, measured and predicted nu_kin, chi, Pr_eff."""
    _, r, _, _ = lbm.lbm_lattice_table(lbm.LBM_D2Q37)
    k = 2 * np.pi / n
    cases = []
    for name, mode in modes(lbm).items():
        for tau in taus:
            base = dict(Pr=Pr, gamma=gamma, kappa=kappa, tau=tau, pr_mode=mode)
            cases.append((name, tau, "shear", dict(nx=4, ny=n, **base), inputs.shear_wave(n)))
            cases.append((name, tau, "thermal", dict(nx=n, ny=4, **base), inputs.isobaric_thermal_wave(n)))
    bt = lbm.Batch([c[3] for c in cases])
    try:
        for i, c in enumerate(cases):
            bt.init(i, *c[4])
        ph_y = np.sin(2 * np.pi * np.arange(n) / n)[:, None]
        ph_x = ph_y.T

        def amp(i, kind):
            m = bt.moments(i)
            return 2 * np.mean(m["u"][0] * ph_y) if kind == "shear" else 2 * np.mean((m["T"] - 1) * ph_x)

        ts, amps = [0], [[amp(i, c[2]) for i, c in enumerate(cases)]]
        for t in range(every, steps + 1, every):
            bt.run(every, tol=0.0, check_every=every)
            ts.append(t)
            amps.append([amp(i, c[2]) for i, c in enumerate(cases)])
    finally:
        bt.close()
    amps = np.array(amps)
    rows = {}
    for i, (name, tau, kind, _, _) in enumerate(cases):
        nu, chi, pe = predicted(name, tau, Pr, r)
        d = nu if kind == "shear" else chi
        row = rows.setdefault((name, tau), dict(mode=name, tau=tau, Pr_set=Pr, nu_pred=nu, chi_pred=chi,
                                                Pr_pred=pe))
        row["nu" if kind == "shear" else "chi"] = _fit_rate(ts, amps[:, i], d * k * k) / (k * k)
    out = []
    for row in rows.values():
        row["Pr_meas"] = row["nu"] / row["chi"]
        out.append(row)
    return out


def startup_series(eta, nu_t, nmax=2000):
    """Eq. CouetteVelocityDimensionless, u/u0 at heights eta (walls at 0 and 1) and
    nu t / L^2 = nu_t."""
    u = np.array(eta, float)
    for m in range(1, nmax + 1):
        e = np.exp(-m * m * np.pi ** 2 * nu_t)
        if e < 1e-18:
            break
        u += 2.0 / np.pi * (-1) ** m / m * e * np.sin(m * np.pi * eta)
    return u


def couette_params(lbm, mode, X=50, Y=400, u0=1.0, tau=1.0, Pr=PAPER_PR, gamma=1.4, kappa=0.2):
    return dict(nx=X, ny=Y, Pr=Pr, gamma=gamma, kappa=kappa, tau=tau, pr_mode=mode, bc_y=lbm.LBM_WALLS,
                wall_u=[[0, 0, 0], [u0, 0, 0]], wall_T=[1.0, 1.0])


def paper_couette(lbm, X=50, Y=400, u0=1.0, tau=1.0, Pr=PAPER_PR, gamma=1.4, kappa=0.2,
                  times=PAPER_TIMES, steady_tol=1e-9, max_steps=3_000_000):
    """Start-up profiles at the paper's times and the steady temperature, both mappings.
    The steady run stops at a per-step relative change of `steady_tol`; FP32 storage
    leaves a rounding floor near 3e-10 at 50 x 400, so the tolerance stays above it.
    Returns a dict per mode: the profiles, their errors against the analytic solutions,
    the fitted heating coefficient and the step counts."""
    _, r, _, _ = lbm.lbm_lattice_table(lbm.LBM_D2Q37)
    Nf = 2.0 / (gamma - 1.0) - 2
    eta = np.arange(Y) / (Y - 1)
    out = {}
    for name, mode in modes(lbm).items():
        nu, chi, pe = predicted(name, tau, Pr, r)
        sim = lbm.Simulation(**couette_params(lbm, mode, X, Y, u0, tau, Pr, gamma, kappa))
        try:
            sim.init(*inputs.rest_channel(X, Y))
            done, prof = 0, []
            for t in times:
                s = int(round(t * r * (Y - 1)))
                sim.step(s - done)
                done = s
                m = sim.moments()
                u = m["u"][0].mean(1) / u0
                ua = startup_series(eta, nu * s / (Y - 1) ** 2)
                prof.append(dict(t=t, steps=s, u=u, u_analytic=ua, max_err=float(np.abs(u - ua).max()),
                                 x_spread=float(np.abs(m["u"][0] - m["u"][0].mean(1, keepdims=True)).max())))
        finally:
            sim.close()
        out[name] = dict(nu=nu, chi=chi, Pr_eff=pe, startup=prof)
    # steady temperature: both mappings in one batch, run to the residual tolerance
    names = list(modes(lbm))
    bt = lbm.Batch([couette_params(lbm, modes(lbm)[nm], X, Y, u0, tau, Pr, gamma, kappa) for nm in names])
    try:
        for i in range(len(names)):
            bt.init(i, *inputs.rest_channel(X, Y))
        t0 = time.perf_counter()
        bt.run(max_steps, tol=steady_tol, check_every=2000)
        secs = time.perf_counter() - t0
        steps, res, act = bt.status()
        for i, nm in enumerate(names):
            m = bt.moments(i)
            T, u = m["T"].mean(1), m["u"][0].mean(1) / u0
            heat = out[nm]["Pr_eff"] * u0 ** 2 / (2 + Nf + 2)
            Ta = 1.0 + heat * eta * (1 - eta)
            coef = float(np.polyfit(eta * (1 - eta), T - 1.0, 1)[0])
            out[nm]["steady"] = dict(steps=int(steps[i]), converged=bool(act[i] == 0), residual=float(res[i]),
                                     T=T, T_analytic=Ta, T_err=float(np.abs(T - Ta).max() / heat * 4),
                                     u_err=float(np.abs(u - eta).max()),
                                     heating_coef=coef, heating_ratio=coef / heat,
                                     heating_ratio_set_Pr=coef / (Pr * u0 ** 2 / (2 + Nf + 2)))
        out["steady_seconds"] = secs
    finally:
        bt.close()
    return out


def main():
    import argparse
    import json
    ap = argparse.ArgumentParser()
    ap.add_argument("--Y", type=int, default=400)
    ap.add_argument("--tau", type=float, default=1.0)
    a = ap.parse_args()
    from . import build, lbm
    build.build()
    rows = transport_vs_tau(lbm)
    for row in rows:
        print(json.dumps({k: (round(v, 5) if isinstance(v, float) else v) for k, v in row.items()}))
    pc = paper_couette(lbm, Y=a.Y, tau=a.tau)
    for nm in ("shifted", "literal"):
        d = pc[nm]
        print(nm, "Pr_eff", round(d["Pr_eff"], 4), "start-up max|u - series|",
              [round(p["max_err"], 5) for p in d["startup"]], "steady", {k: v for k, v in d["steady"].items()
                                                                         if not isinstance(v, np.ndarray)})


if __name__ == "__main__":
    main()
