"""Writes couette_steady_oracle.txt: steady thermal Couette channels computed by the FP64
oracle alone (Sec. VI A set-up with the walls of reading R5), the reference against which
the warm-started and rest-started GPU channels are compared.

The channels are held-out draws from the distribution of the surrogate's training sweep
(Pr in [0.5, 2], gamma in [1.1, 1.67], wall Mach number in [0.01, 0.1], tau in [0.6, 1],
top-wall temperature 1 + dT with dT in [-0.05, 0.05]; bottom wall at rest at T = 1), on
heights the oracle settles in minutes.  Each starts from rest and runs in chunks of m
steps until the change per step times the slowest decay time bounds the distance to the
steady state below 1e-11 (relative, u_x and T).  The steady channel is uniform in x, so
the oracle runs it one cell wide (identical, to the last bit, to a wider periodic
channel).

    python tests/golden/make_couette_steady.py      # under a minute on eight cores
"""
from __future__ import annotations

import multiprocessing as mp
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "couette_steady_oracle.txt")
HEIGHTS = (33, 37, 41, 49, 57, 65)
SEED = 1611
CHUNK = 200
BOUND = 1e-11


def draw_cases():
    rng = np.random.Generator(np.random.PCG64(SEED))
    out = []
    for H in HEIGHTS:
        Pr, gamma, Ma, tau, dT = (float(v) for v in rng.uniform([0.5, 1.1, 0.01, 0.6, -0.05],
                                                                [2.0, 1.67, 0.1, 1.0, 0.05]))
        out.append(dict(H=H, Pr=Pr, gamma=gamma, Ma=Ma, tau=tau, dT=dT, U=float(Ma * np.sqrt(gamma))))
    return out


def settle(case):
    os.environ["OMP_NUM_THREADS"] = "1"
    sys.path.insert(0, ROOT)
    from oracle import oracle as O
    H = case["H"]
    o = O.Sim(O.D2Q37, nx=1, ny=H, walls=True, Pr=case["Pr"], gamma=case["gamma"], kappa=0.2, tau=case["tau"],
              wall_u=[[0, 0, 0], [case["U"], 0, 0]], wall_T=[1.0, 1.0 + case["dT"]])
    o.init(np.ones((H, 1)), np.zeros((2, H, 1)), np.ones((H, 1)))
    r = o.r
    nu = (case["tau"] - 0.5) / r ** 2
    tau_slow = (H - 1) ** 2 * max(1.0, case["Pr"]) / (np.pi ** 2 * nu)
    prev, d_prev, steps = None, None, 0
    while True:
        o.step(CHUNK)
        steps += CHUNK
        m = o.moments()
        X = (m["u"][0][:, 0], m["T"][:, 0])
        if prev is not None:
            d = max(np.linalg.norm(a - b) / np.linalg.norm(a) for a, b in zip(X, prev))
            tau_est = CHUNK / np.log(d_prev / d) if d_prev and d < d_prev else np.inf
            bound = d / CHUNK * max(tau_slow, tau_est if np.isfinite(tau_est) else 0.0)
            if (steps > 3 * tau_slow and bound < BOUND) or d == 0.0 or steps > 5_000_000:
                break
            d_prev = d
        prev = X
    o.close()
    prof = np.stack([m["rho"][:, 0], m["u"][0][:, 0], m["u"][1][:, 0], m["T"][:, 0], m["Pi"][1][:, 0],
                     m["q"][1][:, 0]], 1)
    return dict(case, steps=steps, bound=bound, tau_slow=tau_slow, prof=prof)


def main():
    cases = draw_cases()
    with mp.get_context("spawn").Pool(min(len(cases), os.cpu_count() or 1)) as pool:
        res = pool.map(settle, cases)
    lines = [
        "# Steady thermal Couette channels of the FP64 oracle (oracle/lbm_oracle.c; Sec. VI A set-up,",
        "# walls by reading R5), D2Q37, kappa = 0.2, shifted Prandtl mapping (reading R3), from rest.",
        "# Written by tests/golden/make_couette_steady.py, which calls only the oracle; no value",
        "# here comes from the CUDA path.  Per case: a 'case' line (index, H, Pr, gamma, Ma, tau, dT,",
        "# top-wall velocity U = Ma sqrt(gamma), oracle steps, bound on the relative distance to the",
        "# steady state), then H rows y: rho u_x u_y T Pi_xy q_y.",
    ]
    for k, c in enumerate(res):
        lines.append(f"case {k} {c['H']} {c['Pr']!r} {c['gamma']!r} {c['Ma']!r} {c['tau']!r} {c['dT']!r} "
                     f"{c['U']!r} {c['steps']} {c['bound']:.3e}")
        for y, row in enumerate(c["prof"]):
            lines.append(f"{y} " + " ".join(repr(float(v)) for v in row))
    with open(OUT, "w") as f:
        f.write("\n".join(lines) + "\n")
    for c in res:
        print(c["H"], c["steps"], f"{c['bound']:.2e}", f"tau_slow={c['tau_slow']:.0f}")


def load(path=OUT):
    """[(case dict, profile array [H, 6])] from the golden file."""
    out, cur, rows = [], None, []
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        t = line.split()
        if t[0] == "case":
            if cur is not None:
                out.append((cur, np.array(rows)))
            cur = dict(H=int(t[2]), Pr=float(t[3]), gamma=float(t[4]), Ma=float(t[5]), tau=float(t[6]),
                       dT=float(t[7]), U=float(t[8]), steps=int(t[9]), bound=float(t[10]))
            rows = []
        else:
            rows.append([float(v) for v in t[1:]])
    if cur is not None:
        out.append((cur, np.array(rows)))
    return out


if __name__ == "__main__":
    main()
