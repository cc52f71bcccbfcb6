"""Run one periodic thermal Taylor-Green case through the C ABI and print its MLUPS.

  python -m paper_1611_02409_gb300.run_case --lattice d2q37 --grid 2048 --storage fp16 --steps 10

Used for small profiling captures of single kernels; the timed loop is one
lbm_step launch per lattice step on the handle's stream, timed with CUDA events.
"""
from __future__ import annotations

import argparse
import json

import numpy as np


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--lattice", default="d2q37", choices=["d2q37", "d3q103", "d2q33", "d2q77"])
    ap.add_argument("--grid", type=int, default=2048)
    ap.add_argument("--storage", default="fp32", choices=["fp32", "fp16", "bf16", "fp64"])
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--kernel", default="auto", choices=["auto", "direct", "staged", "paired", "twopass"])
    a = ap.parse_args()
    import torch

    from paper_1611_02409_gb300 import build, inputs, lbm
    build.build()
    n = a.grid
    params = dict(Pr=0.71, gamma=1.4, kappa=0.2, tau=0.528655, storage=a.storage,
                  kernel={"auto": 0, "direct": 1, "staged": 2, "paired": 3, "twopass": 4}[a.kernel])
    if a.lattice in ("d2q37", "d2q33", "d2q77"):
        lat = {"d2q37": lbm.LBM_D2Q37, "d2q33": lbm.LBM_D2Q33, "d2q77": lbm.LBM_D2Q77}[a.lattice]
        sim = lbm.Simulation(lattice=lat, nx=n, ny=n, **params)
        fields = inputs.taylor_green_2d(n)
        cells = n * n
    else:
        sim = lbm.Simulation(lattice=lbm.LBM_D3Q103, nx=n, ny=n, nz=n, **params)
        fields = inputs.taylor_green_3d(n, noise=0.0)
        cells = n ** 3
    sim.init(*fields)
    lbm.lbm_step(sim.h, a.warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(sim.stream)
    for _ in range(a.steps):
        lbm.lbm_step(sim.h, 1)
    e1.record(sim.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / a.steps
    d = sim.diagnostics()
    sim.close()
    print(json.dumps({"lattice": a.lattice, "grid": n, "storage": a.storage, "kernel": a.kernel, "steps": a.steps,
                      "ms_per_step": ms, "mlups": cells / (ms * 1e-3) / 1e6, "bad_cells": d["bad"]}))
    if d["bad"]:
        raise SystemExit("non-finite state")


if __name__ == "__main__":
    main()
