#!/usr/bin/env python
"""Throughput of the fused ES-BGK stream-collide step on GB300 (one JSON line).

Workload: 4096 x 4096 periodic thermal Taylor-Green field (U0 = 0.02, T amplitude 0.01),
D2Q37, Pr = 0.71, gamma = 1.4 (N_f = 3), kappa = 0.2, tau = 0.528655 (nu = 0.02 lattice
units).  One bench step = one lattice time step over the whole grid (one kernel launch).
The headline `value` is FP32-storage MLUPS with the populations resident in HBM; the
FP16 / BF16 shifted-storage forms are timed the same way, and the field error of every
storage against the FP64 oracle is measured on a 128^2 copy of the field after 200 steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (under torchrun) every rank runs its own replica (the step is one domain
per GPU; scaling "weak"); the time is the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS & % HBM peak, FP32 vs FP16-store at ≤1e-3 err; warm-start step savings"
N_GRID = 4096
PARAMS = dict(Pr=0.71, gamma=1.4, kappa=0.2, tau=0.528655)
Q = 37
# the sources the profiled stream-collide kernels are built from (the staged kernel in
# tma_kernel.cuh is not among them)
KERNEL_SOURCES = ["kernels.cuh", "physics.cuh", "lattice.cuh", "dispatch.cuh", "vec2.cuh"]


def workload(storage):
    return (f"thermal Taylor-Green {N_GRID}x{N_GRID} periodic, D2Q37, {storage} storage, Pr=0.71, gamma=1.4 "
            f"(N_f=3), kappa=0.2, tau=0.528655 (nu=0.02 lu), U0=0.02, T amplitude 0.01")


def code_only(src):
    """C++ source without comments and with whitespace runs collapsed (string and character
    literals kept), so that a comment edit leaves the kernel hash unchanged."""
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if c in "\"'":
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        elif src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


def kernel_src_sha():
    """Hash of the kernel sources' code (comments and layout excluded): the key under which
    ncu traffic counters taken on that code stay valid."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1611_02409_gb300", "csrc", f), encoding="utf-8") as fh:
            h.update(code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def profiled_traffic(kernel_tag):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on the current
    kernel source; else None."""
    sha = kernel_src_sha()
    pdir = os.path.join(ROOT, "profiles")
    if not os.path.isdir(pdir):
        return None
    pat = re.compile(r"traffic:\s*kernel=(\S+)\s+src_sha=(\S+)\s+bytes_per_launch=(\d+)")
    for fn in sorted(os.listdir(pdir)):
        if not fn.endswith((".md", ".txt")):
            continue
        for m in pat.finditer(open(os.path.join(pdir, fn)).read()):
            if m.group(1) == kernel_tag and m.group(2) == sha:
                return int(m.group(3))
    return None


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.15)
        self.proc.terminate()
        self.proc.wait()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(torch, value, ws, device="cuda"):
    """The largest of a per-rank number over all ranks (every rank receives it)."""
    if ws <= 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(ws, cells_per_rank, steps, seconds):
    """Cell updates of all ranks (independent replicas, weak scaling) per second, in MLUPS."""
    return ws * cells_per_rank * steps / seconds / 1e6


def time_steps(torch, lbm, sim, steps, warmup, ws, clocks=None):
    """Times `steps` single-step launches on the handle's stream: total and per launch."""
    st = sim.stream
    for _ in range(warmup):
        lbm.lbm_step(sim.h, 1)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(st)
    for k in range(steps):
        ev[k][0].record(st)
        lbm.lbm_step(sim.h, 1)
        ev[k][1].record(st)
    t1.record(st)
    torch.cuda.synchronize()
    clk = clocks.stop() if clocks else None
    total_ms = t0.elapsed_time(t1)
    per_launch = [a.elapsed_time(b) for a, b in ev]
    if ws > 1:
        total_ms = max_over_ranks(torch, total_ms, ws)
        torch.distributed.barrier()
    return total_ms, float(np.mean(per_launch)), clk


def accuracy_vs_oracle(lbm, n=128, steps=200):
    """Field errors of every storage form against the FP64 oracle on an n^2 copy."""
    from oracle import oracle as O
    from paper_1611_02409_gb300 import inputs
    fields = inputs.taylor_green_2d(n)
    o = O.Sim(O.D2Q37, nx=n, ny=n, **PARAMS)
    o.init(*fields)
    o.step(steps)
    mo = o.moments()
    o.close()
    out = {}
    for storage in ("fp32", "fp16", "bf16"):
        sim = lbm.Simulation(nx=n, ny=n, storage=storage, **PARAMS)
        sim.init(*fields)
        sim.step(steps)
        mg = sim.moments()
        sim.close()
        errs = {}
        for k in ("rho", "u", "T"):
            d = np.linalg.norm((mg[k] - mo[k]).ravel())
            errs[k] = float(d / np.linalg.norm(mo[k].ravel()))
            errs[k + "_dev"] = float(d / np.linalg.norm((mo[k] - mo[k].mean()).ravel()))
        errs["max_rel"] = max(errs["rho"], errs["u"], errs["T"])
        out[storage] = errs
    out["case"] = f"thermal Taylor-Green {n}x{n}, {steps} steps, same parameters"
    return out


def oracle_mlups(seconds=12.0, n=512):
    """The oracle as it stands, on this host's cores, on an n^2 sample of the workload."""
    from oracle import oracle as O
    from paper_1611_02409_gb300 import inputs
    o = O.Sim(O.D2Q37, nx=n, ny=n, **PARAMS)
    o.init(*inputs.taylor_green_2d(n))
    o.step(1)
    steps, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        o.step(1)
        steps += 1
    dt = time.perf_counter() - t0
    o.close()
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": n * n * steps / dt / 1e6, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": f"{n}x{n} thermal Taylor-Green sample of the workload, {steps} FP64 steps in {dt:.1f} s"}


_ORACLE_TIMER = r"""
import json, os, sys, time
sys.path.insert(0, sys.argv[1])
from oracle import oracle as O
from paper_1611_02409_gb300 import inputs
kind, seconds = sys.argv[2], float(sys.argv[3])
prm = dict(Pr=0.71, gamma=1.4, kappa=0.2, tau=0.528655)
if kind == "d3q103_32":
    n = 32
    o = O.Sim(O.D3Q103, nx=n, ny=n, nz=n, **prm)
    o.init(*inputs.taylor_green_3d(n, U0=0.02, T_amp=0.01, noise=1e-6))
    cells = n ** 3
elif kind == "d2q37_64":
    o = O.Sim(O.D2Q37, nx=64, ny=64, **prm)
    o.init(*inputs.shear_thermal_wave(64, 64, noise=1e-6, seed=0))
    cells = 64 * 64
else:
    n = 1024
    o = O.Sim(O.D2Q37, nx=n, ny=n, **prm)
    o.init(*inputs.taylor_green_2d(n))
    cells = n * n
o.step(1)
steps, t0 = 0, time.perf_counter()
while time.perf_counter() - t0 < seconds:
    o.step(1)
    steps += 1
dt = time.perf_counter() - t0
print(json.dumps({"mlups": cells * steps / dt / 1e6, "steps": steps, "seconds": dt}))
"""


def cpu_model():
    """The host CPU's model name (lscpu), and its logical core count."""
    name = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() == "Model name":
                name = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return name, os.cpu_count() or 1


def oracle_baselines(seconds=3.0):
    """The oracle, as it stands, single-threaded and on all host cores, on the three CPU
    baseline workloads: the 64^2 shear and thermal wave, the 32^3 copy of the 3-D
    Taylor-Green vortex (D3Q103) and a 1024^2 Taylor-Green sample.  Each timing runs in
    a fresh process (the OpenMP thread count is fixed at its start) for about `seconds`."""
    name, ncpu = cpu_model()
    out = {"cpu_model": name, "nproc": ncpu, "seconds_per_timing": seconds, "unit": "MLUPS"}
    for kind in ("d2q37_64", "d3q103_32", "d2q37_1024"):
        row = {}
        for threads in (1, ncpu):
            env = dict(os.environ, OMP_NUM_THREADS=str(threads))
            try:
                r = subprocess.run([sys.executable, "-c", _ORACLE_TIMER, ROOT, kind, str(seconds)], env=env,
                                   capture_output=True, text=True, timeout=600)
                row[f"threads_{threads}"] = json.loads(r.stdout.strip().splitlines()[-1])
            except Exception as e:
                row[f"threads_{threads}"] = {"error": f"{type(e).__name__}: {e}"}
        out[kind] = row
    return out


def bench_3d(torch, lbm, steps, warmup, peak, n=256):
    """256^3 thermal Taylor-Green vortex on D3Q103 (FP32 and FP16 storage)."""
    from paper_1611_02409_gb300 import inputs
    fields = inputs.taylor_green_3d(n, U0=0.02, T_amp=0.01, noise=1e-6)
    out = {"workload": f"3-D thermal Taylor-Green {n}^3 periodic, D3Q103, Pr=0.71, gamma=1.4, kappa=0.2, "
                       f"tau=0.528655"}
    for storage in ("fp32", "fp16"):
        sim = lbm.Simulation(lattice=lbm.LBM_D3Q103, nx=n, ny=n, nz=n, storage=storage, **PARAMS)
        sim.init(*fields)
        total_ms, launch_ms, _ = time_steps(torch, lbm, sim, steps, warmup, 1)
        sim.close()
        del sim
        torch.cuda.empty_cache()
        b_cell = 2 * 103 * 2 * (4 if storage == "fp32" else 2)
        ach = b_cell * n ** 3 / (launch_ms * 1e-3) / 1e9
        out[storage] = {"mlups": n ** 3 * steps / (total_ms * 1e-3) / 1e6, "launch_ms": launch_ms,
                        "achieved_gbs": ach, "frac": ach / peak, "algorithmic_bytes_per_cell": b_cell,
                        "steps": steps}
    out["accuracy"] = accuracy_3d(lbm)
    return out


def accuracy_3d(lbm, n=32, steps=100):
    """Field errors of FP32 and FP16 storage against the FP64 oracle on an n^3 copy of the
    3-D workload (same parameters and field shape)."""
    from oracle import oracle as O
    from paper_1611_02409_gb300 import inputs
    fields = inputs.taylor_green_3d(n, U0=0.02, T_amp=0.01, noise=1e-6)
    o = O.Sim(O.D3Q103, nx=n, ny=n, nz=n, **PARAMS)
    o.init(*fields)
    o.step(steps)
    mo = o.moments()
    o.close()
    out = {"case": f"3-D thermal Taylor-Green {n}^3, {steps} steps"}
    for storage in ("fp32", "fp16"):
        sim = lbm.Simulation(lattice=lbm.LBM_D3Q103, nx=n, ny=n, nz=n, storage=storage, **PARAMS)
        sim.init(*fields)
        sim.step(steps)
        mg = sim.moments()
        sim.close()
        errs = {k: float(np.linalg.norm((mg[k] - mo[k]).ravel()) / np.linalg.norm(mo[k].ravel()))
                for k in ("rho", "u", "T")}
        errs["max_rel"] = max(errs.values())
        out[storage] = errs
    return out


def bench_batch(torch, lbm, steps, peak):
    """The 512-instance sweep (256 Taylor-Green squares + 256 Couette channels) in one
    batch: tile autotuned, then `steps` graph-replayed steps timed on the device."""
    from paper_1611_02409_gb300 import sweep
    cases = sweep.draw_instances()
    bt = lbm.Batch([c["params"] for c in cases])
    tile = bt.autotune(10)
    for i, c in enumerate(cases):
        bt.init(i, *sweep.initial_fields(c))
    bt.run(100, tol=0.0, check_every=100)  # warm-up window (graph capture)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    done = bt.run(steps, tol=0.0, check_every=100)
    secs = time.perf_counter() - t0
    ncomp = sum(c["params"]["nx"] * (c["params"]["ny"] - (2 if c["kind"] == "channel" else 0)) for c in cases)
    bt.close()
    mlups = ncomp * done / secs / 1e6
    return {"workload": "512 instances: 256 periodic thermal Taylor-Green squares (side 64..512) + 256 thermal "
                        "Couette channels 4 x H (H 64..512), seeded Pr, gamma, tau, wall Mach, dT; D2Q37 FP32",
            "cells": ncomp, "steps": done, "tile": tile, "seconds": secs, "mlups": mlups,
            "frac": mlups * 1e6 * 2 * Q * 2 * 4 / 1e9 / peak, "timing": "host wall clock around graph replays, "
                                                                         "synchronised"}


def bench_couette(lbm):
    """The Pr x gamma thermal Couette grid (4 x 256, U = 0.05, T 1.0 / 1.02, tau = 1), one
    batch: steps to residual 1e-8, then nine decay times of the slowest thermal mode more;
    u and T profiles and the fitted viscous-heating curvature against the analytic steady
    solution (Eq. CouetteDi3, unequal walls).  The same grid at 4 x 64 with tau for
    nu = 0.02 lattice units as a second case."""
    from paper_1611_02409_gb300 import sweep
    r2 = lbm.lbm_lattice_table(lbm.LBM_D2Q37)[1] ** 2
    res = {"workload": "thermal Couette 4xH, top wall U=0.05 T=1.02, bottom T=1.0, Pr x gamma = "
                       "{0.5,0.71,1,2} x {1.3,1.4,1.67}, FP32, one batch; H=256 at tau=1, H=64 at tau=0.528655",
           "errors": "u: max|u - U eta| / U; T: max|T - T_analytic| / (T_top - T_bottom); "
                     "curvature: fitted viscous-heating coefficient / Pr U^2 / (D+N_f+2)"}
    for H, tau in ((256, 1.0), (64, 0.528655)):
        nu = (tau - 0.5) / r2
        cases = sweep.couette_grid(H=H, tau=tau)
        settle = int(9 * (H - 1) ** 2 / (np.pi ** 2 * nu / max(sweep.COUETTE_PR)))
        out = sweep.run_couette(lbm, cases, tol=1e-8, settle_steps=settle, check_every=1000)
        eta = np.arange(H) / (H - 1)
        A = np.stack([eta * (1 - eta), eta - 0.5, np.ones_like(eta)], 1)
        rows = []
        for i, c in enumerate(cases):
            Pr, gamma, U, _, dT = c["inputs"]
            heat = Pr * U ** 2 / (2 + 2.0 / (gamma - 1.0) - 2.0 + 2)
            T_an = 1.0 + dT * eta + heat * eta * (1 - eta)
            err = lambda p: (float(np.abs(p[0] - U * eta).max() / U), float(np.abs(p[1] - T_an).max() / dT))
            eu8, eT8 = err(out["profiles_at_tol"][i])
            eu, eT = err(out["profiles_settled"][i])
            curv = float(np.linalg.lstsq(A, out["profiles_settled"][i][1] - (1.0 + dT * eta), rcond=None)[0][0] / heat)
            rows.append(dict(Pr=float(Pr), gamma=float(gamma), steps_to_1e8=int(out["steps_to_tol"][i]),
                             u_err_at_1e8=eu8, T_err_at_1e8=eT8, u_err=eu, T_err=eT, curvature_ratio=curv))
        res[f"H{H}"] = {"tau": tau, "settle_steps": settle, "seconds_to_1e8": out["seconds_to_tol"],
                        "seconds_settle": out["seconds_settle"], "all_converged": bool(out["converged"].all()),
                        "max_u_err": max(r["u_err"] for r in rows), "max_T_err": max(r["T_err"] for r in rows),
                        "curvature_ratio_range": [min(r["curvature_ratio"] for r in rows),
                                                  max(r["curvature_ratio"] for r in rows)],
                        "cases": rows}
    return res


def gate_errors(f, prof):
    """Relative L2 errors of GPU channel fields [ny, nx] against the oracle's steady
    profiles [ny] (rho, u as a vector field, T)."""
    col = lambda v: np.repeat(v[:, None], f["rho"].shape[1], axis=1)
    rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
    uo = np.stack([col(prof[:, 1]), col(prof[:, 2])])
    return dict(rho=rel(f["rho"], col(prof[:, 0])), u=rel(f["u"], uo), T=rel(f["T"], col(prof[:, 3])))


def bench_warm_start(lbm):
    """The learned warm start: surrogate trained on 256 steady channels (H 64..128), then
    256 held-out 4 x 256 channels from rest and from its prediction, to residual 1e-8.
    Gate against the FP64 oracle: six held-out channels (H 33..65) that the oracle settled
    to within 1e-11 of their steady state (tests/golden/couette_steady_oracle.txt), run
    from rest and from the prediction until the distance to the steady state is bounded
    by 1e-8 (FP64 storage) or 1e-6 (FP32 storage, capped at 60 decay times); final field
    error of each against the oracle."""
    from paper_1611_02409_gb300 import surrogate, sweep
    sys.path.insert(0, os.path.join(ROOT, "tests", "golden"))
    from make_couette_steady import load
    res, _ = surrogate.study(lbm, refine=False, keep_model=True)
    sur = res.pop("model")
    t = res["test"]
    out = {"workload": "256 held-out thermal Couette channels 4x256, seeded Pr, gamma, Ma, tau, dT; surrogate "
                       "5-512-512-512-512-1024 trained on 256 channels of height 64..128 by the lbm_mlp kernels",
           "steps_rest_median": t["steps_rest_median"], "steps_warm_median": t["steps_warm_median"],
           "step_ratio_median": t["step_ratio_median"], "batch_seconds_rest": t["batch_seconds_rest"],
           "batch_seconds_warm": t["batch_seconds_warm"], "converged": [t["rest_converged"], t["warm_converged"]],
           "state_diff_at_1e8": t["state_diff_at_tol"],
           "train_seconds": res["train"]["seconds_total"], "final_loss": res["train"]["losses"][-1][1]}
    gold = load()
    cases = [sweep.channel_case(c["Pr"], c["gamma"], c["Ma"], c["tau"], c["dT"], c["H"]) for c, _ in gold]
    pred = sur.predict(np.array([c["inputs"] for c in cases]))
    gate = {"channels": [c["H"] for c, _ in gold]}
    for storage, bound in (("fp64", 1e-8), ("fp32", 1e-6)):
        rows = surrogate.gate_study(lbm, cases, pred, bound=bound, storage=storage)
        g = {"distance_bound": bound}
        for start in ("rest", "warm"):
            errs = [gate_errors(r[start]["fields"], prof) for r, (_, prof) in zip(rows, gold)]
            g[start] = {"err_vs_oracle_max": max(max(e.values()) for e in errs),
                        "err_u_max": max(e["u"] for e in errs), "err_T_max": max(e["T"] for e in errs),
                        "steps_median": float(np.median([r[start]["steps"] for r in rows])),
                        "seconds_total": float(sum(r[start]["seconds"] for r in rows)),
                        "reached_bound": int(sum(r[start]["distance_bound"] <= bound for r in rows))}
        g["step_ratio_median"] = float(np.median([r["warm"]["steps"] / r["rest"]["steps"] for r in rows]))
        gate[storage] = g
    out["gate_vs_oracle"] = gate
    return out


def bench_shock_tube(torch, lbm, peak, steps_tp=100):
    """D2Q33 (Table D2Q33): the 1-D shock tube of Sec. VI B (1000 x 16, open x ends, 174
    steps) against the exact Riemann solution, and D2Q33 throughput on the 4096^2 thermal
    Taylor-Green field (FP32, direct kernel)."""
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import riemann
    from paper_1611_02409_gb300 import inputs
    X, ny, steps = 1000, 16, 174
    prm = dict(Pr=0.71, gamma=1.4, kappa=0.2, tau=2.0 / 3.0)
    sim = lbm.Simulation(lattice=lbm.LBM_D2Q33, nx=X, ny=ny, bc_x=lbm.LBM_OPEN, **prm)
    rho0 = np.where(np.arange(X) < X // 2, 4.0, 1.0)[None, :].repeat(ny, 0)
    sim.init(rho0, np.zeros((2, ny, X)), np.ones((ny, X)))
    sim.step(steps)
    m = sim.moments()
    r = sim.r
    sim.close()
    t = steps / (X * r)
    s = (np.arange(X) + 0.5 - X / 2) / X / t
    ex = riemann.sample(s, (4.0, 0.0, 4.0), (1.0, 0.0, 1.0), 1.4)
    rho, u, p = m["rho"].mean(0), m["u"][0].mean(0), (m["rho"] * m["T"]).mean(0)
    out = {"workload": "shock tube 1000x16, D2Q33, open x ends, (rho,T,u) = (4,1,0) | (1,1,0), gamma=1.4, "
                       "tau=2/3, 174 steps (t = 0.150)",
           "l1_rel_rho": float(np.abs(rho - ex[0]).mean() / 3), "l1_rel_u": float(np.abs(u - ex[1]).mean() / ex[1].max()),
           "l1_rel_p": float(np.abs(p - ex[2]).mean() / 3), "t": t}
    n = N_GRID
    sim = lbm.Simulation(lattice=lbm.LBM_D2Q33, nx=n, ny=n, **PARAMS)
    sim.init(*inputs.taylor_green_2d(n))
    total_ms, launch_ms, _ = time_steps(torch, lbm, sim, steps_tp, 3, 1)
    sim.close()
    del sim
    torch.cuda.empty_cache()
    b_cell = 2 * 33 * 2 * 4
    ach = b_cell * n * n / (launch_ms * 1e-3) / 1e9
    out["throughput_4096"] = {"mlups": n * n * steps_tp / (total_ms * 1e-3) / 1e6, "launch_ms": launch_ms,
                              "algorithmic_bytes_per_cell": b_cell, "achieved_gbs": ach, "frac": ach / peak}
    return out


def bench_burnett(torch, lbm, peak, steps=60):
    """D2Q77 with the sixth-order (Burnett) equilibrium (Sec. IV): throughput of the default
    two-pass kernel on the 4096^2 thermal Taylor-Green field, FP32 and FP16 storage, at
    2 x 77 x 2 x 4 (FP32) / 2 bytes (FP16) algorithmic bytes per cell."""
    from paper_1611_02409_gb300 import inputs
    n = N_GRID
    out = {"workload": "thermal Taylor-Green 4096x4096 periodic, D2Q77 (sixth-order equilibrium), Pr=0.71, "
                       "gamma=1.4, kappa=0.2, tau=0.528655"}
    fields = inputs.taylor_green_2d(n)
    for st, elem in (("fp32", 4), ("fp16", 2)):
        sim = lbm.Simulation(lattice=lbm.LBM_D2Q77, nx=n, ny=n, storage=st, **PARAMS)
        sim.init(*fields)
        total_ms, launch_ms, _ = time_steps(torch, lbm, sim, steps, 3, 1)
        sim.close()
        del sim
        torch.cuda.empty_cache()
        b_cell = 2 * 77 * 2 * elem
        ach = b_cell * n * n / (launch_ms * 1e-3) / 1e9
        out[st] = {"mlups": n * n * steps / (total_ms * 1e-3) / 1e6, "launch_ms": launch_ms,
                   "algorithmic_bytes_per_cell": b_cell, "achieved_gbs": ach, "frac": ach / peak, "steps": steps}
    return out


def bench_mode_study(lbm):
    """Prandtl-number mappings (Sec. III; Sec. VI A): measured nu_kin, chi and Pr against tau
    for the shifted and the literal mapping, and the paper's 50 x 400 Couette set-up
    (u0 = 1, Pr = 1/1.4, tau = 1): start-up against the series, steady heating against
    Eq. CouetteDi3."""
    from paper_1611_02409_gb300 import mode_study as M
    rows = M.transport_vs_tau(lbm)
    out = {"workload": "shear and isobaric thermal waves, k = 2 pi/128, Pr = 1/1.4, gamma = 1.4, kappa = 0.2, "
                       "FP32, one batch of 36; Couette 50x400 D2Q37, u0 = 1, tau = 1",
           "transport": {m: {f"{r['tau']:g}": {"Pr_meas": r["Pr_meas"], "Pr_pred": r["Pr_pred"],
                                              "nu_ratio": r["nu"] / r["nu_pred"], "chi_ratio": r["chi"] / r["chi_pred"]}
                             for r in rows if r["mode"] == m} for m in ("shifted", "literal")}}
    pc = M.paper_couette(lbm)
    for m in ("shifted", "literal"):
        st = pc[m]["steady"]
        out[f"couette_{m}"] = {"Pr_eff": pc[m]["Pr_eff"],
                               "startup_max_err": {f"t{p['t']:g}": p["max_err"] for p in pc[m]["startup"]},
                               "steady_steps": st["steps"], "converged": st["converged"],
                               "heating_ratio": st["heating_ratio"], "heating_ratio_set_Pr": st["heating_ratio_set_Pr"],
                               "T_err": st["T_err"], "u_err": st["u_err"]}
    out["couette_steady_seconds"] = pc["steady_seconds"]
    return out


def sig(x, n=4):
    """Floats rounded to n significant digits, recursively (keeps the JSON line short)."""
    if isinstance(x, float):
        return float(f"{x:.{n}g}") if np.isfinite(x) else x
    if isinstance(x, dict):
        return {k: sig(v, n) for k, v in x.items()}
    if isinstance(x, (list, tuple)):
        return [sig(v, n) for v in x]
    return x


def summarize(name, d):
    """The short form of one extra measurement for the JSON line (the full form goes to
    the --details file): per-case arrays are reduced to their extremes."""
    if not isinstance(d, dict) or "error" in d:
        return d
    if name == "cpu_baseline":
        w = d.get("workloads", {})
        out = {k: v for k, v in d.items() if k != "workloads"}
        if "cpu_model" in w:
            out["workloads"] = {"cpu_model": w["cpu_model"], "nproc": w["nproc"],
                                "mlups_1_thread_and_all": {k: [w[k].get(f"threads_{t}", {}).get("mlups")
                                                               for t in (1, w["nproc"])]
                                                           for k in ("d2q37_64", "d3q103_32", "d2q37_1024")}}
        return out
    if name == "couette_grid":
        return {h: {k: d[h][k] for k in ("tau", "all_converged", "max_u_err", "max_T_err", "curvature_ratio_range")}
                for h in ("H256", "H64") if h in d}
    if name == "shock_tube_d2q33":
        return {"l1_rel": [d["l1_rel_rho"], d["l1_rel_u"], d["l1_rel_p"]],
                "frac_4096": d.get("throughput_4096", {}).get("frac")}
    if name == "mode_study":
        out = {}
        for m in ("shifted", "literal"):
            rows = d["transport"][m]
            out[f"{m}_Pr_meas_over_pred"] = [min(r["Pr_meas"] / r["Pr_pred"] for r in rows.values()),
                                             max(r["Pr_meas"] / r["Pr_pred"] for r in rows.values())]
            c = d[f"couette_{m}"]
            out[f"couette_{m}"] = {"heating_ratio": c["heating_ratio"], "heating_ratio_set_Pr": c["heating_ratio_set_Pr"],
                                   "startup_max_err": max(c["startup_max_err"].values()), "u_err": c["u_err"]}
        return out
    if name == "accuracy":
        return {k: {f: v[f] for f in ("rho", "u", "T")} for k, v in d.items() if isinstance(v, dict)}
    if name == "d3q103_256":
        out = {st: {k: d[st][k] for k in ("mlups", "frac", "launch_ms")} for st in ("fp32", "fp16") if st in d}
        acc = d.get("accuracy", {})
        out["err_vs_oracle_32cube"] = {st: acc[st]["max_rel"] for st in ("fp32", "fp16") if st in acc}
        return out
    if name == "burnett_d2q77":
        return {st: {k: d[st][k] for k in ("mlups", "frac")} for st in ("fp32", "fp16") if st in d}
    if name == "batched_sweep":
        return {k: d[k] for k in ("cells", "steps", "tile", "mlups", "frac") if k in d}
    if name == "warm_start":
        return {k: d[k] for k in ("steps_rest_median", "steps_warm_median", "step_ratio_median",
                                  "batch_seconds_rest", "batch_seconds_warm", "gate_vs_oracle") if k in d}
    return d


def _extra(out, name, fn):
    """One extra measurement; its failure is recorded, not raised."""
    t0 = time.perf_counter()
    try:
        out[name] = fn()
    except Exception as e:  # the headline line must still print
        out[name] = {"error": f"{type(e).__name__}: {e}"}
    if isinstance(out[name], dict):
        out[name]["wall_seconds"] = time.perf_counter() - t0


def run_reference(args):
    ws, rank, _ = dist_setup()
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_1611_02409_gb300 import inputs
    n = 512
    o = O.Sim(O.D2Q37, nx=n, ny=n, **PARAMS)
    o.init(*inputs.taylor_green_2d(n))
    for _ in range(args.warmup):
        o.step(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.step(1)
    dt = time.perf_counter() - t0
    o.close()
    v = n * n * args.steps / dt / 1e6
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload("fp64 (oracle)"), "sample": f"{n}x{n} per step"},
            "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                             "sample": f"{n}x{n} thermal Taylor-Green sample per step, {args.steps} steps"},
            "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    ws, rank, local = dist_setup()
    if ws > 1:
        torch.cuda.set_device(local)
        torch.distributed.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    from paper_1611_02409_gb300 import build, inputs, lbm
    if rank == 0 or ws == 1:
        build.build()
    if ws > 1:
        torch.distributed.barrier()
    lbm.lib()
    n = N_GRID
    cells = n * n
    rho, u, T = inputs.taylor_green_2d(n)
    peak, peak_kind = measured_peak()
    results = {}
    gpu_index = int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0]) \
        if os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[0].isdigit() else local
    for storage, steps in (("fp32", args.steps), ("fp16", args.steps), ("bf16", max(args.steps // 2, 1))):
        sim = lbm.Simulation(nx=n, ny=n, storage=storage, **PARAMS)
        sim.init(rho, u, T)
        clocks = Clocks(gpu_index) if storage == "fp32" else None
        total_ms, launch_ms, clk = time_steps(torch, lbm, sim, steps, args.warmup, ws, clocks)
        elem = 4 if storage == "fp32" else 2
        b_cell = 2 * Q * 2 * elem
        achieved = b_cell * cells / (launch_ms * 1e-3) / 1e9
        results[storage] = dict(total_ms=total_ms, launch_ms=launch_ms, steps=steps, clocks=clk,
                                mlups=whole_job_mlups(ws, cells, steps, total_ms * 1e-3), b_cell=b_cell,
                                achieved=achieved)
        sim.close()
        del sim
        torch.cuda.empty_cache()
    # end to end through the C ABI with host buffers: H2D of the fields, K steps, D2H of rho, u, T
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    h_rho, h_u, h_T = pin(rho), pin(u), pin(T)
    o_rho, o_u, o_T = (torch.empty(s, dtype=torch.float64).pin_memory() for s in ((n, n), (2, n, n), (n, n)))
    sim = lbm.Simulation(nx=n, ny=n, storage="fp32", **PARAMS)
    ptr = lambda t: t.numpy()
    lbm.lbm_init_fields(sim.h, ptr(h_rho), ptr(h_u), ptr(h_T))
    lbm.lbm_step(sim.h, args.warmup)
    lbm.lbm_moments(sim.h, ptr(o_rho), ptr(o_u), ptr(o_T))
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    lbm.lbm_init_fields(sim.h, ptr(h_rho), ptr(h_u), ptr(h_T))
    lbm.lbm_step(sim.h, args.steps)
    lbm.lbm_moments(sim.h, ptr(o_rho), ptr(o_u), ptr(o_T))
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(torch, e2e_s, ws)
    sim.close()
    h2d = 8 * cells * 4
    d2h = 8 * cells * 4
    extra = {}
    if ws == 1 and args.extras == "all":
        # the other configurations, measured at one GPU only (they hold no other rank)
        _extra(extra, "accuracy", lambda: accuracy_vs_oracle(lbm))
        _extra(extra, "d3q103_256", lambda: bench_3d(torch, lbm, max(args.steps // 8, 20), args.warmup, peak))
        _extra(extra, "batched_sweep", lambda: bench_batch(torch, lbm, max(args.steps // 2, 100), peak))
        _extra(extra, "couette_grid", lambda: bench_couette(lbm))
        _extra(extra, "warm_start", lambda: bench_warm_start(lbm))
        _extra(extra, "shock_tube_d2q33", lambda: bench_shock_tube(torch, lbm, peak))
        _extra(extra, "mode_study", lambda: bench_mode_study(lbm))
        _extra(extra, "burnett_d2q77", lambda: bench_burnett(torch, lbm, peak))
        cpu = oracle_mlups()
        _extra(cpu, "workloads", oracle_baselines)
        extra["cpu_baseline"] = cpu
    if rank != 0:
        return
    r32 = results["fp32"]
    traffic = profiled_traffic("k_stream_collide<D2Q37,fp32,periodic>")
    line = {
        "metric": METRIC, "value": r32["mlups"], "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r32["total_ms"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload("fp32"), "lattice": "D2Q37", "grid": [n, n], "storage": "fp32",
                   "parallelism": f"{ws} independent replica(s), one domain per GPU",
                   "l2": "inputs larger than L2: two 4.97 GB FP32 population buffers, no flush needed"},
        "roofline": {"bound": "hbm", "achieved": r32["achieved"], "peak": peak, "unit": "GB/s",
                     "frac": r32["achieved"] / peak, "traffic": traffic,
                     "kernel": "k_stream_collide<D2Q37,fp32,periodic>",
                     "algorithmic_bytes_per_cell": r32["b_cell"], "launch_ms": r32["launch_ms"],
                     "peak_kind": f"{peak_kind} hbm_gbs"},
        "clocks": r32["clocks"],
        "gpu_launches": args.steps,
        "e2e": {"value": whole_job_mlups(ws, cells, args.steps, e2e_s), "unit": "MLUPS",
                "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
                "what": "lbm_init_fields from pinned host rho,u,T + K steps + lbm_moments of rho,u,T to pinned "
                        "host; bytes per step are the field copies divided by K"},
    }
    variants = {s: {"mlups": results[s]["mlups"], "ms_per_step": results[s]["total_ms"] / results[s]["steps"],
                    "launch_ms": results[s]["launch_ms"], "achieved_gbs": results[s]["achieved"],
                    "frac": results[s]["achieved"] / peak, "algorithmic_bytes_per_cell": results[s]["b_cell"],
                    "steps": results[s]["steps"]} for s in ("fp16", "bf16")}
    if args.details:
        full = dict(line, storage_variants=variants, **extra)
        with open(args.details, "w") as f:
            json.dump(full, f, indent=1, default=float)
    # the line: headline keys first, then each extra's short form, the storage forms last
    # (the headline keys unrounded; the extras to four significant digits)
    if "cpu_baseline" in extra:
        line["cpu_baseline"] = sig(summarize("cpu_baseline", extra.pop("cpu_baseline")))
    for name in ("mode_study", "shock_tube_d2q33", "batched_sweep", "couette_grid", "burnett_d2q77", "warm_start",
                 "d3q103_256", "accuracy"):
        if name in extra:
            line[name] = sig(summarize(name, extra.pop(name)))
    line.update(sig(extra))
    line["storage_variants"] = sig({s: {k: v[k] for k in ("mlups", "frac", "launch_ms")} for s, v in variants.items()})
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--extras", default="all", choices=["all", "none"],
                    help="none: only the timed 4096^2 runs (for profiler launch lists)")
    ap.add_argument("--details", default=None,
                    help="write every measurement in full (per-case arrays included) to this JSON file")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
