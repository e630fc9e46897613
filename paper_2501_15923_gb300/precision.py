"""Precision forms against the plain FP64 solve on the same workload (orchestration only).

Runs the production-size workload (512 x 64 x 128, dynamic maps, cone CME, four probes) for the
same simulated time in FP64, MIXED (FP32 reconstruction / fluxes / sources, FP64 state, update,
dt and near-boundary pressure recovery) and FP32-state form, and reports for n, |v|, |B| and p the
maximum and RMS relative errors against FP64 on the whole grid at the end and along the probe time
series (interpolated onto a common hourly grid), with each form's throughput.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import icarus as ic
from . import inputs as I


def derived(U, gamma):
    rho = U[0]
    v = np.sqrt((U[1:4] ** 2).sum(0)) / rho
    b = np.sqrt((U[5:8] ** 2).sum(0))
    p = (gamma - 1.0) * (U[4] - 0.5 * (U[1:4] ** 2).sum(0) / rho - 0.5 * (U[5:8] ** 2).sum(0))
    return {"n": rho, "|v|": v, "|B|": b, "p": p}


def rel_errors(ref, got):
    out = {}
    for k in ref:
        a, b = ref[k], got[k]
        d = np.abs(b - a)
        out[k] = {"max_rel": float((d / np.maximum(np.abs(a), 1e-300)).max()),
                  "rms_rel": float(math.sqrt((d ** 2).mean() / (a ** 2).mean()))}
    return out


def probe_errors(ref, got):
    """Probe quantities n (1), v_r (2), |B| (9), p (8) on a common hourly grid."""
    t_lo, t_hi = max(ref[0, 0, 0], got[0, 0, 0]), min(ref[-1, 0, 0], got[-1, 0, 0])
    grid = np.arange(t_lo, t_hi + 1e-9, 3600.0)
    out = {}
    for f, name in ((1, "n"), (2, "v_r"), (9, "|B|"), (8, "p")):
        a = np.concatenate([np.interp(grid, ref[:, p, 0], ref[:, p, f]) for p in range(ref.shape[1])])
        b = np.concatenate([np.interp(grid, got[:, p, 0], got[:, p, f]) for p in range(got.shape[1])])
        d = np.abs(b - a)
        out[name] = {"max_rel": float((d / np.maximum(np.abs(a), 1e-300)).max()),
                     "rms_rel": float(math.sqrt((d ** 2).mean() / (a ** 2).mean()))}
    return out


def advance(s, t_target: float, chunk: int, ring: int, recs: list):
    """Step solver s (stop time already at or beyond t_target, code units) until t reaches
    t_target, in graph-replayed chunks of at most 95 % of the steps the remaining time allows at
    the current dt (so that, dt varying slowly, hardly any step runs at dt = 0 after the stop; the
    last steps go one at a time), draining the probe ring after each chunk."""
    while True:
        t, dt = s.time()
        if t >= t_target * (1 - 1e-15) or dt <= 0.0:
            return
        n = max(1, min(chunk, int(0.95 * (t_target - t) / dt)))
        s.step(n)
        rec, got = s.sample(None, cap=ring)
        recs.append(rec[:got])


def advancing_steps(series: np.ndarray) -> int:
    """Steps that advanced the time (probe records with a later time than the previous one)."""
    return int((np.diff(series[:, 0, 0]) > 0).sum())


def run(days: float, grid=(512, 64, 128), chunk: int = 200, ring: int = 1 << 16, n_scale: float = 1.0, log=None):
    import torch
    w = I.dynamic_cme(grid=I.Grid(*grid), days=days, n_scale=n_scale)
    res, states, series = {}, {}, {}
    for name, prec in (("fp64", ic.ICARUS_FP64), ("mixed", ic.ICARUS_MIXED), ("fp32", ic.ICARUS_FP32)):
        s = ic.from_workload(w, precision=prec, ring=ring)
        s.sample(w.traj, cap=1)
        t_end = days * I.DAY / s.scales()["t0"]
        s.set_stop_time(t_end)
        recs = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        advance(s, t_end, chunk, ring, recs)
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
        rc, floors = s.status()
        series[name] = np.concatenate(recs)
        U, t = s.get_state()
        states[name] = derived(U, w.gamma)
        ncell_steps = advancing_steps(series[name])
        res[name] = {"seconds": secs, "steps": ncell_steps, "status": rc, "floor_hits": floors,
                     "mcell_updates_per_s": w.grid.ncell * ncell_steps / secs / 1e6, "t_days": t * s.scales()["t0"] / I.DAY}
        if log:
            log(f"{name}: {res[name]}")
        s.close()
    for name in ("mixed", "fp32"):
        res[name]["grid_error_vs_fp64"] = rel_errors(states["fp64"], states[name])
        res[name]["probe_error_vs_fp64"] = probe_errors(series["fp64"], series[name])
        res[name]["speedup_vs_fp64"] = res[name]["mcell_updates_per_s"] / res["fp64"]["mcell_updates_per_s"]
    return res


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--days", type=float, default=10.0)
    p.add_argument("--grid", default="512x64x128")
    p.add_argument("--n-scale", type=float, default=1.0,
                   help="boundary density factor (2: the inflow is super-Alfvenic and no floor acts before the CME)")
    a = p.parse_args(argv)
    import torch
    torch.cuda.set_device(0)
    res = run(a.days, tuple(int(x) for x in a.grid.split("x")), n_scale=a.n_scale, log=lambda s: print(s, flush=True))
    print(json.dumps(res))


if __name__ == "__main__":
    main()
