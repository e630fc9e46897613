"""The paper-shaped long runs (orchestration only), in FP64 and in the MIXED form, with wall-clock
times, throughput, floor counts and the MIXED form's errors against FP64 along the probe series
and on the grid at the end:

  2019: the dynamic-boundary solar-wind case at its grid and map cadence (inputs.paper2019:
        uniform 600 x 64 x 192, 454 maps at 2 h, 42 simulated days); the paper ran it on 216 CPU
        cores in 57 min (Sect. 4, Table 1);
  2015: the dynamic case with the five CMEs of Table 2 and the CME tracer (inputs.paper2015,
        29.875 days on the same grid); the paper ran it in 1 h 4 min (Table 3).

The paper's times are context (another machine, scheme details it does not state, synthetic
inputs here).
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import icarus as ic
from . import inputs as I
from .precision import advance, advancing_steps, derived, probe_errors, rel_errors


SNAPSHOTS_2015 = (9.0, 10.3, 11.5)     # days: the paper's equatorial-plane snapshots of the CME case


def tracer_stats(c: np.ndarray) -> dict:
    return {"max": float(c.max()), "cells_above_0.5": int((c > 0.5).sum()), "cells_above_0.01": int((c > 0.01).sum())}


def run(days: float | None = None, forms=("fp64", "mixed"), chunk: int = 500, ring: int = 1 << 16, log=None,
        case: str = "2019"):
    import torch
    w = I.paper2019(days=days or 42.0) if case == "2019" else I.paper2015(days=days or 29.875)
    days = w.t_end / I.DAY
    snaps = [d for d in SNAPSHOTS_2015 if d < days] if w.opts.tracer else []
    prec = {"fp64": ic.ICARUS_FP64, "mixed": ic.ICARUS_MIXED, "fp32": ic.ICARUS_FP32}
    res, states, series, tracers = {"workload": w.name, "cells": w.grid.ncell, "maps": int(len(w.t_maps)),
                                    "days": days}, {}, {}, {}
    for name in forms:
        s = ic.from_workload(w, precision=prec[name], ring=ring)
        s.sample(w.traj, cap=1)
        t0u = s.scales()["t0"]
        recs, tracers[name] = [], []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for d in snaps + [days]:
            s.set_stop_time(d * I.DAY / t0u)
            advance(s, d * I.DAY / t0u, chunk, ring, recs)
            if w.opts.tracer:
                tracers[name].append((d, s.get_tracer()))
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
        rc, floors = s.status()
        series[name] = np.concatenate(recs)
        steps = advancing_steps(series[name])
        U, t = s.get_state()
        states[name] = derived(U, w.gamma)
        res[name] = {"seconds": secs, "steps": steps, "status": rc, "floor_hits": floors,
                     "mean_dt_s": days * I.DAY / max(steps, 1),
                     "mcell_updates_per_s": w.grid.ncell * steps / secs / 1e6,
                     "t_days": t * t0u / I.DAY}
        if w.opts.tracer:
            res[name]["tracer"] = {f"{d:g}d": tracer_stats(c) for d, c in tracers[name]}
        if log:
            log(f"{name}: {res[name]}")
        s.close()
    if "fp64" in forms:
        for name in forms:
            if name == "fp64":
                continue
            res[name]["grid_error_vs_fp64"] = rel_errors(states["fp64"], states[name])
            res[name]["probe_error_vs_fp64"] = probe_errors(series["fp64"], series[name])
            res[name]["speedup_vs_fp64"] = res[name]["mcell_updates_per_s"] / res["fp64"]["mcell_updates_per_s"]
            if w.opts.tracer:
                res[name]["tracer_vs_fp64"] = {
                    f"{d:g}d": {"max_abs": float(np.abs(c - cf).max()),
                                "cells_above_0.5_differ": int(((c > 0.5) != (cf > 0.5)).sum())}
                    for (d, c), (_, cf) in zip(tracers[name], tracers["fp64"])}
    return res


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--case", default="2019", choices=["2019", "2015"])
    p.add_argument("--days", type=float, default=None, help="default: 42 (2019) or 29.875 (2015)")
    p.add_argument("--forms", default="fp64,mixed")
    a = p.parse_args(argv)
    import torch
    torch.cuda.set_device(0)
    res = run(a.days, tuple(a.forms.split(",")), log=lambda s: print(s, flush=True), case=a.case)
    print(json.dumps(res, default=float))


if __name__ == "__main__":
    main()
