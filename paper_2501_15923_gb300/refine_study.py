"""Static refinement band against adaptive refinement's purpose (orchestration only): the
production drivers (production maps, one cone CME aimed at probe 0) on three radial grids with the
same 32 x 64 angular grid, stepped from the initial state through the CME's passage at probe 0:

  base     n1 cells, stretched;
  band     the base spacing outside a band around probe 0's orbit and band_refine times narrower
           cells inside it (n1 chosen so that the outside spacing equals the base);
  refined  band_refine x n1 cells everywhere (the reference).

Reported: wall time, cell-updates, steps, and the probe-0 series errors of base and band against
the refined run (n, v_r, |B|, RMS and max relative, on an hourly grid over the CME window).
The paper refines adaptively around the CME and near Earth (Sect. 2); this fixed band is the
structured-grid stand-in: it adds cells only where the probe is, and on a stretched grid does not
shorten dt (the inner-boundary cells stay the narrowest).
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import icarus as ic
from . import inputs as I
from .precision import advance, advancing_steps


def band_cells(n1, x1min, x1max, lo, hi, f):
    """Cells of a banded stretched grid whose outside spacing (in ln r) equals that of n1 cells."""
    u = math.log(x1max / x1min)
    return int(round(n1 * (u + (f - 1) * math.log(hi / lo)) / u))


def probe0_errors(ref, got, t_lo, t_hi):
    grid = np.arange(t_lo, t_hi + 1e-9, 3600.0)
    out = {}
    for f, name in ((1, "n"), (2, "v_r"), (9, "|B|")):
        a = np.interp(grid, ref[:, 0, 0], ref[:, 0, f])
        b = np.interp(grid, got[:, 0, 0], got[:, 0, f])
        d = np.abs(b - a)
        out[name] = {"rms_rel": float(math.sqrt((d ** 2).mean() / (a ** 2).mean())),
                     "max_rel": float((d / np.abs(a)).max())}
    return out


def run(n1=256, n2=32, n3=64, f=4, days=None, precision="fp64", chunk=500, ring=1 << 16, log=None):
    import torch
    w0 = I.dynamic_cme(grid=I.Grid(n1, n2, n3))
    traj = np.asarray(w0.traj)
    r0 = traj[0, :, 1] / I.AU
    lo, hi = float(r0.min()) - 0.15, float(r0.max()) + 0.15
    t_on = float(w0.cmes[0, 0])
    t_end = days * I.DAY if days else t_on + 2.5 * I.DAY
    nb = band_cells(n1, w0.grid.x1min, w0.grid.x1max, lo, hi, f)
    grids = {"base": I.Grid(n1, n2, n3),
             "band": I.Grid(nb, n2, n3, band_refine=f, band_lo=lo, band_hi=hi),
             "refined": I.Grid(f * n1, n2, n3)}
    prec = {"fp64": ic.ICARUS_FP64, "mixed": ic.ICARUS_MIXED, "fp32": ic.ICARUS_FP32}[precision]
    res = {"band_au": [lo, hi], "band_refine": f, "t_on_days": t_on / I.DAY, "t_end_days": t_end / I.DAY,
           "precision": precision}
    series = {}
    for name, g in grids.items():
        w = I.dynamic_cme(grid=g)
        s = ic.from_workload(w, precision=prec, ring=ring)
        s.sample(w.traj, cap=1)
        te = t_end / s.scales()["t0"]
        s.set_stop_time(te)
        recs = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        advance(s, te, chunk, ring, recs)
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
        series[name] = np.concatenate(recs)
        steps = advancing_steps(series[name])
        rc, floors = s.status()
        res[name] = {"n1": g.n1, "cells": g.ncell, "steps": steps, "seconds": secs, "status": rc,
                     "cell_updates": g.ncell * steps, "mcell_updates_per_s": g.ncell * steps / secs / 1e6}
        if log:
            log(f"{name}: {res[name]}")
        s.close()
    for name in ("base", "band"):
        res[name]["probe0_error_vs_refined"] = probe0_errors(series["refined"], series[name], t_on, t_end)
        res[name]["cost_vs_refined"] = res[name]["cell_updates"] / res["refined"]["cell_updates"]
    return res


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--n1", type=int, default=256)
    p.add_argument("--refine", type=int, default=4)
    p.add_argument("--precision", default="fp64")
    a = p.parse_args(argv)
    import torch
    torch.cuda.set_device(0)
    res = run(n1=a.n1, f=a.refine, precision=a.precision, log=lambda s: print(s, flush=True))
    print(json.dumps(res, default=float))


if __name__ == "__main__":
    main()
