"""Throughput of the Icarus heliosphere hot path on GB300: Mcell-updates/s.

Default workload: the production-size run (512 x 64 x 128 stretched spherical grid, 0.1-2 AU,
10 daily boundary maps with a random-walk tilt, one cone CME, four probes), plain FP64. One
"step" is one solver time step: ghost fill with the time-interpolated inner boundary + CME,
reconstruction + fluxes in r, theta, phi, div B, update with sources (two SSP-RK2 stages), the
CFL reduction, and the probe sampling. The state of one copy is 296 MB, larger than the 129 MB
L2, so consecutive steps cannot run from cache (no flush needed).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the plain, untuned checker) on the host cores on a
bounded sample of the same workload; its line carries "impl": "reference". Under torchrun (N > 1)
every rank runs an independent replica on its own GPU (the single-domain solve is not sharded);
value = cell-updates of all ranks / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import platform
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2501_15923_gb300 import inputs as I  # noqa: E402

METRIC = "Mcell-updates/s on one GB300: FP64 plain vs mixed/batched/learned at stated error"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# nominal FP64 / FP32 ALU rates of GB300 (152 SMs x 2 DFMA or 128 FFMA per clock x 2070 MHz): context
# only; the roofline divides by the FMA rate measured in the same run (icarus_fma_rate)
FP64_NOMINAL_TFLOPS = 152 * 4 * 2070e6 / 1e12
FP32_NOMINAL_TFLOPS = 152 * 128 * 2 * 2070e6 / 1e12
# FP64 flops per face of the flux kernels (2 x DFMA + DADD + DMUL thread-instructions per face)
# and their DRAM bytes per face come from the committed ncu summary below.
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "k_flux_r_fp64_256x64x128.md")
KERNEL_SEQUENCES = {"default": 0, "fused": 1, "separate": 2}     # options.fused of the timed solver


def parse_args(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=80)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--grid", default="512x64x128")
    p.add_argument("--precision", default="f64", choices=["f64", "f32", "mixed"])
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline leg")
    p.add_argument("--no-forms", action="store_true", help="skip the FP32 / mixed / batched side measurements")
    p.add_argument("--tracer", action="store_true", help="carry the CME tracer in the timed solver")
    p.add_argument("--glm", action="store_true", help="GLM div-B control instead of Linde diffusion (FP64)")
    p.add_argument("--batch-members", type=int, default=64, help="members of the batched cone-CME ensemble")
    p.add_argument("--batch-only", default="", choices=["", "persistent", "phases", "concurrent"],
                   help="only step the batched ensemble in this form (2 warm-up + 3 timed steps; for profiling)")
    p.add_argument("--kernels", default="default", choices=list(KERNEL_SEQUENCES),
                   help="kernel sequence of the timed solver (options.fused): default; fused (one fused stage "
                        "kernel, FP32 / MIXED); separate (r-, theta-, phi-flux kernels and the update)")
    return p.parse_args(argv)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload(grid_s: str):
    n1, n2, n3 = (int(x) for x in grid_s.split("x"))
    return I.dynamic_cme(grid=I.Grid(n1, n2, n3))


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.proc, self.path = index, None, None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9:
                    rows.append(f)
        except OSError:
            pass
        finally:
            if self.path and os.path.exists(self.path):
                os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def kernel_source_hash():
    """Hash of the sources the FP64 flux kernels are compiled from: the physics header, the flux
    section of the kernel header (flux_tile .. k_flux) and the FP64 instantiation."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2501_15923_gb300", "csrc")
    for f in ("icarus_internal.cuh", "icarus_kernels.cuh", "kern_fp64.cu"):
        txt = open(os.path.join(csrc, f), "rb").read()
        if f == "icarus_kernels.cuh":
            a = txt.index(b"__device__ __forceinline__ void flux_tile(")
            b = txt.index(b"// div B at every cell")
            txt = txt[a:b]
        h.update(txt)
    return h.hexdigest()[:16]


def profile_numbers():
    """FP64 flops/face and DRAM bytes/face of the flux kernels from the committed ncu summary; both
    are dropped when the kernel sources changed since the capture (the counts would be another
    kernel's)."""
    try:
        txt = open(PROFILE_SUMMARY).read()
    except OSError:
        return {}, {}, {}
    vals = {}
    for line in txt.splitlines():
        if line.startswith("machine:"):
            for kv in line[len("machine:"):].split(";"):
                if "=" in kv:
                    k, v = kv.split("=", 1)
                    vals[k.strip()] = v.strip()
    flops = {d: float(vals[f"fp64_flops_per_face_{d[0]}"]) for d in ("r", "theta", "phi")
             if f"fp64_flops_per_face_{d[0]}" in vals}
    dram = {d: float(vals[f"dram_bytes_per_face_{d[0]}"]) for d in ("r", "theta", "phi")
            if f"dram_bytes_per_face_{d[0]}" in vals}
    pipe = {d: float(vals[f"fp64_pipe_busy_{d[0]}"]) / 100.0 for d in ("r", "theta", "phi")
            if f"fp64_pipe_busy_{d[0]}" in vals}
    if vals.get("kernel_hash") != kernel_source_hash():
        return {}, {}, {}
    return flops, dram, pipe


# ---------------------------------------------------------------------------------------------
def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.machine()


def cpu_oracle_rate(w, steps: int, max_seconds: float = 30.0, min_seconds: float = 12.0, threads: int = 0):
    """Time the FP64 oracle as it stands on the host cores (OpenMP; all cores, or `threads`): at
    least `steps` full steps, continued until about min_seconds of CPU work, never beyond
    max_seconds. Returns (Mcell-updates/s, steps, seconds, threads used)."""
    from oracle.oracle import from_workload as ofw, set_threads
    used = set_threads(threads if threads > 0 else (os.cpu_count() or 1))
    o = ofw(w)
    t0 = time.perf_counter()
    n = 0
    while n < steps or time.perf_counter() - t0 < min_seconds:
        o.step()
        n += 1
        if time.perf_counter() - t0 > max_seconds:
            break
    el = time.perf_counter() - t0
    return w.grid.ncell * n / el / 1e6, n, el, used


def cpu_small_case_full():
    """The oracle on the small static-sheet workload (60 x 16 x 32, its 200 steps) in full, on all
    host cores and on one thread."""
    from oracle.oracle import from_workload as ofw, set_threads
    from paper_2501_15923_gb300 import inputs as I
    w0 = I.static_sheet()
    out = {"workload": "static_sheet_60x16x32", "steps": w0.n_steps}
    for label, thr in (("all_cores", os.cpu_count() or 1), ("single_thread", 1)):
        used = set_threads(thr)
        o = ofw(w0)
        t0 = time.perf_counter()
        for _ in range(w0.n_steps):
            o.step()
        el = time.perf_counter() - t0
        out[label] = {"value": w0.grid.ncell * w0.n_steps / el / 1e6, "threads": used, "seconds": el}
    return out


def run_reference(args):
    rank, world, _ = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        if rank != 0:
            dist.barrier()
            return
    w = workload(args.grid)
    cores = os.cpu_count()
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    from oracle.oracle import from_workload as ofw, set_threads
    cores = set_threads(cores)
    o = ofw(w)
    for _ in range(args.warmup):
        o.step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.step()
    el = time.perf_counter() - t0
    v = w.grid.ncell * args.steps / el / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Mcell-updates/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "grid": args.grid, "precision": "f64"},
            "cpu_baseline": {"value": v, "unit": "Mcell-updates/s", "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} full steps of {w.name} ({w.grid.ncell} cells) after {args.warmup} warm-up steps"},
            "e2e": {"value": v, "unit": "Mcell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def run_batched(ic, torch, args):
    """Cone-CME ensemble (seed 3, uneven grids) in mixed precision, each member with its own dt,
    advanced four ways on the same members: the batched step as ONE persistent launch, as one launch
    per phase over all members, as the members' own kernels in parallel branches of one graph (the
    library default), and (the baseline) every member stepped alone through icarus_step, one after
    another. value = sum of member cells x steps / time of the default form."""
    members = I.ensemble(seed=3, n_members=args.batch_members)
    b = ic.Batch(members, precision=ic.ICARUS_MIXED)
    b.register_probes()
    tiles = b.autotune(2)
    steps = max(2, min(args.steps, 10))
    cells = b.ncell

    def timed(fn):
        fn(max(1, args.warmup))
        torch.cuda.synchronize()
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(b.stream)
        fn(steps)
        e.record(b.stream)
        e.synchronize()
        ms = a.elapsed_time(e)
        rc = b.status()
        if rc != 0:
            raise RuntimeError(f"batched ensemble status {rc}")
        return {"value": cells * steps / (ms * 1e-3) / 1e6, "ms_per_step": ms / steps}

    res = {}
    for name, mode in (("persistent", ic.ICARUS_BATCH_PERSISTENT), ("phases", ic.ICARUS_BATCH_PHASES),
                       ("concurrent", ic.ICARUS_BATCH_CONCURRENT)):
        b.set_mode(mode)
        if mode == ic.ICARUS_BATCH_PHASES:
            res["phase_tiles"] = b.autotune(2)[0]
        res[name] = timed(b.step)
        res[name]["launches_per_step"] = {ic.ICARUS_BATCH_PERSISTENT: 1, ic.ICARUS_BATCH_PHASES: 18,
                                          ic.ICARUS_BATCH_CONCURRENT: 17 * len(members)}[mode]
    res["sequential"] = timed(b.step_sequential)
    res["sequential"]["launches_per_step"] = len(members) * 17
    default = "concurrent"      # the library's default form (icarus_batch_set_mode)
    info = b.info()
    dts = sorted(b.time(m)[1] for m in range(len(members)))
    out = {"value": res[default]["value"], "unit": "Mcell-updates/s", "mode": default, "members": len(members),
           "cells": cells, "steps": steps, "ms_per_step": res[default]["ms_per_step"], "status": 0,
           "persistent_blocks": info["blocks"], "graph": info["graph"], "modes": res,
           "batched_over_sequential": {k: res[k]["value"] / res["sequential"]["value"] for k in ("persistent", "phases", "concurrent")},
           "phase_tiles": res.pop("phase_tiles", None),
           "tiles_chosen": {f"{r}/{t}": sum(1 for x in tiles if x == (r, t)) for r in range(3) for t in range(2)
                            if any(x == (r, t) for x in tiles)},
           "member_dt_range_code": [dts[0], dts[-1]]}
    b.close()
    return out


def run_batch_only(ic, torch, args):
    """The batched ensemble in one form only, 2 warm-up and 3 timed steps (a profiling target)."""
    members = I.ensemble(seed=3, n_members=args.batch_members)
    b = ic.Batch(members, precision=ic.ICARUS_MIXED)
    b.register_probes()
    b.autotune(2)
    mode = {"persistent": ic.ICARUS_BATCH_PERSISTENT, "phases": ic.ICARUS_BATCH_PHASES,
            "concurrent": ic.ICARUS_BATCH_CONCURRENT}[args.batch_only]
    b.set_mode(mode)
    if mode == ic.ICARUS_BATCH_PHASES:
        b.autotune(2)
    b.step(2)
    torch.cuda.synchronize()
    a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(b.stream)
    b.step(3)
    e.record(b.stream)
    e.synchronize()
    print(json.dumps({"batch_form": args.batch_only, "members": len(members), "ms_per_step": a.elapsed_time(e) / 3,
                      "status": b.status()}), flush=True)
    b.close()


CLOSURE_WEIGHTS = os.path.join(ROOT, "paper_2501_15923_gb300", "weights", "closure_256x32x64_k10.npz")


def run_learned(ic, torch, args):
    """The learned closure measured in this run: the committed network (trained by
    `python -m paper_2501_15923_gb300.learned --save`) corrects a 2x-coarser FP64 solve every k
    coarse steps over one simulated day of the held-out seed-999 workload (after a 0.25-day spin-up
    of the fine solve), against the plain fine FP64 solve of the same window. The probe errors of
    n, v_r and |B| at the four probes are relative L2 errors of the hourly series; the error of the
    exact restriction of the fine state (sampled on the coarse grid) is the floor any coarse state
    has. value: the fine-equivalent throughput of the corrected run when its n and v_r errors are
    within 1 %, else (fallback to the fine solve) the fine solve's own throughput."""
    from paper_2501_15923_gb300 import learned
    n1, n2, n3 = (int(x) for x in args.grid.split("x"))
    if (n1, n2, n3) != (512, 64, 128) or not os.path.exists(CLOSURE_WEIGHTS):
        return {"unavailable": "the committed closure is trained for the 512x64x128 grid"}
    net, k = learned.load_closure(CLOSURE_WEIGHTS)
    ev = learned.evaluate(net, 999, 0.25, 1.0, k=k, fine=(n1, n2, n3))
    net.close()
    cc = ev["coarse+closure"]
    worst = max(cc["probe_error"]["n"], cc["probe_error"]["v_r"])
    fallback = ev["fallback_to_fine"]
    return {"value": ev["fine_mcell_updates_per_s"] if fallback else cc["fine_equivalent_mcell_updates_per_s"],
            "unit": "Mcell-updates/s (fine-equivalent)", "fallback_to_fine": fallback,
            "accepted_if_within": 0.01, "worst_probe_error_n_vr": worst,
            "fine_equivalent_if_accepted": cc["fine_equivalent_mcell_updates_per_s"],
            "fine_plain": ev["fine_mcell_updates_per_s"], "closure_every": k,
            "probe_error": {"coarse+closure": cc["probe_error"], "coarse": ev["coarse"]["probe_error"],
                            "restricted_fine_floor": ev["restricted_fine"]["probe_error"]},
            "grid_error": {"coarse+closure": cc["grid_error"], "coarse": ev["coarse"]["grid_error"]},
            "window": "seed 999, 0.25 d -> 1.25 d", "coarse_grid": f"{n1 // 2}x{n2 // 2}x{n3 // 2}",
            "weights": os.path.relpath(CLOSURE_WEIGHTS, ROOT)}


def alu_peaks(ic, index):
    """FMA rates of this GPU measured now by the library's own kernel (icarus_fma_rate: 4 blocks of
    256 threads per SM, 8 independent chains per thread, one launch of about 60 ms after a warm-up
    launch and a calibration), with the SM clock sampled meanwhile."""
    out = {}
    with Clocks(index) as clk:
        for name, prec, it0 in (("fp64", ic.ICARUS_FP64, 1 << 12), ("fp32", ic.ICARUS_FP32, 1 << 16)):
            _, ms = ic.icarus_fma_rate(prec, 8, 4, it0)
            it = max(4, int(it0 * 60.0 / max(ms, 1e-3)) // 4 * 4)
            tf, ms = ic.icarus_fma_rate(prec, 8, 4, it)
            out[f"{name}_tflops"] = tf
            out[f"{name}_ms"] = ms
    out["clocks"] = clk.summary()
    out["source"] = "icarus_fma_rate: 4 x 256 threads per SM, 8 independent FMA chains per thread, CUDA events"
    out["nominal_tflops"] = {"fp64": FP64_NOMINAL_TFLOPS, "fp32": FP32_NOMINAL_TFLOPS}
    return out


def aggregate(ms_local: float, cells_per_rank: int, steps: int, dist=None, device=None):
    """Whole-job throughput of independent replicas: the slowest rank's time bounds the job;
    value = cells of all ranks x steps / that time (Mcell-updates/s)."""
    import torch
    world = dist.get_world_size() if dist else 1
    ms = ms_local
    if dist:
        t = torch.tensor([ms_local], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, cells_per_rank * steps * world / (ms * 1e-3) / 1e6


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    rank, world, local = dist_env()
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2501_15923_gb300 import build
    if rank == 0 or not os.path.exists(os.path.join(ROOT, "paper_2501_15923_gb300", "libicarus.so")):
        build.build()
    if dist:
        dist.barrier()
    from paper_2501_15923_gb300 import icarus as ic
    if args.batch_only:
        return run_batch_only(ic, torch, args)
    prec = {"f64": ic.ICARUS_FP64, "f32": ic.ICARUS_FP32, "mixed": ic.ICARUS_MIXED}[args.precision]
    w = workload(args.grid)
    w.opts.tracer = int(args.tracer)
    if args.glm:
        w.opts.divb = I.DIVB_GLM
    ncell = w.grid.ncell
    s = ic.from_workload(w, precision=prec, fused=KERNEL_SEQUENCES[args.kernels])
    s.sample(w.traj, cap=1)
    stream = s.stream

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    s.step(args.warmup)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        barrier()
        e0.record(stream)
        s.step(args.steps)
        e1.record(stream)
        e1.synchronize()
        barrier()
    ms = e0.elapsed_time(e1)
    rc, floor_hits = s.status()
    if rc != 0:
        raise RuntimeError(f"solver status {rc} after the timed steps")
    ms, value = aggregate(ms, ncell, args.steps, dist, torch.device("cuda", local))
    clocks = clk.summary()
    s.sample(None, cap=1 << 20)          # drain the timed steps' records

    peaks_alu = alu_peaks(ic, local)
    fp64_peak = peaks_alu["fp64_tflops"]
    # per-kernel durations (events around each launch, eager) -> roofline of the dominant kernel
    kms = s.time_kernels(3)
    per_step = {k: v * (2 if k not in ("probe", "update_1", "update_2", "fused_1", "fused_2") else 1) for k, v in kms.items()}
    dom = max(per_step, key=per_step.get)
    flops_face, dram_face, pipe_face = profile_numbers()
    n1, n2, n3 = w.grid.n1, w.grid.n2, w.grid.n3
    faces = {"flux_r": (n1 + 1) * n2 * n3, "flux_theta": n1 * (n2 + 1) * n3, "flux_phi": n1 * n2 * (n3 + 1)}
    peaks = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {}
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    dkey = dom.split("_")[-1] if dom in faces else None
    if dkey in flops_face and args.precision == "f64":
        ach = flops_face[dkey] * faces[dom] / (kms[dom] * 1e-3) / 1e12
        roof = {"kernel": f"k_flux ({dom})", "bound": "alu", "achieved": ach, "peak": fp64_peak,
                "unit": "TFLOP/s", "frac": ach / fp64_peak,
                "traffic": dram_face[dkey] * faces[dom] if dkey in dram_face else None,
                "traffic_note": "DRAM bytes/face from the 256x64x128 ncu capture scaled by the faces of one launch",
                "peak_source": "measured in this run (icarus_fma_rate, FP64 FMA chains); "
                               f"nominal {FP64_NOMINAL_TFLOPS:.3f} TFLOP/s",
                "frac_of_nominal": ach / FP64_NOMINAL_TFLOPS}
        if dkey in pipe_face:
            roof["fp64_pipe_busy"] = pipe_face[dkey]
            roof["fp64_pipe_note"] = ("sm__pipe_fp64_cycles_active of the same ncu capture: the FP64 pipe's "
                                      "issue limit; frac counts a DADD or DMUL as one flop, a DFMA as two")
    else:
        roof = {"kernel": dom, "bound": "alu", "achieved": None, "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": None, "traffic": None,
                "note": "flop count of this kernel not profiled yet (or its sources changed since the capture)"}
    bytes_cell_update = 128 if args.precision in ("f64", "mixed") else 64
    roof["hbm_view"] = {"algorithmic_bytes_per_cell_update": bytes_cell_update,
                        "achieved_gbs": value / world * 1e6 * bytes_cell_update / 1e9, "peak_gbs": hbm_peak,
                        "frac": value / world * 1e6 * bytes_cell_update / 1e9 / hbm_peak, "peak_source": "measured"}
    roof["kernel_ms"] = kms

    # end to end through the C ABI with host buffers: per step the boundary maps go host -> device
    # (icarus_set_boundary), one step runs, and the probe records come back (icarus_sample)
    maps_bytes = w.maps.nbytes + w.t_maps.nbytes + w.cmes.nbytes
    # the step's inputs sit in pinned host memory (where a producer would write them)
    maps_pinned = torch.from_numpy(np.ascontiguousarray(w.maps)).pin_memory().numpy()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ne = max(3, min(args.steps, 10))
    for _ in range(ne):
        s.set_boundary(w.t_maps, maps_pinned, w.cmes)
        s.step(1)
        rec, _ = s.sample(None, cap=4)
    el = time.perf_counter() - t0
    e2e = {"value": ncell * ne * world / el / 1e6, "unit": "Mcell-updates/s", "h2d_bytes_per_step": int(maps_bytes),
           "d2h_bytes_per_step": int(len(w.traj) * 13 * 8)}

    forms = {}
    if not args.no_forms and args.precision == "f64":
        for name, pr in (("fp32_state", ic.ICARUS_FP32), ("mixed", ic.ICARUS_MIXED)):
            sf = ic.from_workload(w, precision=pr)
            sf.step(args.warmup)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(sf.stream)
            sf.step(args.steps)
            b.record(sf.stream)
            b.synchronize()
            fms = a.elapsed_time(b)
            fval = ncell * args.steps / (fms * 1e-3) / 1e6
            forms[name] = {"value": fval, "unit": "Mcell-updates/s", "ms_per_step": fms / args.steps}
            # HBM roofline of this form's dominant kernel, from per-launch event times and the
            # algorithmic bytes of one launch (each value read or written once): flux kernels read
            # the primitives (8 x sw per cell) and write the fluxes (8 x sw per face); the update
            # reads W, U, the six face fluxes (each face shared by two cells) and div B and writes
            # U and W, plus U^n in the second stage; where the update forms the r-face fluxes
            # itself (no r-flux kernel launched), only the theta and phi face fluxes are read
            fk = sf.time_kernels(2)
            su, sw = (4, 4) if pr == ic.ICARUS_FP32 else (8, 4)
            n1, n2, n3 = w.grid.n1, w.grid.n2, w.grid.n3
            faces = {"flux_r": (n1 + 1) * n2 * n3, "flux_theta": n1 * (n2 + 1) * n3, "flux_phi": n1 * n2 * (n3 + 1)}
            kbytes = {k: 8 * sw * (ncell + f) for k, f in faces.items()}
            nfd = 3 if fk.get("flux_r", 0.0) > 0.0 else 2
            kbytes["update_1"] = ncell * (8 * sw + 8 * su + nfd * 8 * sw + sw + 8 * su + 8 * sw)
            kbytes["update_2"] = kbytes["update_1"] + ncell * 8 * su
            per_step = {k: fk[k] * (1 if k.startswith("update") else 2) for k in kbytes}
            dk = max(per_step, key=per_step.get)
            ach = kbytes[dk] / (fk[dk] * 1e-3) / 1e9
            # the form's roofline: the scope table's algorithmic bytes per cell-update (the state
            # read and written once: 8 fields of the state type each way) / the measured step time
            bcu = 2 * 8 * su
            fach = fval * 1e6 * bcu / 1e9
            forms[name]["roofline"] = {"bound": "hbm", "achieved": fach, "peak": hbm_peak, "unit": "GB/s",
                                       "frac": fach / hbm_peak, "algorithmic_bytes_per_cell_update": bcu,
                                       "peak_source": "measured (hbm_gbs)"}
            forms[name]["dominant_kernel"] = {"kernel": dk, "bound": "hbm", "achieved": ach, "peak": hbm_peak,
                                              "unit": "GB/s", "frac": ach / hbm_peak,
                                              "algorithmic_bytes": kbytes[dk], "kernel_ms": fk,
                                              "note": "this launch's own bytes (face fluxes included)"}
            sf.close()
        if args.batch_members > 0:
            forms["batched_ensemble"] = run_batched(ic, torch, args)
        forms["learned_closure"] = run_learned(ic, torch, args)

    line = {"metric": METRIC, "value": value, "unit": "Mcell-updates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
            "config": {"workload": w.name, "grid": args.grid, "cells": ncell, "precision": args.precision,
                       "l2": "inputs larger than L2 (state 8 x 8 B x padded cells per copy)",
                       "parallelism": "replicas" if world > 1 else "single GPU", "cme_tracer": bool(args.tracer),
                       "divb": "glm" if args.glm else "linde", "kernels": args.kernels},
            "clocks": clocks, "roofline": roof, "alu_peaks": peaks_alu, "e2e": e2e, "floor_hits": floor_hits,
            "gpu_launches": s.launches_per_step * args.steps, "forms": forms}
    if rank == 0 and not args.no_cpu and world == 1:
        v, n, el, used = cpu_oracle_rate(w, steps=3, max_seconds=25.0)
        v1, n1, el1, _ = cpu_oracle_rate(w, steps=1, max_seconds=20.0, min_seconds=8.0, threads=1)
        line["cpu_baseline"] = {"value": v, "unit": "Mcell-updates/s", "cores": used, "kind": "oracle",
                                "cpu_model": cpu_model(),
                                "sample": f"{n} full steps of {w.name} ({el:.1f} s, OpenMP on {used} threads)",
                                "single_thread": {"value": v1, "sample": f"{n1} full steps ({el1:.1f} s, 1 thread)"},
                                "small_case_full": cpu_small_case_full()}
    s.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
