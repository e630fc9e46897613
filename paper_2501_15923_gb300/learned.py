"""Learned closure of a 2x-coarser solve: pair generation, training, evaluation (orchestration).

Everything numeric runs in libicarus kernels (solver steps, restriction, the network's forward /
backward / Adam on the tensor cores, the correction); this module only sequences the calls and
keeps the training pairs in device memory (PyTorch tensors).

Pairs. From a fine state F(t0) on the fine grid: C0 = R(F(t0)) (volume-weighted restriction onto
the coarse grid), C10 = 10 coarse steps from C0 reaching t0 + T; the fine solve continues to
exactly t0 + T; the target is dU = R(F(t0 + T)) - C10. Consecutive windows of one fine run give
consecutive pairs (the end of one window is the start of the next), after a spin-up from the
initial state. The network maps the normalised C10 to the normalised dU.

Use. Every k = 10 coarse steps the correction is added to the coarse state. The reference is the
plain fine solve: relative L2 errors of v_r, n and |B| at the probes (series interpolated onto a
common hourly grid) and of the restricted state on the whole grid; if the corrected run's probe
error exceeds the threshold (1 %), the result falls back to the plain fine solve.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import icarus as ic
from . import inputs as I


def coarse_grid(g: I.Grid) -> I.Grid:
    assert g.n1 % 2 == 0 and g.n2 % 2 == 0 and g.n3 % 2 == 0
    return I.Grid(g.n1 // 2, g.n2 // 2, g.n3 // 2, g.geometry, g.stretch, g.x1min, g.x1max, g.x2min, g.x2max,
                  g.x3min, g.x3max, g.bc)


def coarse_workload(w: I.Workload) -> I.Workload:
    """Same drivers on the coarse grid: each coarse boundary column takes the mean of the 2x2 fine
    columns it covers (input preparation, on the host)."""
    m = w.maps
    mc = 0.25 * (m[:, :, 0::2, 0::2] + m[:, :, 1::2, 0::2] + m[:, :, 0::2, 1::2] + m[:, :, 1::2, 1::2])
    return I.Workload(w.name + "_coarse", coarse_grid(w.grid), w.opts, w.gamma, w.omega, w.t_maps, mc, w.cmes,
                      w.traj, w.t_end, w.n_steps, dict(w.meta))


def advance_to(s: ic.Solver, t_target: float, chunk: int = 16, max_chunks: int = 100000):
    """Step a solver until its time reaches t_target exactly (dt capped at the target)."""
    s.set_stop_time(t_target)
    for _ in range(max_chunks):
        t, dt = s.time()
        if t >= t_target * (1 - 1e-15) or dt <= 0.0:
            break
        n = max(1, min(chunk, int(math.ceil((t_target - t) / dt)) + 1))
        s.step(n)
    s.set_stop_time(0.0)


class PairSet:
    """Training pairs (C10, dU) as device tensors [8][n3][n2][n1] (float64)."""

    def __init__(self, torch):
        self.torch = torch
        self.inputs, self.targets = [], []

    def __len__(self):
        return len(self.inputs)

    def add(self, U_dev, dU_dev):
        self.inputs.append(U_dev)
        self.targets.append(dU_dev)


def generate_pairs(seeds, windows: int, spinup_days: float, k: int = 10, fine=(512, 64, 128), log=None):
    """Pairs from fine FP64 runs with production drivers (10 daily maps, one cone CME) of the given seeds."""
    import torch
    pairs = PairSet(torch)
    for seed in seeds:
        w = I.dynamic_cme(seed=seed, grid=I.Grid(*fine))
        wc = coarse_workload(w)
        F = ic.from_workload(w, precision=ic.ICARUS_FP64)
        Cs = ic.from_workload(wc, precision=ic.ICARUS_FP64)
        Ct = ic.from_workload(wc, precision=ic.ICARUS_FP64)
        t0 = spinup_days * I.DAY / F.scales()["t0"]
        advance_to(F, t0)
        shape = (8, wc.grid.n3, wc.grid.n2, wc.grid.n1)
        for _ in range(windows):
            ic.icarus_restrict(F.ctx, Cs.ctx)
            Cs.step(k)
            tc, _ = Cs.time()
            advance_to(F, tc)
            ic.icarus_restrict(F.ctx, Ct.ctx)
            U = torch.empty(shape, dtype=torch.float64, device="cuda")
            V = torch.empty(shape, dtype=torch.float64, device="cuda")
            ic.icarus_copy_state(Cs.ctx, U.data_ptr())
            ic.icarus_copy_state(Ct.ctx, V.data_ptr())
            pairs.add(U, V - U)
        if log:
            log(f"seed {seed}: {windows} pairs, fine t = {F.time()[0] * F.scales()['t0'] / I.DAY:.3f} d")
        F.close(); Cs.close(); Ct.close()
    return pairs


def normalisation(pairs: PairSet, n_sample: int = 32):
    """Per field and radial index: mean and RMS deviation of the inputs, RMS of the targets."""
    idx = np.linspace(0, len(pairs) - 1, min(n_sample, len(pairs))).astype(int)
    X = np.stack([pairs.inputs[q].cpu().numpy() for q in idx])     # [S][8][n3][n2][n1]
    Y = np.stack([pairs.targets[q].cpu().numpy() for q in idx])
    mean = X.mean(axis=(0, 2, 3))
    scale = np.sqrt(((X - mean[None, :, None, None, :]) ** 2).mean(axis=(0, 2, 3)))
    oscale = np.sqrt((Y ** 2).mean(axis=(0, 2, 3)))
    floor = lambda a: np.maximum(a, 1e-12 * max(a.max(), 1e-300))
    return mean, floor(scale), floor(oscale)


def train(pairs: PairSet, shape, epochs: int = 10, lr: float = 1e-3, seed: int = 7, log=None):
    n1, n2, n3 = shape
    net = ic.Closure(n1, n2, n3, seed=seed)
    mean, scale, oscale = normalisation(pairs)
    net.set_norm(mean, scale, oscale)
    rng = np.random.default_rng(seed)
    history = []
    t0 = time.perf_counter()
    for ep in range(epochs):
        losses = []
        lr_ep = lr * (0.5 * (1 + math.cos(math.pi * ep / max(epochs, 1))))
        for q in rng.permutation(len(pairs)):
            losses.append(net.train_step(pairs.inputs[q].data_ptr(), pairs.targets[q].data_ptr(), lr_ep))
        history.append(float(np.mean(losses)))
        if log:
            log(f"epoch {ep}: loss {history[-1]:.4e}")
    return net, dict(loss=history, seconds=time.perf_counter() - t0, steps=epochs * len(pairs),
                     norm=(mean, scale, oscale))


def probe_series(solver: ic.Solver):
    rec, n = solver.sample(None, cap=1 << 20)
    return rec[:n]


def series_error(ref, got, fields=(1, 2, 9)):
    """Relative L2 error per probe quantity (n, v_r, |B|) after interpolating both series onto a
    common hourly grid within their overlap."""
    t_lo = max(ref[0, 0, 0], got[0, 0, 0])
    t_hi = min(ref[-1, 0, 0], got[-1, 0, 0])
    grid = np.arange(t_lo, t_hi + 1e-9, 3600.0)
    out = {}
    for f in fields:
        num = den = 0.0
        for p in range(ref.shape[1]):
            a = np.interp(grid, ref[:, p, 0], ref[:, p, f])
            b = np.interp(grid, got[:, p, 0], got[:, p, f])
            num += ((b - a) ** 2).sum()
            den += (a ** 2).sum()
        out[{1: "n", 2: "v_r", 9: "|B|"}[f]] = math.sqrt(num / max(den, 1e-300))
    return out


def evaluate(net, seed: int, spinup_days: float, window_days: float, k: int = 10, fine=(512, 64, 128),
             threshold: float = 0.01, n_scale: float = 1.0, log=None):
    """Fine plain solve vs coarse plain solve vs coarse + closure on a held-out seed (n_scale: the
    boundary density factor of the drivers)."""
    import torch
    w = I.dynamic_cme(seed=seed, grid=I.Grid(*fine), n_scale=n_scale)
    wc = coarse_workload(w)
    F = ic.from_workload(w, precision=ic.ICARUS_FP64)
    t_start = spinup_days * I.DAY / F.scales()["t0"]
    advance_to(F, t_start)
    runs = {}
    for name in ("coarse", "coarse+closure"):
        C = ic.from_workload(wc, precision=ic.ICARUS_FP64)
        ic.icarus_restrict(F.ctx, C.ctx)
        runs[name] = C
    t_end = t_start + window_days * I.DAY / F.scales()["t0"]
    # fine reference with probes; at every hour the fine state is also restricted onto the coarse
    # grid and sampled there: the probe error of the exact restriction, the smallest any coarse
    # state can reach at the probes (what is left is the coarse grid's interpolation at the probe)
    F.sample(w.traj, cap=1)
    Rs = ic.from_workload(wc, precision=ic.ICARUS_FP64)

    def restricted_sample():
        ic.icarus_restrict(F.ctx, Rs.ctx)
        rec, n = Rs.sample(w.traj, cap=4)       # registers the probes, samples once, drains
        return rec[:n]

    restricted = [restricted_sample()]
    torch.cuda.synchronize()
    tf = time.perf_counter()
    hour = 3600.0 / F.scales()["t0"]
    t_next = t_start
    fine_seconds = 0.0
    while t_next < t_end * (1 - 1e-15):
        t_next = min(t_next + hour, t_end)
        t1 = time.perf_counter()
        advance_to(F, t_next)
        torch.cuda.synchronize()
        fine_seconds += time.perf_counter() - t1
        restricted.append(restricted_sample())
    ref = probe_series(F)
    Rs.close()
    fine_steps = len(ref) - 1
    result = {"fine_steps": fine_steps, "fine_seconds": fine_seconds, "fine_cells": w.grid.ncell,
              "restricted_fine": {"probe_error": series_error(ref, np.concatenate(restricted))}}
    if log:
        log(f"restricted fine state sampled on the coarse grid: {result['restricted_fine']}")
    shape_c = (8, wc.grid.n3, wc.grid.n2, wc.grid.n1)
    Rf = ic.from_workload(wc, precision=ic.ICARUS_FP64)
    ic.icarus_restrict(F.ctx, Rf.ctx)
    Uref, _ = Rf.get_state()
    for name, C in runs.items():
        C.sample(w.traj, cap=1)
        C.set_stop_time(t_end)
        torch.cuda.synchronize()
        tc = time.perf_counter()
        steps = 0
        while True:
            t, dt = C.time()
            if t >= t_end * (1 - 1e-15) or dt <= 0.0:
                break
            C.step(k)
            steps += k
            if name == "coarse+closure":
                net.apply(C.ctx)
        torch.cuda.synchronize()
        secs = time.perf_counter() - tc
        got = probe_series(C)
        U, _ = C.get_state()
        grid_err = {v: float(np.linalg.norm(U[q] - Uref[q]) / np.linalg.norm(Uref[q]))
                    for q, v in ((0, "rho"), (4, "e"))}
        result[name] = {"probe_error": series_error(ref, got), "grid_error": grid_err, "seconds": secs,
                        "coarse_steps": steps,
                        "fine_equivalent_mcell_updates_per_s": w.grid.ncell * fine_steps / secs / 1e6}
        if log:
            log(f"{name}: {result[name]}")
        C.close()
    worst = max(result["coarse+closure"]["probe_error"][q] for q in ("n", "v_r"))
    result["fallback_to_fine"] = bool(worst > threshold)
    result["closure_gain"] = {q: result["coarse"]["probe_error"][q] / max(result["coarse+closure"]["probe_error"][q], 1e-300)
                              for q in ("n", "v_r", "|B|")}
    result["fine_mcell_updates_per_s"] = w.grid.ncell * fine_steps / fine_seconds / 1e6
    F.close(); Rf.close()
    return result


def save_closure(path: str, net, norm, k: int):
    """The trained network (FP32 master weights of the four layers), its normalisation and its
    correction interval, as one .npz file."""
    arrays = {"k": np.array(k), "shape": np.array(net.shape)}
    for l, (w, b) in enumerate(net.weights()):
        arrays[f"w{l}"], arrays[f"b{l}"] = w, b
    arrays["in_mean"], arrays["in_scale"], arrays["out_scale"] = norm
    np.savez_compressed(path, **arrays)


def load_closure(path: str):
    """(network on the GPU, correction interval k) from a file written by save_closure."""
    z = np.load(path)
    n1, n2, n3 = (int(x) for x in z["shape"])
    net = ic.Closure(n1, n2, n3, seed=0)
    net.set_norm(z["in_mean"], z["in_scale"], z["out_scale"])
    net.set_weights([(z[f"w{l}"], z[f"b{l}"]) for l in range(4)])
    return net, int(z["k"])


def pair_gain(net, pairs: PairSet, indices):
    """||dU|| / ||dU - predicted dU|| over the given pairs (> 1: the correction helps)."""
    import torch
    num = den = 0.0
    for q in indices:
        out = torch.empty_like(pairs.targets[q])
        net.predict(pairs.inputs[q].data_ptr(), out.data_ptr())
        torch.cuda.synchronize()
        d = pairs.targets[q]
        den += float(torch.linalg.vector_norm(d - out)) ** 2
        num += float(torch.linalg.vector_norm(d)) ** 2
    return math.sqrt(num / max(den, 1e-300))


FLOPS_PER_VOXEL = 2 * 27 * (8 * 32 + 32 * 32 + 32 * 32 + 32 * 8)   # forward of the unpadded network


def time_network(shape=(256, 32, 64), reps: int = 20, seed: int = 5):
    """CUDA-event time of one prediction (forward + normalisation) and of one training step on a
    coarse grid of the given shape, random weights and inputs; with the tensor-core rate of the
    forward from the network's algorithmic flops."""
    import torch
    n1, n2, n3 = shape
    net = ic.Closure(n1, n2, n3, seed=seed, stream=torch.cuda.current_stream().cuda_stream)
    net.set_norm(np.zeros((8, n1)), np.ones((8, n1)), np.ones((8, n1)))
    g = torch.Generator(device="cuda").manual_seed(seed)
    U = torch.randn((8, n3, n2, n1), dtype=torch.float64, device="cuda", generator=g)
    dU = torch.randn((8, n3, n2, n1), dtype=torch.float64, device="cuda", generator=g) * 0.01
    out = torch.empty_like(U)
    res = {}
    for name, fn in (("predict", lambda: net.predict(U.data_ptr(), out.data_ptr())),
                     ("train_step", lambda: net.train_step(U.data_ptr(), dU.data_ptr(), 1e-4))):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        res[name + "_ms"] = e0.elapsed_time(e1) / reps
    vox = n1 * n2 * n3
    res["predict_tflops"] = FLOPS_PER_VOXEL * vox / (res["predict_ms"] * 1e-3) / 1e12
    res["train_step_tflops"] = 3 * FLOPS_PER_VOXEL * vox / (res["train_step_ms"] * 1e-3) / 1e12
    res["shape"] = list(shape)
    net.close()
    return res


def main(argv=None):
    """Full pipeline at production size: pairs, training, held-out evaluation; prints JSON."""
    import argparse
    import json
    import torch
    p = argparse.ArgumentParser()
    p.add_argument("--seeds", type=int, default=8)
    p.add_argument("--windows", type=int, default=25)
    p.add_argument("--spinup", type=float, default=0.25)
    p.add_argument("--epochs", type=int, default=20)
    p.add_argument("--lr", type=float, default=1e-3)
    p.add_argument("--eval-window", type=float, default=1.0)
    p.add_argument("--fine", default="512x64x128")
    p.add_argument("--every", type=int, default=10, help="coarse steps per pair window and between corrections")
    p.add_argument("--save", default="", help="write the trained network to this .npz file")
    p.add_argument("--time-only", action="store_true", help="only time the network kernels on the coarse grid")
    p.add_argument("--load", default="", help="evaluate a network saved with --save instead of training one")
    p.add_argument("--n-scale", type=float, default=1.0, help="boundary density factor of the evaluation drivers")
    a = p.parse_args(argv)
    fine = tuple(int(x) for x in a.fine.split("x"))
    torch.cuda.set_device(0)
    if a.time_only:
        print(json.dumps(time_network((fine[0] // 2, fine[1] // 2, fine[2] // 2))))
        return
    log = lambda s: print(s, flush=True)
    if a.load:
        net, k = load_closure(a.load)
        ev = evaluate(net, 999, a.spinup, a.eval_window, k=k, fine=fine, n_scale=a.n_scale, log=log)
        print(json.dumps({"every": k, "n_scale": a.n_scale, "evaluation": ev}, default=float))
        return
    t0 = time.perf_counter()
    pairs = generate_pairs(range(100, 100 + a.seeds), a.windows, a.spinup, k=a.every, fine=fine, log=log)
    t_pairs = time.perf_counter() - t0
    hold = list(range(len(pairs) - a.windows, len(pairs)))           # the last seed's pairs: held out
    train_set = PairSet(torch)
    for q in range(len(pairs) - a.windows):
        train_set.add(pairs.inputs[q], pairs.targets[q])
    cshape = (fine[0] // 2, fine[1] // 2, fine[2] // 2)
    net, info = train(train_set, cshape, epochs=a.epochs, lr=a.lr, log=log)
    gain_train = pair_gain(net, train_set, range(0, len(train_set), max(1, len(train_set) // 16)))
    gain_hold = pair_gain(net, pairs, hold)
    ev = evaluate(net, 999, a.spinup, a.eval_window, k=a.every, fine=fine, log=log)
    if a.save:
        save_closure(a.save, net, info["norm"], a.every)
    out = {"every": a.every, "pairs": len(pairs), "train_pairs": len(train_set), "pair_seconds": t_pairs,
           "train_seconds": info["seconds"], "train_steps": info["steps"], "loss_first": info["loss"][0],
           "loss_last": info["loss"][-1], "pair_gain_train": gain_train, "pair_gain_heldout": gain_hold,
           "evaluation": ev}
    print(json.dumps(out, default=float))


if __name__ == "__main__":
    main()
