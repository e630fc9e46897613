"""Python binding of libicarus (include/icarus.h): argument marshalling only.

Every function named icarus_* here calls the C entry point of the same name; all computation
runs in the CUDA kernels of libicarus.so. Device memory comes from PyTorch's caching allocator
(registered through the allocator callbacks of icarus_options); the solver runs on its own CUDA
stream, exposed as a torch.cuda.ExternalStream for event timing. There is no CPU fallback: if the
library is missing, loading fails with an error.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import inputs as I

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libicarus.so")

ICARUS_FP64, ICARUS_FP32, ICARUS_MIXED = 0, 1, 2
NREC = 13
ERRORS = {-1: "EINVAL", -2: "ESTATE", -3: "ENOMEM", -4: "ECUDA", -5: "ENONFINITE", -6: "ETIMEOUT"}


class IcarusError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class icarus_grid(C.Structure):
    _fields_ = [("n1", C.c_int), ("n2", C.c_int), ("n3", C.c_int), ("geometry", C.c_int), ("stretch", C.c_int),
                ("x1min", C.c_double), ("x1max", C.c_double), ("x2min", C.c_double), ("x2max", C.c_double),
                ("x3min", C.c_double), ("x3max", C.c_double), ("bc", C.c_int * 6), ("band_refine", C.c_int),
                ("band_lo", C.c_double), ("band_hi", C.c_double)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class icarus_options(C.Structure):
    _fields_ = [("cfl", C.c_double), ("limiter", C.c_int), ("flux", C.c_int), ("gravity", C.c_int),
                ("divb", C.c_int), ("divb_coef", C.c_double), ("rho_floor", C.c_double),
                ("p_floor", C.c_double), ("precision", C.c_int), ("ring_capacity", C.c_int),
                ("cuda_stream", C.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_user", C.c_void_p),
                ("fused", C.c_int), ("init_vphi", C.c_int), ("cme_model", C.c_int),
                ("tracer", C.c_int), ("glm_alpha", C.c_double), ("strict_floors", C.c_int)]


_lib = None

# exported symbols and their signatures (kept in step with include/icarus.h)
SIGNATURES = {
    "icarus_init": (C.c_int, [C.POINTER(icarus_grid), C.c_double, C.c_double, C.POINTER(icarus_options), C.POINTER(C.c_void_p)]),
    "icarus_set_boundary": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "icarus_step": (C.c_int, [C.c_void_p, C.c_int]),
    "icarus_step_recover": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.POINTER(C.c_int)]),
    "icarus_sample": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.POINTER(C.c_int)]),
    "icarus_destroy": (C.c_int, [C.c_void_p]),
    "icarus_get_state": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_double)]),
    "icarus_set_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_double]),
    "icarus_set_stop_time": (C.c_int, [C.c_void_p, C.c_double]),
    "icarus_copy_state": (C.c_int, [C.c_void_p, C.c_void_p]),
    "icarus_set_tracer": (C.c_int, [C.c_void_p, C.c_void_p]),
    "icarus_set_psi": (C.c_int, [C.c_void_p, C.c_void_p]),
    "icarus_get_psi": (C.c_int, [C.c_void_p, C.c_void_p]),
    "icarus_get_tracer": (C.c_int, [C.c_void_p, C.c_void_p]),
    "icarus_time": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "icarus_status": (C.c_int, [C.c_void_p, C.POINTER(C.c_longlong)]),
    "icarus_math_check": (C.c_int, [C.c_int, C.c_void_p, C.c_void_p]),
    "icarus_scales": (C.c_int, [C.c_void_p, C.c_void_p]),
    "icarus_launches_per_step": (C.c_int, [C.c_void_p]),
    "icarus_get_stream": (C.c_void_p, [C.c_void_p]),
    "icarus_time_kernels": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "icarus_batch_init": (C.c_int, [C.c_int, C.c_void_p, C.c_double, C.c_double, C.POINTER(icarus_options), C.POINTER(C.c_void_p)]),
    "icarus_batch_member": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_void_p)]),
    "icarus_batch_autotune": (C.c_int, [C.c_void_p, C.c_int]),
    "icarus_batch_tiles": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "icarus_batch_step": (C.c_int, [C.c_void_p, C.c_int]),
    "icarus_batch_set_tiles": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int]),
    "icarus_batch_set_mode": (C.c_int, [C.c_void_p, C.c_int]),
    "icarus_batch_status": (C.c_int, [C.c_void_p]),
    "icarus_batch_barrier_selftest": (C.c_int, [C.c_int, C.c_int, C.c_longlong]),
    "icarus_batch_info": (C.c_int, [C.c_void_p, C.c_void_p]),
    "icarus_batch_stream": (C.c_void_p, [C.c_void_p]),
    "icarus_batch_destroy": (C.c_int, [C.c_void_p]),
    "icarus_closure_create": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_ulonglong, C.c_void_p, C.POINTER(C.c_void_p)]),
    "icarus_closure_destroy": (C.c_int, [C.c_void_p]),
    "icarus_closure_wait_selftest": (C.c_int, [C.c_int, C.c_int]),
    "icarus_closure_set_norm": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "icarus_closure_train_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.POINTER(C.c_double)]),
    "icarus_closure_predict": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "icarus_closure_apply": (C.c_int, [C.c_void_p, C.c_void_p]),
    "icarus_closure_weights": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int]),
    "icarus_restrict": (C.c_int, [C.c_void_p, C.c_void_p]),
    "icarus_conv3d_layer": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int] + [C.c_void_p] * 8),
    "icarus_cfl_dt_noalloc": (C.c_int, [C.POINTER(icarus_grid), C.c_double, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p]),
    "icarus_fma_rate": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_longlong, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "icarus_last_error": (C.c_char_p, []),
}


def load():
    """Load libicarus.so (built by __graft_entry__.build() or paper_2501_15923_gb300/build.py)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libicarus.so not built at {LIB_PATH}; run __graft_entry__.build()")
        lib = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype, f.argtypes = res, args
        _lib = lib
    return _lib


def _check(rc):
    if rc != 0:
        raise IcarusError(rc, load().icarus_last_error().decode())
    return rc


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class _TorchAllocator:
    """Device memory from PyTorch's caching allocator, handed to the C library by callbacks."""

    def __init__(self, device):
        import torch
        self.torch, self.device, self.live = torch, device, {}
        self.alloc_cb = ALLOC_FN(self._alloc)
        self.free_cb = FREE_FN(self._free)

    def _alloc(self, nbytes, user):
        try:
            t = self.torch.empty(int(nbytes), dtype=self.torch.uint8, device=self.device)
        except Exception:
            return None
        self.live[t.data_ptr()] = t
        return t.data_ptr()

    def _free(self, ptr, user):
        self.live.pop(ptr, None)


def make_grid(g: I.Grid) -> icarus_grid:
    return icarus_grid(g.n1, g.n2, g.n3, g.geometry, g.stretch, g.x1min, g.x1max, g.x2min, g.x2max,
                       g.x3min, g.x3max, (C.c_int * 6)(*g.bc), g.band_refine, g.band_lo, g.band_hi)


def make_options(o: I.Options, precision=ICARUS_FP64, ring=4096, stream=None, allocator=None,
                 fused=False) -> icarus_options:
    opt = icarus_options()
    opt.fused = int(fused)           # False / 0: default kernels, True / 1: fused stage, 2: separate kernels
    opt.init_vphi = int(o.init_vphi)
    opt.cme_model = int(o.cme_model)
    opt.tracer = int(o.tracer)
    opt.glm_alpha = float(o.glm_alpha)
    opt.strict_floors = int(getattr(o, "strict_floors", 0))
    opt.cfl, opt.limiter, opt.flux, opt.gravity, opt.divb = o.cfl, o.limiter, o.flux, o.gravity, o.divb
    opt.divb_coef, opt.rho_floor, opt.p_floor = o.divb_coef, o.rho_floor, o.p_floor
    opt.precision, opt.ring_capacity = precision, ring
    opt.cuda_stream = stream
    if allocator is not None:
        opt.alloc, opt.free = allocator.alloc_cb, allocator.free_cb
    return opt


# ---- the C entry points under their own names ------------------------------------------------
def icarus_init(grid: icarus_grid, gamma: float, omega_rot: float, opts: icarus_options) -> C.c_void_p:
    ctx = C.c_void_p()
    _check(load().icarus_init(C.byref(grid), gamma, omega_rot, C.byref(opts), C.byref(ctx)))
    return ctx


def icarus_set_boundary(ctx, t_maps, maps, cmes=None):
    t_maps, maps = _f64(t_maps), _f64(maps)
    cm = _f64(cmes if cmes is not None and len(cmes) else np.zeros((0, 8)))
    _check(load().icarus_set_boundary(ctx, int(t_maps.size), _ptr(t_maps), _ptr(maps), int(cm.shape[0]),
                                      _ptr(cm) if cm.size else None))


def icarus_step(ctx, n: int = 1):
    _check(load().icarus_step(ctx, int(n)))


def icarus_step_recover(ctx, n: int = 1, max_retries: int = 3) -> int:
    """n steps with restore-and-halve-CFL retries; returns the halvings used (raises on failure)."""
    h = C.c_int(0)
    _check(load().icarus_step_recover(ctx, int(n), int(max_retries), C.byref(h)))
    return h.value


_registered_probes = {}


def icarus_sample(ctx, traj=None, cap: int = 1, out=None):
    """Returns (records [n][n_probes][13], n_written). traj registers / samples now when given."""
    lib = load()
    nw = C.c_int(0)
    key = ctx.value if isinstance(ctx, C.c_void_p) else int(ctx)
    if traj is not None:
        traj = _f64(traj)
        P, K = traj.shape[0], traj.shape[1]
        _registered_probes[key] = P
    else:
        P, K = 0, 0
    nprobe = _registered_probes.get(key, 0)
    if out is None:
        out = np.zeros((max(cap, 1), max(nprobe, 1), NREC))
    _check(lib.icarus_sample(ctx, P, K, _ptr(traj) if traj is not None else None, _ptr(out), int(cap), C.byref(nw)))
    return out[: nw.value], nw.value


def icarus_destroy(ctx):
    _check(load().icarus_destroy(ctx))


def icarus_get_state(ctx, shape):
    U = np.empty(shape)
    t = C.c_double()
    _check(load().icarus_get_state(ctx, _ptr(U), C.byref(t)))
    return U, t.value


def icarus_set_state(ctx, U, t=0.0):
    U = _f64(U)
    _check(load().icarus_set_state(ctx, _ptr(U), float(t)))


def icarus_set_tracer(ctx, c):
    c = _f64(c)
    _check(load().icarus_set_tracer(ctx, _ptr(c)))


def icarus_get_tracer(ctx, shape):
    c = np.empty(shape)
    _check(load().icarus_get_tracer(ctx, _ptr(c)))
    return c


def icarus_copy_state(ctx, U_dev_ptr):
    _check(load().icarus_copy_state(ctx, C.c_void_p(U_dev_ptr)))


def icarus_set_stop_time(ctx, t_stop):
    _check(load().icarus_set_stop_time(ctx, float(t_stop)))


def icarus_time(ctx):
    t, dt = C.c_double(), C.c_double()
    _check(load().icarus_time(ctx, C.byref(t), C.byref(dt)))
    return t.value, dt.value


def icarus_status(ctx):
    fh = C.c_longlong()
    rc = load().icarus_status(ctx, C.byref(fh))
    return rc, fh.value


def icarus_scales(ctx):
    s = np.empty(5)
    _check(load().icarus_scales(ctx, _ptr(s)))
    return dict(t0=s[0], p0=s[1], b0=s[2], omega=s[3], gm=s[4])


def icarus_launches_per_step(ctx) -> int:
    return int(load().icarus_launches_per_step(ctx))


def icarus_get_stream(ctx) -> int:
    return int(load().icarus_get_stream(ctx) or 0)


KERNEL_CLASSES = ("ghost_fill", "flux_r", "flux_theta", "flux_phi", "divb", "update_1", "update_2", "probe",
                  "fused_1", "fused_2")


def icarus_time_kernels(ctx, n_steps: int) -> dict:
    ms = np.zeros(len(KERNEL_CLASSES))
    _check(load().icarus_time_kernels(ctx, int(n_steps), _ptr(ms)))
    return dict(zip(KERNEL_CLASSES, ms.tolist()))


def icarus_cfl_dt_noalloc(grid: icarus_grid, gamma: float, cfl: float, U_dev_ptr: int, dt_dev_ptr: int, stream=None):
    """Allocation-free CFL time step of a state the caller already holds on the device (device
    pointers in and out; see include/icarus.h)."""
    _check(load().icarus_cfl_dt_noalloc(C.byref(grid), float(gamma), float(cfl), C.c_void_p(U_dev_ptr),
                                        C.c_void_p(dt_dev_ptr), C.c_void_p(stream or 0)))


def icarus_fma_rate(precision: int, chains: int = 8, blocks_per_sm: int = 4, iters: int = 1 << 14):
    """Measured FMA rate of the GPU: (TFLOP/s, ms of the timed launch)."""
    tf, ms = C.c_double(), C.c_double()
    _check(load().icarus_fma_rate(int(precision), int(chains), int(blocks_per_sm), int(iters), C.byref(tf), C.byref(ms)))
    return tf.value, ms.value


# ---- convenience wrapper -----------------------------------------------------------------------
class Solver:
    """One solver context on the current CUDA device, memory from torch's caching allocator."""

    def __init__(self, grid: I.Grid, gamma: float, omega: float, opts: I.Options, precision=ICARUS_FP64,
                 ring=4096, device="cuda", fused=False):
        import torch
        self.torch = torch
        self.grid, self.precision = grid, precision
        self._alloc = _TorchAllocator(torch.device(device))
        self._opts = make_options(opts, precision, ring, None, self._alloc, fused)
        self._grid = make_grid(grid)
        self.ctx = icarus_init(self._grid, gamma, omega, self._opts)
        self.shape = (8, grid.n3, grid.n2, grid.n1)
        self.stream = torch.cuda.ExternalStream(icarus_get_stream(self.ctx))

    def close(self):
        if getattr(self, "ctx", None):
            icarus_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_boundary(self, t_maps, maps, cmes=None):
        icarus_set_boundary(self.ctx, t_maps, maps, cmes)

    def step(self, n=1):
        icarus_step(self.ctx, n)

    def step_recover(self, n=1, max_retries=3):
        return icarus_step_recover(self.ctx, n, max_retries)

    def sample(self, traj=None, cap=1):
        return icarus_sample(self.ctx, traj, cap)

    def get_state(self):
        return icarus_get_state(self.ctx, self.shape)

    def set_state(self, U, t=0.0):
        icarus_set_state(self.ctx, U, t)

    def set_tracer(self, c):
        """CME tracer c of the interior cells [n3][n2][n1] (rho c from the current rho)."""
        icarus_set_tracer(self.ctx, c)

    def get_tracer(self):
        return icarus_get_tracer(self.ctx, self.shape[1:])

    def set_psi(self, p):
        """GLM psi of the interior cells [n3][n2][n1] (divb = DIVB_GLM)."""
        p = _f64(p)
        _check(load().icarus_set_psi(self.ctx, _ptr(p)))

    def get_psi(self):
        p = np.empty(self.shape[1:])
        _check(load().icarus_get_psi(self.ctx, _ptr(p)))
        return p

    def set_stop_time(self, t_stop):
        icarus_set_stop_time(self.ctx, t_stop)

    def time(self):
        return icarus_time(self.ctx)

    def status(self):
        return icarus_status(self.ctx)

    def scales(self):
        return icarus_scales(self.ctx)

    def time_kernels(self, n_steps):
        return icarus_time_kernels(self.ctx, n_steps)

    @property
    def launches_per_step(self):
        return icarus_launches_per_step(self.ctx)


def from_workload(w: I.Workload, precision=ICARUS_FP64, ring=4096, fused=False) -> Solver:
    s = Solver(w.grid, w.gamma, w.omega, w.opts, precision, ring, fused=fused)
    s.set_boundary(w.t_maps, w.maps, w.cmes)
    return s


# ---- batched ensemble ---------------------------------------------------------------------------
def icarus_batch_init(grids, gamma, omega_rot, opts):
    arr = (icarus_grid * len(grids))(*grids)
    b = C.c_void_p()
    _check(load().icarus_batch_init(len(grids), C.cast(arr, C.c_void_p), gamma, omega_rot, C.byref(opts), C.byref(b)))
    return b


def icarus_batch_member(b, m):
    c = C.c_void_p()
    _check(load().icarus_batch_member(b, int(m), C.byref(c)))
    return c


def icarus_batch_autotune(b, reps=3):
    _check(load().icarus_batch_autotune(b, int(reps)))


def icarus_batch_tiles(b, m):
    cfg = np.zeros(2, dtype=np.int32)
    _check(load().icarus_batch_tiles(b, int(m), _ptr(cfg)))
    return tuple(int(x) for x in cfg)


def icarus_batch_set_tiles(b, m, cfg_r, cfg_t):
    _check(load().icarus_batch_set_tiles(b, int(m), int(cfg_r), int(cfg_t)))


def icarus_batch_step(b, n=1):
    _check(load().icarus_batch_step(b, int(n)))


def icarus_batch_status(b):
    return load().icarus_batch_status(b)


def icarus_batch_info(b):
    info = np.zeros(4, dtype=np.int32)
    _check(load().icarus_batch_info(b, _ptr(info)))
    return dict(members=int(info[0]), blocks=int(info[1]), graph=bool(info[2]), mode=int(info[3]))


ICARUS_BATCH_PERSISTENT, ICARUS_BATCH_PHASES, ICARUS_BATCH_CONCURRENT = 0, 1, 2


def icarus_batch_set_mode(b, mode):
    _check(load().icarus_batch_set_mode(b, int(mode)))


def icarus_batch_destroy(b):
    _check(load().icarus_batch_destroy(b))


class Batch:
    """An ensemble of independent members advanced together by one graph launch per step: the
    members' own kernels as parallel branches (ICARUS_BATCH_CONCURRENT, the default), one persistent
    kernel (ICARUS_BATCH_PERSISTENT) or one launch per phase over all members (ICARUS_BATCH_PHASES)."""

    def __init__(self, workloads, precision=ICARUS_MIXED, ring=4096, device="cuda", mode=None):
        import torch
        self.torch = torch
        self._alloc = _TorchAllocator(torch.device(device))
        w0 = workloads[0]
        self._opts = make_options(w0.opts, precision, ring, None, self._alloc)
        self._grids = [make_grid(w.grid) for w in workloads]
        self.b = icarus_batch_init(self._grids, w0.gamma, w0.omega, self._opts)
        self.workloads = workloads
        self.ctx = [icarus_batch_member(self.b, m) for m in range(len(workloads))]
        self.shapes = [(8, w.grid.n3, w.grid.n2, w.grid.n1) for w in workloads]
        for c, w in zip(self.ctx, workloads):
            icarus_set_boundary(c, w.t_maps, w.maps, w.cmes)
        self.stream = torch.cuda.ExternalStream(int(load().icarus_batch_stream(self.b) or 0))
        if mode is not None:
            icarus_batch_set_mode(self.b, mode)

    def set_mode(self, mode):
        icarus_batch_set_mode(self.b, mode)

    def step_sequential(self, n=1):
        """Each member advanced alone through icarus_step (its own captured step), one after another
        on the batch stream: the baseline the batched launch is measured against."""
        for _ in range(n):
            for c in self.ctx:
                icarus_step(c, 1)

    def register_probes(self):
        for c, w in zip(self.ctx, self.workloads):
            icarus_sample(c, w.traj, cap=1)

    def autotune(self, reps=3):
        icarus_batch_autotune(self.b, reps)
        return [icarus_batch_tiles(self.b, m) for m in range(len(self.ctx))]

    def set_tiles(self, cfg_r, cfg_t):
        for m in range(len(self.ctx)):
            icarus_batch_set_tiles(self.b, m, cfg_r, cfg_t)

    def step(self, n=1):
        icarus_batch_step(self.b, n)

    def status(self):
        return icarus_batch_status(self.b)

    def info(self):
        return icarus_batch_info(self.b)

    def get_state(self, m):
        return icarus_get_state(self.ctx[m], self.shapes[m])

    def set_state(self, m, U, t):
        icarus_set_state(self.ctx[m], U, t)

    def time(self, m):
        return icarus_time(self.ctx[m])

    def sample(self, m, cap=1):
        return icarus_sample(self.ctx[m], None, cap)

    @property
    def ncell(self):
        return sum(w.grid.ncell for w in self.workloads)

    def close(self):
        if getattr(self, "b", None):
            icarus_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- learned closure ----------------------------------------------------------------------------
LAYER_SHAPES = ((16, 32), (32, 32), (32, 32), (32, 16))   # padded (C_in, C_out) per layer


def icarus_conv3d_layer(x, w, b, g, act):
    """One layer through the closure's tensor-core kernels. x [n3][n2][n1][C], w [O][27][C]."""
    x, w, b, g = (np.ascontiguousarray(a, dtype=np.float32) for a in (x, w, b, g))
    n3, n2, n1, Cc = x.shape
    O = w.shape[0]
    y = np.empty((n3, n2, n1, O), np.float32)
    dx, dw, db = np.empty_like(x), np.empty_like(w), np.empty(O, np.float32)
    _check(load().icarus_conv3d_layer(n1, n2, n3, Cc, O, int(act), *(_ptr(a) for a in (x, w, b, g, y, dx, dw, db))))
    return y, dx, dw, db


def icarus_restrict(fine_ctx, coarse_ctx):
    _check(load().icarus_restrict(fine_ctx, coarse_ctx))


class Closure:
    """The learned correction network of a coarse grid (weights on the GPU)."""

    def __init__(self, n1, n2, n3, seed=0, stream=0):
        self.shape = (n1, n2, n3)
        self.h = C.c_void_p()
        _check(load().icarus_closure_create(n1, n2, n3, seed, C.c_void_p(stream), C.byref(self.h)))

    def set_norm(self, in_mean, in_scale, out_scale):
        """Per-field, per-radial-index statistics, each [8][n1] (the C call reads 8 n1 doubles)."""
        a = [np.ascontiguousarray(x, dtype=np.float64) for x in (in_mean, in_scale, out_scale)]
        if any(x.size != 8 * self.shape[0] for x in a):
            raise ValueError(f"normalisation arrays must hold 8 x n1 = {8 * self.shape[0]} values")
        _check(load().icarus_closure_set_norm(self.h, *(_ptr(x) for x in a)))

    def train_step(self, U_dev_ptr, dU_dev_ptr, lr):
        loss = C.c_double()
        _check(load().icarus_closure_train_step(self.h, C.c_void_p(U_dev_ptr), C.c_void_p(dU_dev_ptr), float(lr),
                                                C.byref(loss)))
        return loss.value

    def predict(self, U_dev_ptr, dU_dev_ptr):
        _check(load().icarus_closure_predict(self.h, C.c_void_p(U_dev_ptr), C.c_void_p(dU_dev_ptr)))

    def apply(self, ctx):
        _check(load().icarus_closure_apply(self.h, ctx))

    def weights(self):
        out = []
        for l, (ci, co) in enumerate(LAYER_SHAPES):
            w, b = np.empty((co, 27, ci), np.float32), np.empty(co, np.float32)
            _check(load().icarus_closure_weights(self.h, l, _ptr(w), _ptr(b), 0))
            out.append((w, b))
        return out

    def set_weights(self, wb):
        for l, (w, b) in enumerate(wb):
            w, b = np.ascontiguousarray(w, np.float32), np.ascontiguousarray(b, np.float32)
            _check(load().icarus_closure_weights(self.h, l, _ptr(w), _ptr(b), 1))

    def close(self):
        if getattr(self, "h", None):
            load().icarus_closure_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
