"""ctypes wrapper of the FP64 CPU oracle (liboracle.so) -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference arm may use this
module. It takes plain numpy arrays; grids and options are passed as flat int/double arrays so
that no struct layout is shared with the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None
NV = 8
NG = 2


def lib():
    global _lib
    if _lib is None:
        # ORACLE_SO names another build of the same sources (the mutation tests load copies of
        # the oracle with one planted mistake); by default the in-tree library is built and loaded
        _lib = C.CDLL(os.environ.get("ORACLE_SO") or _build.build())
        P, D, I, L = C.c_void_p, C.c_double, C.c_int, C.c_long
        sig = {
            "orc_create": (P, [P, P, D, D, P, P]),
            "orc_destroy": (None, [P]),
            "orc_set_threads": (None, [I]),
            "orc_riemann": (None, [P, P, P, I, P]),
            "orc_set_tracer": (None, [P, P]),
            "orc_get_tracer": (None, [P, P]),
            "orc_max_threads": (I, []),
            "orc_set_boundary": (I, [P, I, P, P, I, P]),
            "orc_init_state": (I, [P]),
            "orc_set_state": (None, [P, P, D]),
            "orc_get_state": (None, [P, P, P]),
            "orc_set_state_padded": (None, [P, P, D]),
            "orc_get_state_padded": (None, [P, P]),
            "orc_fill_ghosts": (None, [P, D]),
            "orc_cfl_dt": (D, [P]),
            "orc_apply_floors": (None, [P]),
            "orc_step": (D, [P, D]),
            "orc_residual": (None, [P, D, D, P]),
            "orc_divb": (None, [P, P]),
            "orc_volumes": (None, [P, P]),
            "orc_centres": (None, [P, I, P]),
            "orc_edges": (None, [P, I, P]),
            "orc_set_psi": (None, [P, P]),
            "orc_get_psi": (None, [P, P]),
            "orc_glm_ch": (D, [P]),
            "orc_glm_dmin": (D, [P]),
            "orc_boundary_values": (None, [P, D, P, P]),
            "orc_floor_hits": (L, [P]),
            "orc_time": (D, [P]),
            "orc_scales": (None, [P, P]),
            "orc_sample": (None, [P, I, I, P, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(_lib, name)
            f.restype = res
            f.argtypes = args
        for name, args in {"orc_conv3d_forward": [P, P, P, P, I, I, I, I, I, I],
                           "orc_conv3d_backward": [P, P, P, P, P, P, P, I, I, I, I, I, I],
                           "orc_restrict": [P, P, P, I, I, I]}.items():
            f = getattr(_lib, name)
            f.restype = None
            f.argtypes = args
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _c(a, dtype=np.float64):
    return np.ascontiguousarray(a, dtype=dtype)


class Oracle:
    """One oracle solver instance. Times are code units unless a name says _si."""

    def __init__(self, grid, gamma: float, omega: float, opts):
        self.grid, self.opts = grid, opts
        ig = np.array([grid.n1, grid.n2, grid.n3, grid.geometry, grid.stretch, *grid.bc, grid.band_refine],
                      dtype=np.int32)
        dg = np.array([grid.x1min, grid.x1max, grid.x2min, grid.x2max, grid.x3min, grid.x3max,
                       grid.band_lo, grid.band_hi])
        od = np.array([opts.cfl, opts.divb_coef, opts.rho_floor, opts.p_floor, opts.glm_alpha])
        oi = np.array([opts.limiter, opts.flux, opts.gravity, opts.divb, opts.init_vphi, opts.cme_model,
                       opts.tracer], dtype=np.int32)
        self.h = lib().orc_create(_ptr(ig), _ptr(dg), gamma, omega, _ptr(od), _ptr(oi))
        self.shape = (NV, grid.n3, grid.n2, grid.n1)
        self.pshape = (NV, grid.n3 + 2 * NG, grid.n2 + 2 * NG, grid.n1 + 2 * NG)

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_destroy(self.h)
            self.h = None

    def set_boundary(self, t_maps, maps, cmes=None):
        t_maps, maps = _c(t_maps), _c(maps)
        cm = _c(cmes if cmes is not None and len(cmes) else np.zeros((0, 8)))
        lib().orc_set_boundary(self.h, int(t_maps.size), _ptr(t_maps), _ptr(maps), int(cm.shape[0]), _ptr(cm))

    def init_state(self):
        if lib().orc_init_state(self.h) != 0:
            raise RuntimeError("orc_init_state needs a spherical grid and boundary maps")

    def set_state(self, U, t=0.0):
        U = _c(U)
        assert U.shape == self.shape
        lib().orc_set_state(self.h, _ptr(U), float(t))

    def get_state(self):
        U = np.empty(self.shape)
        t = C.c_double()
        lib().orc_get_state(self.h, _ptr(U), C.byref(t))
        return U, t.value

    def set_state_padded(self, Up, t=0.0):
        Up = _c(Up)
        assert Up.shape == self.pshape
        lib().orc_set_state_padded(self.h, _ptr(Up), float(t))

    def get_state_padded(self):
        Up = np.empty(self.pshape)
        lib().orc_get_state_padded(self.h, _ptr(Up))
        return Up

    def fill_ghosts(self, tau):
        lib().orc_fill_ghosts(self.h, float(tau))

    def cfl_dt(self) -> float:
        return lib().orc_cfl_dt(self.h)

    def apply_floors(self):
        """The density and pressure floors of a stage end, applied to the interior state."""
        lib().orc_apply_floors(self.h)

    def step(self, dt_max: float = 0.0) -> float:
        dt = lib().orc_step(self.h, float(dt_max))
        if dt < 0:
            raise FloatingPointError("oracle state became non-finite")
        return dt

    def residual(self, tau, dt):
        L = np.empty(self.shape)
        lib().orc_residual(self.h, float(tau), float(dt), _ptr(L))
        return L

    def divb(self):
        out = np.empty(self.shape[1:])
        lib().orc_divb(self.h, _ptr(out))
        return out

    def volumes(self):
        out = np.empty(self.shape[1:])
        lib().orc_volumes(self.h, _ptr(out))
        return out

    def centres(self, d):
        n = (self.grid.n1, self.grid.n2, self.grid.n3)[d]
        out = np.empty(n + 2 * NG)
        lib().orc_centres(self.h, d, _ptr(out))
        return out

    def edges(self, d):
        """The n + 1 interior cell edges of direction d."""
        n = (self.grid.n1, self.grid.n2, self.grid.n3)[d]
        out = np.empty(n + 1)
        lib().orc_edges(self.h, d, _ptr(out))
        return out

    def set_psi(self, p):
        """GLM psi of the interior cells [n3][n2][n1]."""
        a = _c(p)
        assert a.shape == self.shape[1:]
        lib().orc_set_psi(self.h, _ptr(a))

    def get_psi(self) -> np.ndarray:
        out = np.empty(self.shape[1:])
        lib().orc_get_psi(self.h, _ptr(out))
        return out

    def glm_ch(self) -> float:
        return lib().orc_glm_ch(self.h)

    def glm_dmin(self) -> float:
        return lib().orc_glm_dmin(self.h)

    def boundary_values(self, tau):
        g = self.grid
        out = np.empty((5, g.n2, g.n3))
        hit = np.empty((g.n2, g.n3), dtype=np.int32)
        lib().orc_boundary_values(self.h, float(tau), _ptr(out), _ptr(hit))
        return out, hit

    def set_tracer(self, c):
        """CME tracer values c of the interior cells [n3][n2][n1] (rho c from the current rho)."""
        a = _c(c)
        assert a.shape == self.shape[1:]
        lib().orc_set_tracer(self.h, _ptr(a))

    def get_tracer(self) -> np.ndarray:
        out = np.empty(self.shape[1:])
        lib().orc_get_tracer(self.h, _ptr(out))
        return out

    def riemann(self, wl, wr, d: int) -> np.ndarray:
        """Face flux of the configured Riemann solver for primitive states wl, wr (code units)."""
        f = np.empty(8)
        a, b = _c(wl), _c(wr)
        lib().orc_riemann(self.h, _ptr(a), _ptr(b), int(d), _ptr(f))
        return f

    @property
    def floor_hits(self) -> int:
        return lib().orc_floor_hits(self.h)

    @property
    def t(self) -> float:
        return lib().orc_time(self.h)

    def scales(self):
        s = np.empty(5)
        lib().orc_scales(self.h, _ptr(s))
        return dict(t0=s[0], p0=s[1], b0=s[2], omega=s[3], gm=s[4])

    def sample(self, traj):
        traj = _c(traj)
        P, K = traj.shape[0], traj.shape[1]
        out = np.empty((P, 13))
        lib().orc_sample(self.h, P, K, _ptr(traj), _ptr(out))
        return out


def from_workload(w) -> Oracle:
    """Oracle set up with a workload's grid, options, boundary maps and initial state."""
    o = Oracle(w.grid, w.gamma, w.omega, w.opts)
    o.set_boundary(w.t_maps, w.maps, w.cmes)
    o.init_state()
    return o


def cons_from_prim(W: np.ndarray, gamma: float) -> np.ndarray:
    """Conserved variables from primitives (rho, v1, v2, v3, p, B1, B2, B3) along axis 0."""
    U = np.empty_like(W)
    U[0] = W[0]
    U[1:4] = W[0] * W[1:4]
    U[4] = W[4] / (gamma - 1.0) + 0.5 * W[0] * (W[1:4] ** 2).sum(0) + 0.5 * (W[5:8] ** 2).sum(0)
    U[5:8] = W[5:8]
    return U


def prim_from_cons(U: np.ndarray, gamma: float) -> np.ndarray:
    W = np.empty_like(U)
    W[0] = U[0]
    W[1:4] = U[1:4] / U[0]
    W[4] = (gamma - 1.0) * (U[4] - 0.5 * U[0] * (W[1:4] ** 2).sum(0) - 0.5 * (U[5:8] ** 2).sum(0))
    W[5:8] = U[5:8]
    return W


# ---- learned-closure layers -------------------------------------------------------------------
def conv3d_forward(x, w, b, act):
    """x [n3][n2][n1][C], w [O][27][C], b [O] -> y [n3][n2][n1][O] (FP64)."""
    x, w, b = _c(x), _c(w), _c(b)
    n3, n2, n1, Cc = x.shape
    O = w.shape[0]
    y = np.empty((n3, n2, n1, O))
    lib().orc_conv3d_forward(_ptr(x), _ptr(w), _ptr(b), _ptr(y), n1, n2, n3, Cc, O, int(act))
    return y


def conv3d_backward(x, w, y, g, act):
    """Gradients (dx, dw, db) of L with dL/dy = g, y the forward output."""
    x, w, y, g = _c(x), _c(w), _c(y), _c(g)
    n3, n2, n1, Cc = x.shape
    O = w.shape[0]
    dx, dw, db = np.empty_like(x), np.empty_like(w), np.empty(O)
    lib().orc_conv3d_backward(_ptr(x), _ptr(w), _ptr(y), _ptr(g), _ptr(dx), _ptr(dw), _ptr(db), n1, n2, n3, Cc, O, int(act))
    return dx, dw, db


def restrict(Uf, vol_f):
    """Volume-weighted 2x2x2 restriction of a fine state [8][2n3][2n2][2n1]."""
    Uf, vol_f = _c(Uf), _c(vol_f)
    _, f3, f2, f1 = Uf.shape
    Uc = np.empty((8, f3 // 2, f2 // 2, f1 // 2))
    lib().orc_restrict(_ptr(Uf), _ptr(vol_f), _ptr(Uc), f1 // 2, f2 // 2, f3 // 2)
    return Uc


def set_threads(n: int) -> int:
    """Number of host threads the oracle's OpenMP loops use (for timing only); returns the new
    maximum."""
    lib().orc_set_threads(int(n))
    return int(lib().orc_max_threads())
