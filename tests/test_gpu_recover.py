"""Recovery from a failed attempt (icarus_step_recover): the snapshot taken before the steps is
restored, the CFL number halved and the steps run again.

The failure comes from the flow, not from the device: two cold streams (rho 1, v = +-20, p 1e-4,
gamma 1.5: Mach 1600) collide at the middle of a 128-cell line. At CFL 0.8 the scheme overshoots
at the collision and the recovered pressure turns negative within the first steps (the oracle
counts the floor activations); at CFL 0.4 the 40 steps keep every pressure at its initial 1e-4, far
above the floor. With options.strict_floors the floor activation is the step's EFLOOR status, so
the recovering call must end with exactly the state of a plain run at CFL 0.4 (bit for bit: the
same kernels from the restored snapshot), the oracle's state at CFL 0.4 (to 1e-12), and the
configured CFL back in force for the next dt.
"""
import ctypes as C

import numpy as np
import pytest

from oracle import oracle as O
from paper_2501_15923_gb300 import inputs as I

from .helpers import cart_grid, opts

EFLOOR = -7
N_STEPS = 40


@pytest.fixture(scope="module")
def ic():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_15923_gb300 import build
    build.build()
    from paper_2501_15923_gb300 import icarus
    return icarus


def collision(cfl, strict=1):
    n1 = 128
    g = cart_grid(n1, bc=(I.BC_CONT,) * 2 + (I.BC_PERIODIC,) * 4)
    o = opts(cfl=cfl, gravity=0, divb=0, p_floor=1e-10, rho_floor=1e-10, strict_floors=strict)
    x = (np.arange(n1) + 0.5) / n1
    W = np.zeros((8, 1, 1, n1))
    W[0] = 1.0
    W[1] = np.where(x < 0.5, 20.0, -20.0)
    W[4] = 1e-4
    return g, o, O.cons_from_prim(W, 1.5)


def oracle_run(cfl, n):
    g, o, U0 = collision(cfl)
    orc = O.Oracle(g, 1.5, 0.0, o)
    orc.set_state(U0, 0.0)
    for _ in range(n):
        orc.step()
    return orc


def solver(ic, cfl, precision=0, strict=1):
    g, o, U0 = collision(cfl, strict)
    s = ic.Solver(g, 1.5, 0.0, o, precision)
    s.set_state(U0, 0.0)
    return s, U0


def test_the_flow_fails_at_the_configured_cfl_only():
    """The premise, on the oracle (CPU): floor activations at CFL 0.8, none at 0.4."""
    assert oracle_run(0.8, N_STEPS).floor_hits > 0
    orc = oracle_run(0.4, N_STEPS)
    assert orc.floor_hits == 0
    U, _ = orc.get_state()
    assert O.prim_from_cons(U, 1.5)[4].min() > 0.5e-4


@pytest.mark.gpu
def test_recovery_halves_the_cfl_and_equals_the_half_cfl_run(ic):
    rec, U0 = solver(ic, 0.8)
    assert rec.step_recover(N_STEPS, max_retries=3) == 1
    Ur, tr = rec.get_state()                                   # status clear: no exception
    plain, _ = solver(ic, 0.4)
    plain.step(N_STEPS)
    Up, tp = plain.get_state()
    assert tr == tp and np.array_equal(Ur, Up)
    orc = oracle_run(0.4, N_STEPS)
    Uo, to = orc.get_state()
    scale = np.abs(Uo).reshape(8, -1).max(axis=1)[:, None, None, None] + 1e-300
    assert (np.abs(Ur - Uo) / scale).max() <= 1e-12
    assert abs(tr - to) <= 1e-12 * to
    # the configured CFL is back: the next dt is exactly twice the CFL 0.4 run's (the same speed)
    assert rec.time()[1] == 2.0 * plain.time()[1]
    assert rec.status() == (0, 0)                              # the failed attempt's floors dropped
    rec.step(1)
    assert rec.status()[0] == 0
    rec.close()
    plain.close()


@pytest.mark.gpu
def test_spent_retries_restore_the_snapshot_and_keep_the_status(ic):
    s, U0 = solver(ic, 0.8)
    lib = ic.load()
    h = C.c_int(-1)
    assert lib.icarus_step_recover(s.ctx, N_STEPS, 0, C.byref(h)) == EFLOOR and h.value == 0
    assert "strict_floors" in lib.icarus_last_error().decode()
    U = np.empty(s.shape)
    t = C.c_double(-1.0)
    assert lib.icarus_get_state(s.ctx, U.ctypes.data_as(C.c_void_p), C.byref(t)) == EFLOOR
    assert t.value == 0.0 and np.array_equal(U, U0)             # the snapshot, bit for bit
    assert lib.icarus_step(s.ctx, 1) == EFLOOR                  # sticky, as after icarus_step
    assert lib.icarus_step_recover(s.ctx, 1, 3, None) == EFLOOR # returned at once, no stepping
    s.set_state(U0, 0.0)                                        # clears it
    assert s.step_recover(N_STEPS, max_retries=1) == 1
    s.close()


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [0, 2])
def test_without_failure_it_is_a_plain_step(ic, precision):
    """No failure: the same state, time, tracer and probe records as icarus_step (production
    drivers on a small spherical grid, CME tracer on)."""
    w = I.dynamic_cme(grid=I.Grid(48, 12, 24))
    w.opts = I.Options(tracer=1)
    runs = []
    for recover in (False, True):
        s = ic.from_workload(w, precision=precision)
        s.sample(w.traj, cap=1)
        s.sample(None, cap=16)
        if recover:
            assert s.step_recover(6, max_retries=2) == 0
        else:
            s.step(6)
        U, t = s.get_state()
        rec, n = s.sample(None, cap=16)
        runs.append((U, t, s.get_tracer(), rec[:n], s.time()[1]))
        s.close()
    (Ua, ta, ca, ra, da), (Ub, tb, cb, rb, db) = runs
    assert ta == tb and da == db and np.array_equal(Ua, Ub) and np.array_equal(ca, cb)
    assert len(ra) == 6 and np.array_equal(ra, rb)
