"""GPU (libicarus, through the C ABI) against the FP64 CPU oracle, step by step.

Tolerance: one FP64 step from the same state agrees to <= 1e-12 relative per field, where a
field's error is max|GPU - oracle| over the grid divided by the largest magnitude of that field
(vector components share the scale of their vector). dt agrees to <= 1e-13. Probe stencil
indices are compared exactly; probe values to <= 1e-12 of each quantity's scale.
"""
import math

import numpy as np
import pytest

from oracle.oracle import Oracle, cons_from_prim, prim_from_cons
from oracle.oracle import from_workload as oracle_workload
from paper_2501_15923_gb300 import inputs as I

from .helpers import cart_grid, sph_grid

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module")
def ic():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_15923_gb300 import build
    build.build()
    from paper_2501_15923_gb300 import icarus
    return icarus


def field_errors(Ug, Uo):
    sc = np.empty(8)
    sc[0] = np.abs(Uo[0]).max()
    sc[1:4] = np.sqrt((Uo[1:4] ** 2).sum(0)).max()
    sc[4] = np.abs(Uo[4]).max()
    sc[5:8] = np.sqrt((Uo[5:8] ** 2).sum(0)).max()
    sc[sc == 0] = 1.0
    return np.abs(Ug - Uo).reshape(8, -1).max(1) / sc


def step_both(gpu, orc, U, t, dt_cap=0.0):
    gpu.set_state(U, t)
    orc.set_state(U, t)
    if dt_cap:
        gpu.set_stop_time(t + dt_cap)
    gpu.step(1)
    dto = orc.step(dt_cap)
    Ug, tg = gpu.get_state()
    Uo, to = orc.get_state()
    return Ug, Uo, tg, to, dto


def assert_step(gpu, orc, U, t, tol=TOL, dt_cap=0.0):
    Ug, Uo, tg, to, dto = step_both(gpu, orc, U, t, dt_cap)
    err = field_errors(Ug, Uo)
    assert err.max() <= tol, err
    assert abs(tg - to) <= 1e-13 * max(abs(to), 1e-300) + 1e-300, (tg, to)
    return Ug, tg


# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("init_vphi", [I.IC_COROTATING, I.IC_INERTIAL_RADIAL])
def test_initial_state_matches(ic, init_vphi):
    w = I.static_sheet()
    w.opts.init_vphi = init_vphi
    gpu, orc = ic.from_workload(w), oracle_workload(w)
    Ug, _ = gpu.get_state()
    Uo, _ = orc.get_state()
    assert field_errors(Ug, Uo).max() <= 1e-14
    gpu.close()


def test_static_sheet_per_step_parity_20_steps(ic):
    """Twenty consecutive steps of the static-sheet workload (60 x 16 x 32); at every step the oracle restarts from
    the GPU state, so each comparison is one step from an identical state."""
    w = I.static_sheet()
    gpu, orc = ic.from_workload(w), oracle_workload(w)
    U, t = gpu.get_state()
    for _ in range(20):
        U, t = assert_step(gpu, orc, U, t)
    gpu.close()


@pytest.mark.parametrize("lim,flux,divb,grav", [
    (I.LIM_MINMOD, I.FLUX_TVDLF, I.DIVB_LINDE, 1),
    (I.LIM_MC, I.FLUX_HLL, I.DIVB_LINDE, 1),
    (I.LIM_VANLEER, I.FLUX_HLL, I.DIVB_NONE, 0),
    (I.LIM_VANLEER, I.FLUX_TVDLF, I.DIVB_POWELL, 1),
])
def test_options_perturbed_state(ic, lim, flux, divb, grav):
    """Randomly perturbed static-sheet state (every component nonzero, limiter branches mixed)."""
    w = I.static_sheet()
    w.opts = I.Options(limiter=lim, flux=flux, divb=divb, gravity=grav)
    gpu, orc = ic.from_workload(w), oracle_workload(w)
    U, t = gpu.get_state()
    Up = I.perturbed_state(U.shape, 11, U, 2e-2)
    Up[2] += 0.05 * np.abs(U[1]).max() * I.perturbed_state(U.shape[1:], 12, np.ones(U.shape[1:]), 1.0)
    Up[6] += 0.05 * np.abs(U[5]).max() * I.perturbed_state(U.shape[1:], 13, np.ones(U.shape[1:]), 1.0)
    f0 = gpu.status()[1]
    assert_step(gpu, orc, Up, 0.01)
    # this state has cells with negative pressure: the floors fire, and the counts (density and
    # pressure resets over both stages, decided in FP64 on both sides) agree exactly
    assert orc.floor_hits > 0
    assert gpu.status()[1] - f0 == orc.floor_hits
    gpu.close()


@pytest.mark.parametrize("lim,divb,grav", [(I.LIM_VANLEER, I.DIVB_LINDE, 1), (I.LIM_MC, I.DIVB_NONE, 0)])
def test_hlld_perturbed_state(ic, lim, divb, grav):
    """HLLD flux (its own kernel instantiation) on a perturbed static-sheet state. The perturbation is
    made in primitive variables so that the pressure stays positive: HLLD's intermediate states
    have no meaning for negative pressures (the oracle's step turns non-finite there too)."""
    w = I.static_sheet()
    w.opts = I.Options(limiter=lim, flux=I.FLUX_HLLD, divb=divb, gravity=grav)
    gpu, orc = ic.from_workload(w), oracle_workload(w)
    U, _ = gpu.get_state()
    W = prim_from_cons(U, w.gamma)
    Wp = I.perturbed_state(W.shape, 11, W, 2e-2)
    noise = lambda seed: I.perturbed_state(W.shape[1:], seed, np.ones(W.shape[1:]), 1.0) - 1.0
    Wp[2] += 0.1 * np.abs(W[1]) * noise(12)
    Wp[6] += 0.1 * np.sqrt((W[5:8] ** 2).sum(0)) * noise(13)
    U1, t1 = assert_step(gpu, orc, cons_from_prim(Wp, w.gamma), 0.01)
    for _ in range(4):
        U1, t1 = assert_step(gpu, orc, U1, t1)
    gpu.close()


def test_dynamic_maps_and_cme_window(ic):
    """Production drivers (10 daily maps, one cone CME) on a reduced grid: time between two maps and inside the CME window,
    then a step that crosses the end of the window (boundary values change between stages)."""
    g = I.Grid(48, 12, 24)
    w = I.dynamic_cme(grid=g)
    gpu, orc = ic.from_workload(w), oracle_workload(w)
    sc = orc.scales()
    U, _ = gpu.get_state()
    t_on = w.cmes[0, 0] / sc["t0"]
    for t in (t_on + 0.3 * 3600 / sc["t0"], 1.37 * I.DAY / sc["t0"]):
        assert_step(gpu, orc, U, t)
    # straddle the end of the insertion window: stage 1 inside, stage 2 outside
    t_end = (w.cmes[0, 0] + w.cmes[0, 1]) / sc["t0"]
    gpu.set_state(U, t_end - 1e-9)
    _, dt = gpu.time()
    assert dt > 1e-9
    assert_step(gpu, orc, U, t_end - 0.5 * dt)
    _, hit = orc.boundary_values(t_on + 1e-6)
    assert hit.sum() > 0
    gpu.close()


def test_sphere_cme_crossing(ic):
    """Spherical-cloud CME option: steps while the cloud crosses the inner boundary (footprint
    growing, full, shrinking) and one after it has passed; the footprint is decided by the same
    FP64 operations on both sides, so the boundary ghosts agree exactly."""
    g = I.Grid(48, 12, 24)
    w = I.dynamic_cme(grid=g)
    w.opts.cme_model = I.CME_SPHERE
    gpu, orc = ic.from_workload(w), oracle_workload(w)
    sc = orc.scales()
    U, _ = gpu.get_state()
    t_on = w.cmes[0, 0] / sc["t0"]
    cross = 2.0 * g.x1min * math.sin(w.cmes[0, 4]) / (w.cmes[0, 5] / 1e5)
    for f in (0.2, 0.37, 0.8, 1.3):
        assert_step(gpu, orc, U, t_on + f * cross)
    _, hit = orc.boundary_values(t_on + 0.37 * cross)
    assert hit.sum() > 0
    _, hit = orc.boundary_values(t_on + 1.01 * cross)
    assert hit.sum() == 0
    gpu.close()


def test_uniform_radial_grid_two_hour_maps(ic):
    """The paper-shaped 2019 drivers (uniform radial spacing, maps every 2 h) on a reduced grid:
    steps between maps and across a map time."""
    w = I.paper2019(grid=I.Grid(60, 16, 48, stretch=0))
    gpu, orc = ic.from_workload(w), oracle_workload(w)
    sc = orc.scales()
    U, _ = gpu.get_state()
    for t in (3.3 * 3600.0 / sc["t0"], (2 * 7200.0 - 1.0) / sc["t0"]):
        assert_step(gpu, orc, U, t)
    gpu.close()


def test_ragged_grid_sizes(ic):
    """Sizes that are not multiples of any block edge (ragged tails in every kernel)."""
    for n in ((37, 9, 7), (129, 17, 33), (2, 10, 3)):
        g = I.Grid(*n)
        w = I.dynamic_cme(grid=g)
        gpu, orc = ic.from_workload(w), oracle_workload(w)
        U, t = gpu.get_state()
        for _ in range(2):
            U, t = assert_step(gpu, orc, U, t)
        gpu.close()


def test_cartesian_shock_tube_and_periodic_box(ic):
    """Verification geometry: a Brio-Wu tube along y and a fully periodic 3-D box."""
    g = cart_grid(1, 200, 1, L=(1e3, 1.0, 1e3), bc=(I.BC_PERIODIC,) * 2 + (I.BC_CONT,) * 2 + (I.BC_PERIODIC,) * 2)
    o = I.Options(divb=I.DIVB_NONE)
    gpu = ic.Solver(g, 2.0, 0.0, o)
    orc = Oracle(g, 2.0, 0.0, o)
    y = (np.arange(200) + 0.5) / 200
    W = np.zeros((8, 1, 200, 1))
    W[0, 0, :, 0] = np.where(y < 0.5, 1.0, 0.125)
    W[4, 0, :, 0] = np.where(y < 0.5, 1.0, 0.1)
    W[6] = 0.75
    W[5, 0, :, 0] = np.where(y < 0.5, 1.0, -1.0)
    U = cons_from_prim(W, 2.0)
    t = 0.0
    for _ in range(10):
        U, t = assert_step(gpu, orc, U, t)
    gpu.close()
    g = cart_grid(24, 20, 16)
    o = I.Options(divb=I.DIVB_LINDE)
    gpu, orc = ic.Solver(g, 5 / 3, 0.0, o), Oracle(g, 5 / 3, 0.0, o)
    rng = np.random.default_rng(5)
    W = np.zeros((8, 16, 20, 24))
    W[0] = 1.0 + 0.2 * rng.random(W.shape[1:])
    W[1:4] = 0.3 * rng.standard_normal((3,) + W.shape[1:])
    W[4] = 1.0 + 0.2 * rng.random(W.shape[1:])
    W[5:8] = 0.5 * rng.standard_normal((3,) + W.shape[1:])
    assert_step(gpu, orc, cons_from_prim(W, 5 / 3), 0.0)
    gpu.close()


def test_reflecting_shell(ic):
    g = sph_grid(20, 10, 16, bc=(I.BC_REFLECT,) * 4 + (I.BC_PERIODIC,) * 2, r=(0.3, 1.0))
    o = I.Options(gravity=0)
    gpu, orc = ic.Solver(g, 1.5, I.OMEGA_SUN, o), Oracle(g, 1.5, I.OMEGA_SUN, o)
    rng = np.random.default_rng(9)
    W = np.zeros((8, 16, 10, 20))
    W[0] = 1.0 + 0.3 * rng.random(W.shape[1:])
    W[1:4] = 0.2 * rng.standard_normal((3,) + W.shape[1:])
    W[4] = 2.0 + rng.random(W.shape[1:])
    W[5:8] = 0.4 * rng.standard_normal((3,) + W.shape[1:])
    assert_step(gpu, orc, cons_from_prim(W, 1.5), 0.0)
    gpu.close()


def test_stop_time_caps_dt(ic):
    w = I.static_sheet()
    gpu, orc = ic.from_workload(w), oracle_workload(w)
    U, t = gpu.get_state()
    _, dt = gpu.time()
    Ug, tg = assert_step(gpu, orc, U, t, dt_cap=0.3 * dt)
    assert abs(tg - (t + 0.3 * dt)) <= 1e-15 * tg
    gpu.set_state(Ug, tg)
    gpu.set_stop_time(tg)
    gpu.step(3)                    # at the stop time the steps are no-ops
    U2, t2 = gpu.get_state()
    assert t2 == tg and np.array_equal(U2, Ug)
    gpu.close()


# ---------------------------------------------------------------------------------------------
def test_probe_parity_indices_exact(ic):
    w = I.dynamic_cme(grid=I.Grid(96, 24, 48))
    gpu, orc = ic.from_workload(w), oracle_workload(w)
    U, _ = gpu.get_state()
    sc = orc.scales()
    for t_si in (0.0, 3.3 * 3600, 2.71 * I.DAY, 9.99 * I.DAY, 12 * I.DAY):
        t = t_si / sc["t0"]
        gpu.set_state(U, t)
        orc.set_state(U, t)
        rec, n = gpu.sample(w.traj, cap=1)
        ref = orc.sample(w.traj)
        assert n == 1
        g = rec[0]
        assert np.array_equal(g[:, 10:13], ref[:, 10:13]), (g[:, 10:13], ref[:, 10:13])
        scale = np.abs(ref).max(0)
        scale[scale == 0] = 1
        assert np.all(np.abs(g[:, :10] - ref[:, :10]) <= TOL * scale[:10])
    gpu.close()


def test_probe_ring_records_every_step(ic):
    w = I.static_sheet()
    gpu = ic.from_workload(w)
    gpu.sample(w.traj, cap=1)
    gpu.step(7)
    rec, n = gpu.sample(None, cap=16)
    assert n == 7
    t = rec[:, 0, 0]
    assert np.all(np.diff(t) > 0)
    assert np.all(rec[:, :, 1] > 0)
    gpu.close()


def test_full_size_one_step_parity(ic):
    """512 x 64 x 128 (the production-size grid) from the production initial state at a time in the
    CME window: one step compared on the whole grid."""
    w = I.dynamic_cme()
    gpu, orc = ic.from_workload(w), oracle_workload(w)
    U, _ = gpu.get_state()
    t = (w.cmes[0, 0] + 1800.0) / orc.scales()["t0"]
    assert_step(gpu, orc, U, t)
    gpu.close()


# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("prec,tol", [(1, 2e-5), (2, 2e-5)])
def test_reduced_precision_step(ic, prec, tol):
    """FP32 state and MIXED: one step from the same state within single-precision error."""
    w = I.static_sheet()
    gpu, orc = ic.from_workload(w, precision=prec), oracle_workload(w)
    U, t = gpu.get_state()
    gpu.set_state(U, t)
    orc.set_state(U, t)
    gpu.step(1)
    orc.step()
    Ug, _ = gpu.get_state()
    Uo, _ = orc.get_state()
    err = field_errors(Ug, Uo)
    assert err.max() <= tol, err
    gpu.close()


@pytest.mark.parametrize("prec", [1, 2])
def test_hlld_single_precision_forms(ic, prec):
    """HLLD in the FP32-state and MIXED forms: one step on the perturbed static-sheet state of
    test_hlld_perturbed_state, within the single-precision bar (2e-5 of each field's scale)."""
    w = I.static_sheet()
    w.opts = I.Options(flux=I.FLUX_HLLD)
    gpu, orc = ic.from_workload(w, precision=prec), oracle_workload(w)
    U, _ = gpu.get_state()
    W = prim_from_cons(U, w.gamma)
    Wp = I.perturbed_state(W.shape, 11, W, 2e-2)
    Ug, Uo, tg, to, _ = step_both(gpu, orc, cons_from_prim(Wp, w.gamma), 0.01)
    err = field_errors(Ug, Uo)
    assert err.max() <= 2e-5, err
    assert abs(tg - to) <= 1e-5 * abs(to - 0.01)
    gpu.close()
