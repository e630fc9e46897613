"""Allocation-free CFL time step (icarus_cfl_dt_noalloc) against the allocating path.

icarus_cfl_dt_noalloc is for callers that cannot allocate device memory where they need a time
step; its reduction scratch is a fixed device array inside the library. Here it is called through
the C ABI on device buffers the test owns, twice in a row on different states, and each result is
compared with the dt the context-based path reports (icarus_set_state + icarus_time) for the same
state, to the 1e-12 relative tolerance of the parity tests. This file is collected last so that a
run stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_2501_15923_gb300 import inputs as I

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_15923_gb300 import build
    build.build()
    from paper_2501_15923_gb300 import icarus as ic
    return ic, torch


def reference_dt(solver, U, t):
    solver.set_state(U, t)
    _, dt = solver.time()
    return dt


def noalloc_dt(ic, torch, grid_c, gamma, cfl, U):
    U_dev = torch.from_numpy(np.ascontiguousarray(U)).cuda()
    dt_dev = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    ic.icarus_cfl_dt_noalloc(grid_c, gamma, cfl, U_dev.data_ptr(), dt_dev.data_ptr(), None)
    torch.cuda.synchronize()
    return float(dt_dev.item())


GRIDS = {
    "stretched sphere 64x16x32": I.Grid(64, 16, 32),
    "stretched sphere 512x64x128": I.Grid(512, 64, 128),
    "uniform-radius sphere": I.Grid(48, 12, 20, stretch=0),
    "stretched sphere with a refined band": I.Grid(72, 12, 24, band_refine=4, band_lo=0.8, band_hi=1.2),
    "uniform sphere with a refined band": I.Grid(60, 10, 16, stretch=0, band_refine=3, band_lo=0.5, band_hi=1.1),
}


@pytest.mark.parametrize("name", list(GRIDS))
def test_noalloc_dt_matches_allocating_path_twice(env, name):
    ic, torch = env
    w = I.dynamic_cme(grid=GRIDS[name])
    s = ic.from_workload(w)
    grid_c = ic.make_grid(w.grid)
    U_a, t = s.get_state()
    U_b = I.perturbed_state(U_a.shape, 21, U_a, 5e-2)          # a second, different state
    for U in (U_a, U_b):                                        # two calls in a row
        ref = reference_dt(s, U, t)
        got = noalloc_dt(ic, torch, grid_c, w.gamma, w.opts.cfl, U)
        assert ref > 0 and abs(got - ref) <= TOL * ref, (got, ref)
    s.close()


def test_noalloc_dt_cartesian_grid(env):
    """The Cartesian branch (widths dx, dy, dz) on a box with three different widths."""
    ic, torch = env
    g = I.Grid(40, 12, 9, geometry=I.GEOM_CARTESIAN, stretch=0, x1min=0.0, x1max=2.0, x2min=0.0,
               x2max=0.3, x3min=-1.0, x3max=1.0, bc=(I.BC_PERIODIC,) * 6)
    s = ic.Solver(g, 1.5, 0.0, I.Options(gravity=0))
    rng = np.random.default_rng(5)
    W = np.empty((8, g.n3, g.n2, g.n1))
    W[0] = rng.uniform(0.5, 2.0, W.shape[1:])
    W[1:4] = rng.uniform(-1.0, 1.0, (3,) + W.shape[1:])
    W[4] = rng.uniform(0.2, 1.0, W.shape[1:])
    W[5:8] = rng.uniform(-1.0, 1.0, (3,) + W.shape[1:])
    U = np.empty_like(W)
    U[0], U[1:4], U[5:8] = W[0], W[0] * W[1:4], W[5:8]
    U[4] = W[4] / 0.5 + 0.5 * W[0] * (W[1:4] ** 2).sum(0) + 0.5 * (W[5:8] ** 2).sum(0)
    for Uc in (U, U[:, :, :, ::-1].copy()):
        ref = reference_dt(s, Uc, 0.0)
        got = noalloc_dt(ic, torch, ic.make_grid(g), 1.5, 0.8, Uc)
        assert ref > 0 and abs(got - ref) <= TOL * ref, (got, ref)
    s.close()


def test_noalloc_dt_flags_a_non_finite_state(env):
    """A NaN in one cell gives the documented dt = -1 (fmax alone would drop it); the next call on
    a finite state gives the right dt again (the flag does not stick between calls)."""
    ic, torch = env
    w = I.dynamic_cme(grid=I.Grid(64, 16, 32))
    s = ic.from_workload(w)
    U, t = s.get_state()
    bad = U.copy()
    bad[4, 7, 3, 11] = np.nan
    assert noalloc_dt(ic, torch, ic.make_grid(w.grid), w.gamma, w.opts.cfl, bad) == -1.0
    ref = reference_dt(s, U, t)
    got = noalloc_dt(ic, torch, ic.make_grid(w.grid), w.gamma, w.opts.cfl, U)
    assert abs(got - ref) <= TOL * ref
    s.close()


@pytest.mark.parametrize("change,msg", [(dict(x1min=0.0), "r_in"), (dict(x2min=0.02), "colatitude"),
                                        (dict(band_refine=4, band_lo=0.05, band_hi=1.0), "band"),
                                        (dict(x1max=0.05), "empty")])
def test_noalloc_rejects_grids_icarus_init_rejects(env, change, msg):
    ic, torch = env
    kw = dict(n1=32, n2=8, n3=16)
    kw.update(change)
    g = ic.make_grid(I.Grid(**kw))
    dt_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    U_dev = torch.zeros(8, dtype=torch.float64, device="cuda")  # never read: rejected before launch
    with pytest.raises(ic.IcarusError) as e:
        ic.icarus_cfl_dt_noalloc(g, 1.5, 0.8, U_dev.data_ptr(), dt_dev.data_ptr(), None)
    assert e.value.code == -1 and msg in str(e.value)


def test_noalloc_rejects_grids_beyond_its_scratch(env):
    ic, torch = env
    g = ic.make_grid(I.Grid(512, 64, 129))                      # one phi column more than the limit
    dt_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    U_dev = torch.zeros(8, dtype=torch.float64, device="cuda")  # never read: rejected before launch
    with pytest.raises(ic.IcarusError) as e:
        ic.icarus_cfl_dt_noalloc(g, 1.5, 0.8, U_dev.data_ptr(), dt_dev.data_ptr(), None)
    assert e.value.code == -1 and "ICARUS_NOALLOC_MAX_CELLS" in str(e.value)
