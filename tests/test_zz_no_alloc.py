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


@pytest.mark.parametrize("shape", [(64, 16, 32), (512, 64, 128)])
def test_noalloc_dt_matches_allocating_path_twice(env, shape):
    ic, torch = env
    w = I.dynamic_cme(grid=I.Grid(*shape))
    s = ic.from_workload(w)
    grid_c = ic.make_grid(w.grid)
    U_a, t = s.get_state()
    U_b = I.perturbed_state(U_a.shape, 21, U_a, 5e-2)          # a second, different state
    for U in (U_a, U_b):                                        # two calls in a row
        ref = reference_dt(s, U, t)
        got = noalloc_dt(ic, torch, grid_c, w.gamma, w.opts.cfl, U)
        assert ref > 0 and abs(got - ref) <= TOL * ref, (got, ref)
    s.close()


def test_noalloc_rejects_grids_beyond_its_scratch(env):
    ic, torch = env
    g = ic.make_grid(I.Grid(512, 64, 129))                      # one phi column more than the limit
    dt_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    U_dev = torch.zeros(8, dtype=torch.float64, device="cuda")  # never read: rejected before launch
    with pytest.raises(ic.IcarusError) as e:
        ic.icarus_cfl_dt_noalloc(g, 1.5, 0.8, U_dev.data_ptr(), dt_dev.data_ptr(), None)
    assert e.value.code == -1 and "ICARUS_NOALLOC_MAX_CELLS" in str(e.value)
