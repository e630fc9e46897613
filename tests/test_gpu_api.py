"""Behaviour of the C ABI on the GPU beyond single-step parity: a multi-step call (replayed from
the CUDA graph, the launch configuration the bench times) equals the same number of single steps
bit for bit; calls out of order are rejected with ESTATE; the single-precision forms match the
FP64 oracle on the full production-size grid within single-precision error (the tolerance of
test_gpu_fused: <= 2e-5 of each field's scale for one step)."""
import numpy as np
import pytest

from oracle.oracle import from_workload as oracle_workload
from paper_2501_15923_gb300 import inputs as I

from .test_gpu_parity import field_errors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ic():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_15923_gb300 import build
    build.build()
    from paper_2501_15923_gb300 import icarus
    return icarus


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_graph_steps_equal_single_steps(ic, prec):
    """step(7) (graph replay, dt kept on the device) against seven step(1) calls, through a CME
    window, with probes registered: identical state, time and probe records."""
    w = I.dynamic_cme(grid=I.Grid(64, 16, 32))
    a, b = ic.from_workload(w, precision=prec), ic.from_workload(w, precision=prec)
    U, _ = a.get_state()
    t = (w.cmes[0, 0] - 120.0) / a.scales()["t0"]
    for s in (a, b):
        s.set_state(U, t)
        s.sample(w.traj, cap=1)
    a.step(7)
    for _ in range(7):
        b.step(1)
    Ua, ta = a.get_state()
    Ub, tb = b.get_state()
    assert ta == tb and np.array_equal(Ua, Ub)
    ra, na = a.sample(None, cap=64)
    rb, nb = b.sample(None, cap=64)
    assert na == nb and na >= 7 and np.array_equal(ra[:na], rb[:nb])
    a.close(); b.close()


def test_calls_out_of_order_rejected(ic):
    w = I.static_sheet()
    s = ic.Solver(w.grid, w.gamma, w.omega, w.opts)
    with pytest.raises(ic.IcarusError) as e:
        s.step(1)
    assert "ESTATE" in str(e.value)
    with pytest.raises(ic.IcarusError) as e:
        s.sample(w.traj, cap=4)
    assert "ESTATE" in str(e.value)
    s.close()


@pytest.mark.parametrize("prec", [1, 2])
def test_full_size_single_precision_forms(ic, prec):
    """512 x 64 x 128, one step from the initial state at a time in the CME window."""
    w = I.dynamic_cme()
    gpu, orc = ic.from_workload(w, precision=prec), oracle_workload(w)
    U, _ = gpu.get_state()
    t = (w.cmes[0, 0] + 1800.0) / orc.scales()["t0"]
    gpu.set_state(U, t)
    orc.set_state(U, t)
    gpu.step(1)
    orc.step()
    Ug, tg = gpu.get_state()
    Uo, to = orc.get_state()
    err = field_errors(Ug, Uo)
    assert err.max() <= 2e-5, err
    assert abs(tg - to) <= 1e-5 * abs(to - t)
    gpu.close()


def test_new_maps_of_the_same_shape_reach_the_captured_step(ic):
    """icarus_set_boundary with tables of unchanged shape keeps the captured step (the device
    tables are rewritten in place): the next step must see the new values, bit for bit as a
    context that was given them from the start."""
    w = I.dynamic_cme(grid=I.Grid(48, 12, 24))
    maps2 = w.maps * np.array([1.1, 0.9, 1.05, 1.0, 0.95])[None, :, None, None]
    a = ic.from_workload(w)
    U, _ = a.get_state()
    t = 1.5 * I.DAY / a.scales()["t0"]
    a.set_state(U, t)
    a.step(1)                                   # the step is captured with the first tables
    a.set_boundary(w.t_maps, maps2, w.cmes)
    a.set_state(U, t)
    a.step(1)
    w2 = I.dynamic_cme(grid=I.Grid(48, 12, 24))
    w2.maps = maps2
    b = ic.from_workload(w2)
    b.set_state(U, t)
    b.step(1)
    Ua, ta = a.get_state()
    Ub, tb = b.get_state()
    assert ta == tb and np.array_equal(Ua, Ub)
    a.close(); b.close()
