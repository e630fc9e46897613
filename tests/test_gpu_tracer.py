"""CME tracer on the GPU (options.tracer = 1) against the FP64 oracle's tracer, one step at a
time from the same state and tracer field: before the CME, inside the insertion window (driven
ghosts at c = 1 in the footprint), across the end of the window (stage 1 inside, stage 2
outside), for both CME models. FP64: the MHD fields to <= 1e-12 of their scale (as in
test_gpu_parity) and c to <= 1e-12 absolute (c lies in [0, 1]); the single-precision forms to
2e-5 of the field scales and 2e-5 in c."""
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


def tracer_workload(cme_model):
    w = I.dynamic_cme(grid=I.Grid(48, 12, 24))
    w.opts.tracer = 1
    w.opts.cme_model = cme_model
    return w


def step_pair(gpu, orc, U, c, t):
    for s in (gpu, orc):
        s.set_state(U, t)
        s.set_tracer(c)
    gpu.step(1)
    orc.step()
    Ug, _ = gpu.get_state()
    Uo, _ = orc.get_state()
    return Ug, Uo, gpu.get_tracer(), orc.get_tracer()


@pytest.mark.parametrize("cme_model", [I.CME_WINDOW, I.CME_SPHERE])
@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 2e-5), (2, 2e-5)])
def test_tracer_steps_match_oracle(ic, cme_model, prec, tol):
    w = tracer_workload(cme_model)
    gpu, orc = ic.from_workload(w, precision=prec), oracle_workload(w)
    sc = orc.scales()
    U, _ = gpu.get_state()
    rng = np.random.default_rng(11)
    c = rng.uniform(0.0, 1.0, U.shape[1:])
    c[:, :, :4] = 0.0                      # unmarked plasma next to the driven face
    c[:, :3, 10:20] = 1.0                  # a marked patch at the theta edge
    t_on = w.cmes[0, 0] / sc["t0"]
    dur = (w.cmes[0, 1] if cme_model == I.CME_WINDOW
           else 2.0 * w.grid.x1min * np.sin(w.cmes[0, 4]) / (w.cmes[0, 5] / 1e5) * sc["t0"])
    t_end = t_on + dur / sc["t0"]
    gpu.set_state(U, t_end - 1e-9)
    _, dt = gpu.time()
    times = (t_on - 3600.0 / sc["t0"], t_on + 0.3 * dur / sc["t0"], t_end - 0.5 * dt)
    marked = 0
    for t in times:
        Ug, Uo, cg, co = step_pair(gpu, orc, U, c, t)
        err = field_errors(Ug, Uo)
        assert err.max() <= tol, (t, err)
        assert np.abs(cg - co).max() <= tol, (t, np.abs(cg - co).max())
        assert co.min() >= 0.0 and co.max() <= 1.0
        marked = max(marked, int((co[:, :, 0] > c[:, :, 0] + 1e-3).sum()))
    assert marked > 0                      # the insertion raised c in the first radial cells
    gpu.close()


def test_tracer_round_trip_launches_and_errors(ic):
    w = tracer_workload(I.CME_WINDOW)
    gpu = ic.from_workload(w)
    U, t = gpu.get_state()
    c = np.random.default_rng(3).uniform(0.0, 1.0, U.shape[1:])
    gpu.set_tracer(c)
    assert np.abs(gpu.get_tracer() - c).max() <= 1e-15
    w0 = I.dynamic_cme(grid=I.Grid(48, 12, 24))
    plain = ic.from_workload(w0)
    assert gpu.launches_per_step == plain.launches_per_step + 4   # ghost + update per stage
    with pytest.raises(ic.IcarusError) as e:
        plain.set_tracer(c)
    assert "EINVAL" in str(e.value)
    # set_state keeps rho c: doubling rho halves c
    U2 = U.copy()
    U2[0] *= 2.0
    gpu.set_state(U2, t)
    assert np.allclose(gpu.get_tracer(), 0.5 * c, rtol=1e-15, atol=0)
    gpu.close(); plain.close()
