"""Checkpoint and resume through the C ABI: the state and time read with icarus_get_state after
some steps, written into a fresh context with icarus_set_state (same drivers), continue exactly as
the run that was never interrupted. The next time step after the resume is computed from the same
state by the time-step kernel and, in the uninterrupted run, by the second-stage update's fused
reduction; both give the exact maximum over the cells, so the runs agree bit for bit: state, time
and the probe records of the later steps. FP64 and the mixed form (whose single-precision
primitive mirror is rebuilt from the FP64 state on resume), with the CME tracer in FP64 (set from
c, so rho c is one rounding away: the tracer agrees to 1e-13, the MHD state bit for bit)."""
import numpy as np
import pytest

from paper_2501_15923_gb300 import inputs as I

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


@pytest.mark.parametrize("prec,tracer", [(0, False), (2, False), (0, True)])
def test_resumed_run_is_bit_identical(ic, prec, tracer):
    w = I.dynamic_cme(grid=I.Grid(48, 12, 24))
    w.opts = I.Options(tracer=int(tracer))
    whole = ic.from_workload(w, precision=prec)
    whole.sample(w.traj, cap=1)
    whole.step(5)
    U5, t5 = whole.get_state()
    c5 = whole.get_tracer() if tracer else None
    whole.sample(None, cap=16)                  # drain the first five steps' records
    whole.step(4)
    U9, t9 = whole.get_state()
    rec_w, n_w = whole.sample(None, cap=16)

    resumed = ic.from_workload(w, precision=prec)
    resumed.set_state(U5, t5)
    if tracer:
        resumed.set_tracer(c5)
    resumed.sample(w.traj, cap=1)               # registers the probes (one record at t5)
    resumed.sample(None, cap=16)
    resumed.step(4)
    U9r, t9r = resumed.get_state()
    rec_r, n_r = resumed.sample(None, cap=16)
    assert t9r == t9 and np.array_equal(U9r, U9)
    assert n_r == n_w == 4 and np.array_equal(rec_r[:n_r], rec_w[:n_w])
    if tracer:
        # icarus_set_tracer takes c and stores rho c = rho x c, one rounding away from the
        # uninterrupted run's rho c: the passive tracer agrees to rounding, the MHD state exactly
        assert np.abs(resumed.get_tracer() - whole.get_tracer()).max() <= 1e-13
    whole.close()
    resumed.close()
