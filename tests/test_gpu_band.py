"""Static refinement band (a radial band of narrower cells, the fixed stand-in for adaptive
refinement) on the GPU against the FP64 oracle: the metric tables built from the band's edges, one
step inside the CME window and one between maps (<= 1e-12 of each field's scale), and the probe
stencil indices (exact) for probes on both sides of and inside the band."""
import numpy as np
import pytest

from oracle.oracle import from_workload as oracle_workload
from paper_2501_15923_gb300 import inputs as I

from .test_gpu_parity import TOL, assert_step

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


@pytest.mark.parametrize("stretch,f,band", [(1, 4, (0.8, 1.2)), (0, 3, (0.5, 1.1))])
def test_band_step_parity(ic, stretch, f, band):
    g = I.Grid(72, 12, 24, stretch=stretch, band_refine=f, band_lo=band[0], band_hi=band[1])
    w = I.dynamic_cme(grid=g)
    gpu, orc = ic.from_workload(w), oracle_workload(w)
    sc = orc.scales()
    U, _ = gpu.get_state()
    for t in ((w.cmes[0, 0] + 1800.0) / sc["t0"], 1.37 * I.DAY / sc["t0"]):
        assert_step(gpu, orc, U, t)
    gpu.close()


def test_band_probe_indices(ic):
    g = I.Grid(72, 12, 24, band_refine=4, band_lo=0.8, band_hi=1.2)
    w = I.dynamic_cme(grid=g)
    gpu, orc = ic.from_workload(w), oracle_workload(w)
    e = orc.edges(0)
    assert np.diff(np.log(e)).min() < 0.3 * np.diff(np.log(e)).max()     # the band is there
    U, _ = gpu.get_state()
    sc = orc.scales()
    for t_si in (0.0, 2.71 * I.DAY, 9.99 * I.DAY):
        t = t_si / sc["t0"]
        gpu.set_state(U, t)
        orc.set_state(U, t)
        rec, n = gpu.sample(w.traj, cap=1)
        ref = orc.sample(w.traj)
        assert n == 1
        assert np.array_equal(rec[0][:, 10:13], ref[:, 10:13])
        scale = np.abs(ref).max(0)
        scale[scale == 0] = 1
        assert np.all(np.abs(rec[0][:, :10] - ref[:, :10]) <= TOL * scale[:10])
    gpu.close()
