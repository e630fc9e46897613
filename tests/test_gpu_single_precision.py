"""The single-precision forms (FP32 state, MIXED) against the FP64 oracle, two consecutive steps
from perturbed states inside the CME window, within the reduced-precision bar (2e-5 of each
field's scale): sizes ragged in every direction (one phi plane, three, 37), TVDLF with Linde
diffusion and HLL without div-B control, spherical and a random periodic Cartesian box."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from oracle.oracle import from_workload as oracle_workload
from paper_2501_15923_gb300 import inputs as I

from .helpers import cart_grid
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


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("shape", [(37, 9, 7), (64, 12, 37), (40, 10, 3), (33, 16, 16), (20, 10, 1), (96, 16, 48)])
@pytest.mark.parametrize("flux,divb", [(I.FLUX_TVDLF, I.DIVB_LINDE), (I.FLUX_HLL, I.DIVB_NONE),
                                       (I.FLUX_TVDLF, I.DIVB_POWELL)])
def test_single_precision_steps_match_oracle(ic, prec, shape, flux, divb):
    w = I.dynamic_cme(grid=I.Grid(*shape))
    w.opts = I.Options(flux=flux, divb=divb)
    s, orc = ic.from_workload(w, precision=prec), oracle_workload(w)
    U, _ = s.get_state()
    Up = I.perturbed_state(U.shape, 41, U, 1e-3)
    t = (w.cmes[0, 0] + 1800.0) / orc.scales()["t0"]
    for _ in range(2):
        s.set_state(Up, t)
        orc.set_state(Up, t)
        s.step(1)
        orc.step()
        Ug, tg = s.get_state()
        Uo, to = orc.get_state()
        assert field_errors(Ug, Uo).max() <= 2e-5, field_errors(Ug, Uo)
        assert abs(tg - to) <= 1e-5 * to
        Up, t = Ug, tg
    s.close()


@pytest.mark.parametrize("prec", [1, 2])
def test_single_precision_cartesian_periodic_box(ic, prec):
    """A random periodic box (every face of every direction non-trivial), one step."""
    g = cart_grid(24, 10, 35)
    opts = I.Options(gravity=0)
    s = ic.Solver(g, 5.0 / 3.0, 0.0, opts, precision=prec)
    o = Oracle(g, 5.0 / 3.0, 0.0, opts)
    rng = np.random.default_rng(3)
    W = np.empty((8, g.n3, g.n2, g.n1))
    W[0] = rng.uniform(0.5, 1.5, W.shape[1:])
    W[1:4] = rng.uniform(-0.5, 0.5, (3,) + W.shape[1:])
    W[4] = rng.uniform(0.5, 1.0, W.shape[1:])
    W[5:8] = rng.uniform(-0.5, 0.5, (3,) + W.shape[1:])
    U = np.empty_like(W)
    U[0], U[1:4], U[5:8] = W[0], W[0] * W[1:4], W[5:8]
    U[4] = W[4] / (5.0 / 3.0 - 1.0) + 0.5 * W[0] * (W[1:4] ** 2).sum(0) + 0.5 * (W[5:8] ** 2).sum(0)
    s.set_state(U, 0.0)
    o.set_state(U, 0.0)
    s.step(1)
    o.step()
    assert field_errors(s.get_state()[0], o.get_state()[0]).max() <= 2e-5
    s.close()
