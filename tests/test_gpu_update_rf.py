"""The single-precision forms' default update, which forms the r-face fluxes itself (options.fused
= 0), against the separate r-flux kernel + update (options.fused = 2) and against the FP64 oracle.

Both GPU paths form the same limited slopes, face states and TVDLF / HLL fluxes (Sect. 2.1 scheme)
in single precision and the same update; they differ in where the r fluxes are kept between the two
(shared memory or an HBM array) and in the update kernel the separate path takes: MIXED uses the
same one-cell-per-thread update in both (measured bit-identical at 512 x 64 x 128), FP32 the
two-cells-per-thread update in the separate path, which the compiler may contract into fused
multiply-adds differently. So MIXED holds the two paths to <= 1e-6 of each field's scale per step,
FP32 to the single-precision bar. Against the FP64 oracle one step agrees to <= 2e-5 of each
field's scale, the single-precision bar. Radial sizes cover one row segment, several equal segments
with a ragged last one, and a segment shorter than a warp.
"""
import numpy as np
import pytest

from oracle.oracle import from_workload as oracle_workload
from paper_2501_15923_gb300 import inputs as I

from .test_gpu_parity import field_errors

pytestmark = pytest.mark.gpu
FP32, MIXED = 1, 2
DEFAULT, SEPARATE = 0, 2
TOL_ORACLE = 2e-5
TOL_PATHS = {MIXED: 1e-6, FP32: TOL_ORACLE}


@pytest.fixture(scope="module")
def ic():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_15923_gb300 import build
    build.build()
    from paper_2501_15923_gb300 import icarus
    return icarus


def pair(ic, w, prec):
    return (ic.from_workload(w, precision=prec, fused=DEFAULT),
            ic.from_workload(w, precision=prec, fused=SEPARATE))


@pytest.mark.parametrize("prec", [FP32, MIXED])
@pytest.mark.parametrize("shape", [(37, 9, 7), (300, 10, 5), (520, 10, 3), (20, 10, 1), (64, 12, 37)])
@pytest.mark.parametrize("flux,divb", [(I.FLUX_TVDLF, I.DIVB_LINDE), (I.FLUX_HLL, I.DIVB_NONE),
                                       (I.FLUX_TVDLF, I.DIVB_POWELL)])
def test_update_rf_matches_separate_kernels_and_oracle(ic, prec, shape, flux, divb):
    w = I.dynamic_cme(grid=I.Grid(*shape))
    w.opts = I.Options(flux=flux, divb=divb)
    rf, plain = pair(ic, w, prec)
    assert rf.launches_per_step == plain.launches_per_step - 2          # no r-flux kernel per stage
    orc = oracle_workload(w)
    U, _ = rf.get_state()
    U0 = I.perturbed_state(U.shape, 43, U, 1e-3)
    t0 = (w.cmes[0, 0] + 1800.0) / orc.scales()["t0"]
    Ur, tr, Up, tp = U0, t0, U0, t0
    for n in range(2):
        rf.set_state(Ur, tr)
        plain.set_state(Up, tp)
        rf.step(1)
        plain.step(1)
        Ur, tr = rf.get_state()
        Up, tp = plain.get_state()
        assert field_errors(Ur, Up).max() <= TOL_PATHS[prec] * (n + 1), field_errors(Ur, Up)
        assert abs(tr - tp) <= 1e-6 * abs(tp - t0)
    orc.set_state(U0, t0)
    orc.step()
    rf.set_state(U0, t0)
    rf.step(1)
    Ur, tr = rf.get_state()
    Uo, to = orc.get_state()
    assert field_errors(Ur, Uo).max() <= TOL_ORACLE, field_errors(Ur, Uo)
    assert abs(tr - to) <= 1e-5 * abs(to - t0)
    assert rf.status()[0] == 0
    rf.close()
    plain.close()


@pytest.mark.parametrize("prec", [FP32, MIXED])
@pytest.mark.parametrize("opts", [I.Options(flux=I.FLUX_HLLD), I.Options(tracer=1), I.Options(divb=I.DIVB_GLM)])
def test_update_rf_not_taken_where_not_available(ic, prec, opts):
    """HLLD, the tracer (it reads the r mass fluxes) and GLM keep the separate kernels in the
    default sequence too: the same launches and the same result as options.fused = 2."""
    w = I.dynamic_cme(grid=I.Grid(40, 10, 6))
    w.opts = opts
    a, b = pair(ic, w, prec)
    assert a.launches_per_step == b.launches_per_step
    a.step(3)
    b.step(3)
    Ua, ta = a.get_state()
    Ub, tb = b.get_state()
    assert ta == tb and np.array_equal(Ua, Ub)
    a.close()
    b.close()


@pytest.mark.parametrize("prec", [FP32, MIXED])
def test_update_rf_production_grid(ic, prec):
    """The 512 x 64 x 128 production grid (four full row segments), three steps from the
    relaxed-wind start: the two GPU paths within the path tolerance, dt likewise; MIXED bit for
    bit."""
    w = I.dynamic_cme()
    rf, plain = pair(ic, w, prec)
    rf.step(3)
    plain.step(3)
    Ur, tr = rf.get_state()
    Up, tp = plain.get_state()
    assert field_errors(Ur, Up).max() <= 3 * TOL_PATHS[prec], field_errors(Ur, Up)
    assert abs(tr - tp) <= 1e-6 * tp
    if prec == MIXED:
        assert tr == tp and np.array_equal(Ur, Up)
    assert rf.status()[0] == 0
    rf.close()
    plain.close()
