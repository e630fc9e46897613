"""The fused one-kernel stage of the single-precision forms (FP32 state, MIXED; options.fused)
against the separate flux / div-B / update kernels and against the FP64 oracle.

Both GPU paths compute the same face states, Riemann fluxes, div B and update in single precision
(Sect. 2.1 scheme); they may differ only by the order in which the compiler contracts products into
fused multiply-adds, so one step agrees to <= 1e-6 of each field's scale (a few float ulps of the
largest term). Against the FP64 oracle one step agrees to <= 2e-5 of each field's scale, the
single-precision rounding of the flux differences that form the update. dt agrees to <= 1e-6.
"""
import numpy as np
import pytest

from oracle.oracle import Oracle, cons_from_prim, prim_from_cons
from oracle.oracle import from_workload as oracle_workload
from paper_2501_15923_gb300 import inputs as I

from .helpers import cart_grid, sph_grid
from .test_gpu_parity import field_errors

pytestmark = pytest.mark.gpu
PRECS = [1, 2]     # ICARUS_FP32, ICARUS_MIXED
TOL_PATHS, TOL_ORACLE = 1e-6, 2e-5


@pytest.fixture(scope="module")
def ic():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_15923_gb300 import build
    build.build()
    from paper_2501_15923_gb300 import icarus
    return icarus


def one_step(s, U, t):
    s.set_state(U, t)
    s.step(1)
    return s.get_state()


def compare_paths(ic, make, U, t, prec, orc=None, steps=1):
    fused, plain = make(prec, False), make(prec, True)
    assert fused.launches_per_step < plain.launches_per_step
    Uf, tf, Up, tp = U, t, U, t
    for _ in range(steps):
        Uf, tf = one_step(fused, Uf, tf)
        Up, tp = one_step(plain, Up, tp)
    assert field_errors(Uf, Up).max() <= TOL_PATHS * steps, field_errors(Uf, Up)
    assert abs(tf - tp) <= 1e-6 * abs(tp - t) * steps + 1e-300
    if orc is not None and steps == 1:
        orc.set_state(U, t)
        orc.step()
        Uo, to = orc.get_state()
        assert field_errors(Uf, Uo).max() <= TOL_ORACLE, field_errors(Uf, Uo)
        assert abs(tf - to) <= 1e-5 * abs(to - t)
    assert fused.status()[0] == 0
    fused.close()
    plain.close()


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n", [(60, 16, 32), (37, 9, 7), (129, 17, 33), (2, 10, 3), (70, 12, 80)])
def test_fused_stage_grids(ic, prec, n):
    """Ragged tiles in r and theta, a phi chunk that is cut short (80 = 5 x 16), tiny grids."""
    w = I.dynamic_cme(grid=I.Grid(*n))
    make = lambda p, unf: ic.from_workload(w, precision=p, fused=not unf)
    s = make(prec, False)
    U, t = s.get_state()
    s.close()
    compare_paths(ic, make, U, t, prec, oracle_workload(w))


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("lim,flux,divb,grav", [
    (I.LIM_MINMOD, I.FLUX_TVDLF, I.DIVB_LINDE, 1),
    (I.LIM_MC, I.FLUX_HLL, I.DIVB_LINDE, 1),
    (I.LIM_VANLEER, I.FLUX_HLL, I.DIVB_NONE, 0),
])
def test_fused_stage_options_perturbed(ic, prec, lim, flux, divb, grav):
    w = I.static_sheet()
    w.opts = I.Options(limiter=lim, flux=flux, divb=divb, gravity=grav)
    make = lambda p, unf: ic.from_workload(w, precision=p, fused=not unf)
    s = make(prec, False)
    U, _ = s.get_state()
    s.close()
    # perturbed in primitive space so that the pressure stays positive: a state whose recovered
    # pressure is a near-total cancellation of its energy has no single-precision answer
    W = prim_from_cons(U, w.gamma)
    Wp = I.perturbed_state(W.shape, 11, W, 2e-2)
    noise = lambda seed: I.perturbed_state(W.shape[1:], seed, np.ones(W.shape[1:]), 1.0) - 1.0
    Wp[2] += 0.05 * np.abs(W[1]) * noise(12)
    Wp[6] += 0.05 * np.sqrt((W[5:8] ** 2).sum(0)) * noise(13)
    compare_paths(ic, make, cons_from_prim(Wp, w.gamma), 0.01, prec, oracle_workload(w))


@pytest.mark.parametrize("prec", PRECS)
def test_fused_stage_twenty_steps_with_cme(ic, prec):
    """Twenty consecutive steps through the CME insertion window on a reduced grid."""
    w = I.dynamic_cme(grid=I.Grid(48, 12, 24))
    make = lambda p, unf: ic.from_workload(w, precision=p, fused=not unf)
    s = make(prec, False)
    U, _ = s.get_state()
    s.close()
    t = (w.cmes[0, 0] + 600.0) / oracle_workload(w).scales()["t0"]
    compare_paths(ic, make, U, t, prec, steps=20)


@pytest.mark.parametrize("prec", PRECS)
def test_fused_stage_cartesian_and_reflecting(ic, prec):
    """Cartesian periodic box with Linde cleaning and a reflecting spherical shell."""
    rng = np.random.default_rng(5)
    g = cart_grid(40, 20, 18)
    o = I.Options(divb=I.DIVB_LINDE)
    W = np.zeros((8, 18, 20, 40))
    W[0] = 1.0 + 0.2 * rng.random(W.shape[1:])
    W[1:4] = 0.3 * rng.standard_normal((3,) + W.shape[1:])
    W[4] = 1.0 + 0.2 * rng.random(W.shape[1:])
    W[5:8] = 0.5 * rng.standard_normal((3,) + W.shape[1:])
    make = lambda p, unf: ic.Solver(g, 5 / 3, 0.0, o, precision=p, fused=not unf)
    compare_paths(ic, make, cons_from_prim(W, 5 / 3), 0.0, prec, Oracle(g, 5 / 3, 0.0, o))
    g = sph_grid(20, 10, 16, bc=(I.BC_REFLECT,) * 4 + (I.BC_PERIODIC,) * 2, r=(0.3, 1.0))
    o = I.Options(gravity=0)
    W = np.zeros((8, 16, 10, 20))
    W[0] = 1.0 + 0.3 * rng.random(W.shape[1:])
    W[1:4] = 0.2 * rng.standard_normal((3,) + W.shape[1:])
    W[4] = 2.0 + rng.random(W.shape[1:])
    W[5:8] = 0.4 * rng.standard_normal((3,) + W.shape[1:])
    make = lambda p, unf: ic.Solver(g, 1.5, I.OMEGA_SUN, o, precision=p, fused=not unf)
    compare_paths(ic, make, cons_from_prim(W, 1.5), 0.0, prec, Oracle(g, 1.5, I.OMEGA_SUN, o))
