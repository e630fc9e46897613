"""GLM div-B control on the GPU (divb = DIVB_GLM) against the oracle's GLM, one step at
a time from the same state and psi: the Cartesian standing wave of the P12 pin (dt fixed by a stop
time, so c_h is the same on both sides), a perturbed spherical state whose field has divergence,
with a random psi, several steps, and the driven production workload inside its CME window.
State fields to <= 1e-12 of their scale (as in test_gpu_parity), psi to <= 1e-12 of its largest
magnitude."""
import numpy as np
import pytest

from oracle.oracle import Oracle, cons_from_prim, prim_from_cons
from oracle.oracle import from_workload as oracle_workload
from paper_2501_15923_gb300 import inputs as I

from .helpers import cart_grid
from .test_gpu_parity import TOL, field_errors

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


def step_pair(gpu, orc, U, psi, t, dt_cap=0.0, mom_floor=0.0):
    for s in (gpu, orc):
        s.set_state(U, t)
        s.set_psi(psi)
    if dt_cap:
        gpu.set_stop_time(t + dt_cap)
    gpu.step(1)
    orc.step(dt_cap)
    Ug, tg = gpu.get_state()
    Uo, to = orc.get_state()
    pg, po = gpu.get_psi(), orc.get_psi()
    err = field_errors(Ug, Uo)
    if mom_floor:
        # momenta that start at zero grow only by rounding-level amounts in a few steps: their
        # scale is floored at rho c_s so that the relative bar stays meaningful
        mscale = max(np.sqrt((Uo[1:4] ** 2).sum(0)).max(), mom_floor)
        err[1:4] = np.abs(Ug[1:4] - Uo[1:4]).max() / mscale
    assert err.max() <= TOL, err
    assert abs(tg - to) <= 1e-13 * abs(to) + 1e-300
    assert np.abs(pg - po).max() <= TOL * max(np.abs(po).max(), 1e-300), np.abs(pg - po).max()
    return Uo, po, to


def test_glm_standing_wave(ic):
    g = cart_grid(64, 4, 4)
    o = I.Options(divb=I.DIVB_GLM, glm_alpha=0.0, gravity=0)
    gpu, orc = ic.Solver(g, 1.5, 0.0, o), Oracle(g, 1.5, 0.0, o)
    x = (np.arange(64) + 0.5) / 64
    W = np.zeros((8, 4, 4, 64))
    W[0], W[4], W[6] = 1.0, 1.0, 0.3
    W[5] = 0.5 + 1e-3 * np.sin(2 * np.pi * x)
    U, psi, t = cons_from_prim(W, 1.5), np.zeros((4, 4, 64)), 0.0
    for _ in range(6):
        U, psi, t = step_pair(gpu, orc, U, psi, t, dt_cap=0.25 / 64, mom_floor=np.sqrt(1.5))
    assert np.abs(psi).max() > 1e-5                 # the wave has moved field into psi
    gpu.close()


@pytest.mark.parametrize("alpha", [0.0, 0.1])
def test_glm_perturbed_sphere(ic, alpha):
    w = I.static_sheet()
    w.opts = I.Options(divb=I.DIVB_GLM, glm_alpha=alpha)
    gpu, orc = ic.from_workload(w), oracle_workload(w)
    U, _ = gpu.get_state()
    Wp = I.perturbed_state(U.shape, 21, prim_from_cons(U, w.gamma), 2e-2)
    psi = 1e-3 * (I.perturbed_state(U.shape[1:], 22, np.ones(U.shape[1:]), 1.0) - 1.0)
    U1, p1, t1 = step_pair(gpu, orc, cons_from_prim(Wp, w.gamma), psi, 0.01)
    for _ in range(3):
        U1, p1, t1 = step_pair(gpu, orc, U1, p1, t1)
    gpu.close()


@pytest.mark.parametrize("prec", [1, 2])
def test_glm_single_precision_forms(ic, prec):
    """GLM in the FP32-state and MIXED forms: one step on the perturbed spherical state with psi,
    within the single-precision bar (2e-5 of each field's and of psi's scale)."""
    w = I.static_sheet()
    w.opts = I.Options(divb=I.DIVB_GLM)
    gpu, orc = ic.from_workload(w, precision=prec), oracle_workload(w)
    U, _ = gpu.get_state()
    Wp = I.perturbed_state(U.shape, 21, prim_from_cons(U, w.gamma), 2e-2)
    psi = 1e-3 * (I.perturbed_state(U.shape[1:], 22, np.ones(U.shape[1:]), 1.0) - 1.0)
    Up = cons_from_prim(Wp, w.gamma)
    for s in (gpu, orc):
        s.set_state(Up, 0.01)
        s.set_psi(psi)
    gpu.step(1)
    orc.step()
    Ug, _ = gpu.get_state()
    Uo, _ = orc.get_state()
    assert field_errors(Ug, Uo).max() <= 2e-5
    po = orc.get_psi()
    assert np.abs(gpu.get_psi() - po).max() <= 2e-5 * np.abs(po).max()
    gpu.close()


def test_glm_driven_cme_window(ic):
    w = I.dynamic_cme(grid=I.Grid(48, 12, 24))
    w.opts = I.Options(divb=I.DIVB_GLM)
    gpu, orc = ic.from_workload(w), oracle_workload(w)
    U, _ = gpu.get_state()
    t = (w.cmes[0, 0] + 1800.0) / orc.scales()["t0"]
    step_pair(gpu, orc, U, np.zeros(U.shape[1:]), t)
    gpu.close()


def test_psi_needs_glm(ic):
    w = I.static_sheet()
    gpu = ic.from_workload(w)
    with pytest.raises(ic.IcarusError) as e:
        gpu.set_psi(np.zeros(gpu.shape[1:]))
    assert "EINVAL" in str(e.value)
    gpu.close()
