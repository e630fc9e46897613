"""The solver's sticky failure status on the GPU: a non-finite state (ENONFINITE) and, with
options.strict_floors, a floor activation (EFLOOR).

The faults are made on the host: a NaN written into one cell through icarus_set_state, or a
state with negative pressures (the perturbed static-sheet state whose floor counts the parity
tests compare with the oracle). Nothing on the device faults: the update kernel records what it
sees in the status word, the synchronising calls report it, and icarus_step reads its host-mapped
copy without synchronising and launches nothing while it is set. icarus_set_state clears it.
"""
import numpy as np
import pytest

from paper_2501_15923_gb300 import inputs as I

pytestmark = pytest.mark.gpu
ENONFINITE, EFLOOR = -5, -7


@pytest.fixture(scope="module")
def ic():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_15923_gb300 import build
    build.build()
    from paper_2501_15923_gb300 import icarus
    return icarus


def raw_step(ic, s, n=1):
    return ic.load().icarus_step(s.ctx, n)


def status_code(ic, s):
    return s.status()[0]          # icarus_status: (return code, floor activations)


def floor_state(U):
    Up = I.perturbed_state(U.shape, 11, U, 2e-2)
    Up[2] += 0.05 * np.abs(U[1]).max() * I.perturbed_state(U.shape[1:], 12, np.ones(U.shape[1:]), 1.0)
    Up[6] += 0.05 * np.abs(U[5]).max() * I.perturbed_state(U.shape[1:], 13, np.ones(U.shape[1:]), 1.0)
    return Up


@pytest.mark.parametrize("precision", [0, 2, 1])
def test_nan_in_the_state_is_reported_and_sticky(ic, precision):
    w = I.static_sheet()
    s = ic.from_workload(w, precision=precision)
    U, t = s.get_state()
    bad = U.copy()
    bad[0, 9, 5, 30] = np.nan
    s.set_state(bad, t)
    assert raw_step(ic, s, 2) in (0, ENONFINITE)            # may still be in flight: no sync here
    assert status_code(ic, s) == ENONFINITE                 # the synchronising call reports it
    assert raw_step(ic, s, 1) == ENONFINITE                 # sticky: icarus_step launches nothing
    assert "non-finite" in ic.load().icarus_last_error().decode()
    with pytest.raises(ic.IcarusError) as e:
        s.get_state()
    assert e.value.code == ENONFINITE
    s.set_state(U, t)                                       # a finite state clears the status
    assert raw_step(ic, s, 3) == 0
    assert status_code(ic, s) == 0 and raw_step(ic, s, 1) == 0
    s.close()


def test_strict_floors_report_efloor(ic):
    """The same floor-active state: counted silently by default, EFLOOR (sticky) in strict mode,
    with the same floor count, the same stepped state and no effect on a floor-free state."""
    w = I.static_sheet()
    lax = ic.from_workload(w)
    w.opts = I.Options(strict_floors=1)
    strict = ic.from_workload(w)
    U, t = lax.get_state()
    assert status_code(ic, strict) == 0
    assert raw_step(ic, strict, 2) == 0 and status_code(ic, strict) == 0   # no floor: no error
    Up = floor_state(U)
    res = []
    for s in (lax, strict):
        s.set_state(Up, 0.01)
        f0 = s.status()[1]
        assert raw_step(ic, s, 1) == 0
        code, hits = s.status()
        res.append((code, hits - f0, s))
    assert res[0][0] == 0 and res[0][1] > 0
    assert res[1][0] == EFLOOR and res[1][1] == res[0][1]    # the same floors, counted the same
    assert raw_step(ic, strict, 1) == EFLOOR
    assert "strict_floors" in ic.load().icarus_last_error().decode()
    with pytest.raises(ic.IcarusError) as e:
        strict.get_state()
    assert e.value.code == EFLOOR
    lax.close()
    strict.close()
