"""The square root of the FP64 Riemann flux's wave speeds against the correctly rounded one.

The fast magnetosonic speeds inside the flux take their two roots from a single-precision
reciprocal-root estimate and two Newton corrections (five FP64 operations): after the first the
relative error is about 1.5 e^2 for an estimate error e below 2^-22.9 + 2^-24, after the second
e times that, so only the final rounding remains: within one ulp of the correctly rounded root,
and equal to it almost everywhere. Checked here against the library's sqrt on the device and
numpy's on the host, over the whole normal range, both ends of the mantissa interval [1, 4) and
the special values, which take the library root.
"""
import ctypes as C

import numpy as np
import pytest

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


def roots(ic, x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.zeros(2 * len(x))
    rc = ic.load().icarus_root_check(len(x), x.ctypes.data_as(C.c_void_p), y.ctypes.data_as(C.c_void_p))
    assert rc == 0
    return y[0::2], y[1::2]


def test_within_one_ulp_of_the_correctly_rounded_root(ic):
    rng = np.random.default_rng(7)
    tiny = np.finfo(np.float64).tiny
    x = np.concatenate([10.0 ** rng.uniform(-307, 308, 200_000),
                        rng.uniform(0.0, 4.0, 100_000) + tiny,
                        np.ldexp(1.0, np.arange(-1022, 1024)),                       # m = 1
                        np.ldexp(np.nextafter(4.0, 0.0), np.arange(-1022, 1022, 2)),  # m just below 4
                        np.ldexp(np.nextafter(2.0, 0.0), np.arange(-1022, 1022, 2)),
                        [tiny, np.finfo(np.float64).max, 1.0, 2.0, 3.0]])
    y, ref = roots(ic, x)
    assert np.array_equal(ref, np.sqrt(x))                  # the library root is correctly rounded
    ulps = np.abs(y - ref) / np.spacing(ref)
    assert ulps.max() <= 1.0, (ulps.max(), x[np.argmax(ulps)])
    assert np.mean(y == ref) > 0.999, np.mean(y == ref)


def test_special_values_take_the_library_root(ic):
    x = np.array([0.0, -0.0, 5e-324, 1e-310, np.inf, -1.0, -np.inf, np.nan])
    y, ref = roots(ic, x)
    same = (y == ref) | (np.isnan(y) & np.isnan(ref))
    assert same.all(), (y, ref)
    assert np.isnan(y[5]) and y[0] == 0.0 and y[4] == np.inf
