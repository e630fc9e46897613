"""The FP64 kernels' square root and reciprocal against the correctly rounded ones.

The fast magnetosonic speeds inside the FP64 Riemann flux take their roots, and the face
densities, the van Leer slope sums and rho their reciprocals, from single-precision estimates
(relative error about 2^-23) refined by two Newton steps on the FP64 pipe: after the first the
error is of order e^2, after the second e^3 (root) or e^4 (reciprocal), so only the final rounding
remains: within one ulp of the correctly rounded result, and equal to it in more than 99.9 % (root)
and 99 % (reciprocal, measured 99.3 %) of the cases.
Checked here against the library's sqrt and division on the device and numpy's on the host, over
the whole range each is used on, both ends of the mantissa interval, and the special values,
which take the library operation.
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


def evaluate(ic, x):
    """(root, library root, reciprocal, library reciprocal) of every x on the device."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.zeros(4 * len(x))
    rc = ic.load().icarus_math_check(len(x), x.ctypes.data_as(C.c_void_p), y.ctypes.data_as(C.c_void_p))
    assert rc == 0
    return y[0::4], y[1::4], y[2::4], y[3::4]


def normal_values(rng):
    tiny = np.finfo(np.float64).tiny
    return np.concatenate([10.0 ** rng.uniform(-307, 308, 200_000),
                           rng.uniform(0.0, 4.0, 100_000) + tiny,
                           np.ldexp(1.0, np.arange(-1022, 1024)),                       # m = 1
                           np.ldexp(np.nextafter(4.0, 0.0), np.arange(-1022, 1022, 2)),  # m just below 4
                           np.ldexp(np.nextafter(2.0, 0.0), np.arange(-1022, 1022, 2)),
                           [tiny, np.finfo(np.float64).max, 1.0, 2.0, 3.0]])


def assert_within_one_ulp(y, ref, equal_share):
    ulps = np.abs(y - ref) / np.spacing(np.abs(ref))
    assert ulps.max() <= 1.0, (ulps.max(), np.argmax(ulps))
    assert np.mean(y == ref) > equal_share, np.mean(y == ref)


def test_root_within_one_ulp(ic):
    x = normal_values(np.random.default_rng(7))
    y, ref, _, _ = evaluate(ic, x)
    assert np.array_equal(ref, np.sqrt(x))                  # the library root is correctly rounded
    assert_within_one_ulp(y, ref, 0.999)


def test_reciprocal_within_one_ulp(ic):
    x = normal_values(np.random.default_rng(8))
    x = np.concatenate([x, -x])
    _, _, y, ref = evaluate(ic, x)
    assert np.array_equal(ref, 1.0 / x)                     # the library division is correctly rounded
    assert_within_one_ulp(y, ref, 0.99)


def test_special_values_take_the_library_operation(ic):
    x = np.array([0.0, -0.0, 5e-324, 1e-310, np.inf, -1.0, -np.inf, np.nan])
    y, ref, q, qref = evaluate(ic, x)
    same = (y == ref) | (np.isnan(y) & np.isnan(ref))
    assert same.all(), (y, ref)
    assert np.isnan(y[5]) and y[0] == 0.0 and y[4] == np.inf
    # the reciprocal also leaves the magnitudes outside [2^-1021, 2^1021] to the library
    big = np.ldexp(1.0, 1022)
    x = np.concatenate([x, [big, -big, 2.3e-308, np.finfo(np.float64).max]])
    _, _, q, qref = evaluate(ic, x)
    same = (q == qref) | (np.isnan(q) & np.isnan(qref))
    assert same.all(), (q, qref)
    assert q[0] == np.inf and q[1] == -np.inf and q[4] == 0.0
