"""Pins of the learned-closure oracle (FP64 conv3d layer, its gradients, the restriction)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2501_15923_gb300 import inputs as I


def rnd(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


def test_forward_brute_force_definition():
    """One output value written out from the definition (padding by index arithmetic)."""
    x, w, b = rnd((3, 4, 5, 2), 1), rnd((3, 27, 2), 2), rnd(3, 3)
    y = O.conv3d_forward(x, w, b, 0)
    n3, n2, n1, _ = x.shape
    for (k, j, i) in [(0, 0, 0), (2, 3, 4), (1, 2, 0), (0, 3, 2)]:
        for o in range(3):
            s = b[o]
            for d3 in (-1, 0, 1):
                for d2 in (-1, 0, 1):
                    for d1 in (-1, 0, 1):
                        t = (d3 + 1) * 9 + (d2 + 1) * 3 + (d1 + 1)
                        ii = min(max(i + d1, 0), n1 - 1)          # replicate
                        jj = min(max(j + d2, 0), n2 - 1)          # replicate
                        kk = (k + d3) % n3                        # circular
                        s += w[o, t] @ x[kk, jj, ii]
            assert abs(y[k, j, i, o] - s) < 1e-12


def test_relu_and_identity_on_constant_input():
    """Constant input: every output equals b + x * sum(w) (the padding copies the constant)."""
    x = np.full((3, 3, 4, 2), 0.7)
    w, b = rnd((2, 27, 2), 4), np.array([0.1, -50.0])
    y = O.conv3d_forward(x, w, b, 1)
    ref = np.maximum(b + 0.7 * w.sum(axis=(1, 2)), 0.0)
    assert np.allclose(y, ref[None, None, None, :], rtol=1e-13)


@pytest.mark.parametrize("act", [0, 1])
def test_gradients_central_differences(act):
    """dx, dw, db against central finite differences of L = sum(g * y)."""
    x, w, b = rnd((3, 3, 4, 2), 5), rnd((3, 27, 2), 6), rnd(3, 7) * 0.1
    g = rnd((3, 3, 4, 3), 8)
    y = O.conv3d_forward(x, w, b, act)
    dx, dw, db = O.conv3d_backward(x, w, y, g, act)
    L = lambda xx, ww, bb: float((g * O.conv3d_forward(xx, ww, bb, act)).sum())
    h = 1e-6
    rng = np.random.default_rng(9)
    for _ in range(12):
        idx = tuple(rng.integers(0, s) for s in x.shape)
        xp, xm = x.copy(), x.copy()
        xp[idx] += h; xm[idx] -= h
        assert abs((L(xp, w, b) - L(xm, w, b)) / (2 * h) - dx[idx]) < 1e-6 * (1 + abs(dx[idx]))
        idw = tuple(rng.integers(0, s) for s in w.shape)
        wp, wm = w.copy(), w.copy()
        wp[idw] += h; wm[idw] -= h
        assert abs((L(x, wp, b) - L(x, wm, b)) / (2 * h) - dw[idw]) < 1e-6 * (1 + abs(dw[idw]))
    for o in range(3):
        bp, bm = b.copy(), b.copy()
        bp[o] += h; bm[o] -= h
        assert abs((L(x, w, bp) - L(x, w, bm)) / (2 * h) - db[o]) < 1e-6 * (1 + abs(db[o]))


def test_backward_is_adjoint_of_forward():
    """<g, conv(x)> = <dx, x> + <db, 1>-part for the linear layer: exact linearity check."""
    x, w = rnd((2, 3, 4, 3), 10), rnd((2, 27, 3), 11)
    b = np.zeros(2)
    g = rnd((2, 3, 4, 2), 12)
    y = O.conv3d_forward(x, w, b, 0)
    dx, dw, _ = O.conv3d_backward(x, w, y, g, 0)
    assert abs((g * y).sum() - (dx * x).sum()) < 1e-10 * abs((g * y).sum())
    assert abs((g * y).sum() - (dw * w).sum()) < 1e-10 * abs((g * y).sum())


def test_restriction_conserves_volume_integrals():
    g = I.Grid(8, 4, 6)
    o = O.Oracle(g, 1.5, 0.0, I.Options())
    vol = o.volumes()
    Uf = rnd((8,) + vol.shape, 13) + 3.0
    Uc = O.restrict(Uf, vol)
    volc = vol.reshape(3, 2, 2, 2, 4, 2).sum(axis=(1, 3, 5))
    for v in range(8):
        assert abs((Uc[v] * volc).sum() - (Uf[v] * vol).sum()) < 1e-12 * np.abs(Uf[v] * vol).sum()
    # a constant stays constant
    Uc1 = O.restrict(np.ones_like(Uf), vol)
    assert np.allclose(Uc1, 1.0, rtol=1e-15)
