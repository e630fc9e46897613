"""The closure's tensor-core conv kernels against the FP64 oracle layer.

Inputs, weights and output gradients are rounded to BF16 first and handed to both sides, so the
GPU result differs from the oracle only by its FP32 accumulation (relative ~1e-6); the bar is
2e-5 of each tensor's largest magnitude. This checks the forward pass and the three gradients the
GPU training uses (data, weight, bias), including the ReLU mask and the padding's adjoint. The
shapes cover the tensor-core forward's tiling: ragged 128-voxel tiles along r, several tiles per
r-line, columns walked along k in chunks of 8 with a ring of k-planes that wraps (n3 = 9, 19),
and a single k-plane; and the weight gradient's split of the padded positions over one block per
SM: one 64-position stage per block on the small shapes, four stages (both shared-memory buffers
refilled) on 128 x 16 x 16.
"""
import numpy as np
import pytest

from oracle import oracle as O

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


def bf16(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16      # round to nearest even
    return r.astype(np.uint32).view(np.float32)


@pytest.mark.parametrize("C,Oc,act,shape", [(16, 32, 1, (11, 6, 5)), (32, 32, 1, (9, 7, 4)), (32, 16, 0, (13, 5, 6)),
                                            (32, 32, 1, (40, 12, 10)), (32, 32, 1, (150, 5, 3)),
                                            (16, 32, 1, (256, 3, 2)), (32, 16, 0, (129, 4, 3)),
                                            (32, 32, 1, (140, 3, 19)), (16, 32, 1, (20, 2, 9)),
                                            (32, 16, 0, (7, 3, 1)), (32, 32, 1, (128, 16, 16))])
def test_layer_forward_and_gradients_match_oracle(ic, C, Oc, act, shape):
    n1, n2, n3 = shape
    rng = np.random.default_rng(C * 100 + Oc + n1)
    x = bf16(rng.standard_normal((n3, n2, n1, C)))
    w = bf16(rng.standard_normal((Oc, 27, C)) * 0.1)
    b = bf16(rng.standard_normal(Oc) * 0.1)
    g = bf16(rng.standard_normal((n3, n2, n1, Oc)))
    yo = O.conv3d_forward(x.astype(np.float64), w.astype(np.float64), b.astype(np.float64), act)
    if act:
        # a pre-activation within the FP32 accumulation's rounding of 0 may fall on either side of
        # the ReLU on the GPU; those outputs get a zero gradient on both sides (so the mask there
        # does not matter), and their number is bounded explicitly
        zo = O.conv3d_forward(x.astype(np.float64), w.astype(np.float64), b.astype(np.float64), 0)
        edge = np.abs(zo) <= 1e-5 * np.abs(zo).max()
        assert edge.sum() <= 1e-3 * edge.size + 2, edge.sum()
        g = np.where(edge, np.float32(0), g).astype(np.float32)
    y, dx, dw, db = ic.icarus_conv3d_layer(x, w, b, g, act)
    # the oracle's backward pass takes its own forward output (its ReLU mask), nothing of the GPU's
    dxo, dwo, dbo = O.conv3d_backward(x.astype(np.float64), w.astype(np.float64), yo, g.astype(np.float64), act)
    for got, ref in ((y, yo), (dx, dxo), (dw, dwo), (db, dbo)):
        scale = np.abs(ref).max()
        assert np.abs(got - ref).max() <= 2e-5 * scale, (np.abs(got - ref).max(), scale)


def test_restriction_matches_oracle(ic):
    """icarus_restrict (volume-weighted 2x2x2 average of a fine FP64 state onto the half-resolution
    grid) against the oracle's restriction of the same fine state, on a stretched spherical grid
    with a perturbed state (every cell different)."""
    from oracle.oracle import Oracle, from_workload as oracle_workload
    from paper_2501_15923_gb300 import inputs as I, learned
    w = I.dynamic_cme(grid=I.Grid(32, 24, 16))     # coarse 16 x 12 x 8 keeps its ghosts off the pole
    fine = ic.from_workload(w)
    coarse = ic.from_workload(learned.coarse_workload(w))
    U, t = fine.get_state()
    U = U * I.perturbed_state(U.shape, 5, np.ones(U.shape), 1e-3)
    fine.set_state(U, t)
    ic.icarus_restrict(fine.ctx, coarse.ctx)
    Uc, tc = coarse.get_state()
    vol = oracle_workload(w).volumes()
    ref = O.restrict(U, vol)
    assert tc == t
    np.testing.assert_allclose(Uc, ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())
    fine.close(); coarse.close()


def test_tensor_core_wait_is_bounded(ic):
    """The closure kernels' barrier wait gives up when nothing arrives, and the device stays usable.

    The failure is a shared-memory barrier that expects one arrival and never gets it; after 4096
    polls the wait records the failure and the call returns ETIMEOUT (the status is read and
    cleared). The same wait with its arrival completes, and the tcgen05 forward and gradients
    still match the oracle afterwards.
    """
    lib = ic.load()
    ETIMEOUT = -6
    assert lib.icarus_closure_wait_selftest(1, 4096) == 0
    assert lib.icarus_closure_wait_selftest(0, 4096) == ETIMEOUT
    assert "expired" in lib.icarus_last_error().decode()
    assert lib.icarus_closure_wait_selftest(1, 4096) == 0
    test_layer_forward_and_gradients_match_oracle(ic, 32, 32, 1, (9, 7, 4))
