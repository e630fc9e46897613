"""Batched ensemble (one persistent cooperative launch per step) against members run alone.

Every member of a batch must be bit-identical to the same member advanced by its own context:
the per-face and per-cell arithmetic is shared, only the work distribution differs. Members have
uneven grids and different drivers, so their dt (and t) differ.
"""
import numpy as np
import pytest

from paper_2501_15923_gb300 import inputs as I

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


def members():
    shapes = [(40, 10, 16), (64, 12, 24), (33, 9, 20), (96, 16, 32)]
    ws = []
    for q, s in enumerate(shapes):
        w = I.dynamic_cme(seed=40 + q, grid=I.Grid(*s))
        ws.append(w)
    return ws


@pytest.mark.parametrize("prec", [0, 2])
def test_batch_members_bit_identical_to_single_runs(ic, prec):
    ws = members()
    b = ic.Batch(ws, precision=prec)
    tiles = b.autotune(2)
    assert all(0 <= r < 3 and 0 <= t < 2 for r, t in tiles)
    b.step(4)
    assert b.status() == 0
    times = []
    for m, w in enumerate(ws):
        Ub, tb = b.get_state(m)
        s = ic.from_workload(w, precision=prec)
        s.step(4)
        Us, ts = s.get_state()
        if prec == 2:
            # the configured ensemble form: bit-identical to the member run alone
            assert ts == tb, (m, ts, tb)
            assert np.array_equal(Ub, Us), (m, np.abs(Ub - Us).max())
        else:
            # FP64: the same operations, compiled into a different kernel; the compiler's choice of
            # fused multiply-adds may differ, so agreement is to rounding (1e-13 of the scale)
            scale = np.abs(Us).reshape(8, -1).max(1)[:, None]
            assert np.all(np.abs(Ub - Us).reshape(8, -1) <= 1e-13 * scale), (m, np.abs(Ub - Us).max())
            assert abs(ts - tb) <= 1e-13 * ts
        times.append(tb)
        s.close()
    assert len(set(times)) == len(times)      # every member advanced with its own dt
    b.close()


def test_batch_probes_and_tile_variants(ic):
    """Every tile candidate gives the same bits; probes are recorded per member per step."""
    ws = members()[:2]
    ref = None
    for cfg_r in range(3):
        for cfg_t in range(2):
            b = ic.Batch(ws, precision=2)
            b.register_probes()
            b.set_tiles(cfg_r, cfg_t)
            b.step(2)
            assert b.status() == 0
            U, _ = b.get_state(1)
            if ref is None:
                ref = U
            assert np.array_equal(U, ref), (cfg_r, cfg_t)
            rec, n = b.sample(0, cap=8)
            assert n == 2 and np.all(rec[:, :, 1] > 0)
            info = b.info()
            assert info["members"] == 2 and info["blocks"] >= 152
            b.close()


def test_barrier_wait_is_bounded(ic):
    """A block that never reaches the batched form's grid barrier makes the others give up.

    The failure is made by a block that skips the barrier (nothing else ever releases the
    waiters), the wait limit is about a millisecond; the waiters record ETIMEOUT and return,
    and the device stays usable: a full barrier and a batched step still succeed afterwards.
    """
    lib = ic.load()
    ETIMEOUT = -6
    assert lib.icarus_batch_barrier_selftest(16, -1, 2_000_000) == 0
    assert lib.icarus_batch_barrier_selftest(16, 5, 2_000_000) == ETIMEOUT
    assert "never arrived" in lib.icarus_last_error().decode()
    assert lib.icarus_batch_barrier_selftest(16, 0, 2_000_000) == ETIMEOUT
    assert lib.icarus_batch_barrier_selftest(64, -1, 2_000_000) == 0
    b = ic.Batch(members()[:2], precision=2)
    b.step(2)
    assert b.status() == 0
    b.close()


# ---------------------------------------------------------------------------------------------
# production-size members against the FP64 oracle
PROD_SHAPES = [(512, 64, 128), (128, 32, 64), (384, 48, 96), (256, 40, 80)]


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (2, 2e-5)])
def test_batch_production_members_match_oracle(ic, mode, prec, tol):
    """Members of the sizes the ensemble workload draws (the 512 x 64 x 128 grid among them), each
    stepped by the batched launch (persistent kernel, mode 0; one launch per phase, mode 1; the
    members' own kernels as parallel branches of one graph, mode 2) from a
    perturbed state at a time inside its CME window, compared field by field with one oracle step
    from the same state: FP64 within 1e-12 and MIXED within 2e-5 of each field's scale (the
    single-solver bars), dt within 1e-13 (FP64). Two consecutive steps; the oracle restarts from the
    batch's state at each."""
    from oracle.oracle import from_workload as oracle_workload
    from .test_gpu_parity import field_errors
    ws = [I.dynamic_cme(seed=60 + q, grid=I.Grid(*s)) for q, s in enumerate(PROD_SHAPES)]
    b = ic.Batch(ws, precision=prec, mode=mode)
    b.autotune(1)
    t0 = 1.495978707e11 / 1e5
    starts = []
    for m, w in enumerate(ws):
        U, _ = b.get_state(m)
        Up = I.perturbed_state(U.shape, 70 + m, U, 1e-3)
        t = (w.cmes[0, 0] + 1800.0) / t0
        b.set_state(m, Up, t)
        starts.append((Up, t))
    for _ in range(2):
        b.step(1)
        assert b.status() == 0
        nxt = []
        for m, w in enumerate(ws):
            orc = oracle_workload(w)
            orc.set_state(*starts[m])
            orc.step()
            Uo, to = orc.get_state()
            Ub, tb = b.get_state(m)
            err = field_errors(Ub, Uo)
            assert err.max() <= tol, (m, w.grid.n1, err)
            if prec == 0:
                assert abs(tb - to) <= 1e-13 * to, (m, tb, to)
            else:
                assert abs(tb - to) <= 1e-5 * to, (m, tb, to)
            nxt.append((Ub, tb))
            del orc
        starts = nxt
    b.close()


def test_batch_modes_agree(ic):
    """The three launch forms give the same MIXED step (same per-cell arithmetic)."""
    ws = members()
    out = []
    for mode in (0, 1, 2):
        b = ic.Batch(ws, precision=2, mode=mode)
        b.set_tiles(1, 1)
        b.step(3)
        assert b.status() == 0 and b.info()["mode"] == mode
        out.append([b.get_state(m) for m in range(len(ws))])
        b.close()
    for other in out[1:]:
        for (Ua, ta), (Ub, tb) in zip(out[0], other):
            assert abs(ta - tb) <= 1e-6 * ta
            scale = np.abs(Ua).reshape(8, -1).max(1)[:, None]
            assert np.all(np.abs(Ua - Ub).reshape(8, -1) <= 1e-6 * scale)
