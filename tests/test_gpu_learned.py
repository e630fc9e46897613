"""The learned closure end to end on a small grid: solver-generated pairs, GPU training with the
closure's own kernels, and the gain of the trained network on pairs it has not seen."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_15923_gb300 import build
    build.build()
    from paper_2501_15923_gb300 import learned
    return learned, torch


def test_pairs_training_and_heldout_gain(env):
    learned, torch = env
    pairs = learned.generate_pairs([100, 101, 102], windows=6, spinup_days=0.05, fine=(64, 24, 32))
    assert len(pairs) == 18
    train = learned.PairSet(torch)
    for q in range(12):
        train.add(pairs.inputs[q], pairs.targets[q])
    # the target is a genuine coarse/fine discrepancy: nonzero and small against the state
    d = float(torch.linalg.vector_norm(pairs.targets[0])) / float(torch.linalg.vector_norm(pairs.inputs[0]))
    assert 1e-8 < d < 0.2
    net, info = learned.train(train, (32, 12, 16), epochs=40, lr=2e-3)
    assert info["loss"][-1] < 0.5 * info["loss"][0], info["loss"]
    g_train = learned.pair_gain(net, train, range(12))
    g_hold = learned.pair_gain(net, pairs, range(12, 18))     # seed 102: never trained on
    assert g_train > 1.2, g_train
    assert g_hold > 1.05, g_hold
    net.close()


def test_closure_apply_and_evaluation_report(env):
    learned, torch = env
    pairs = learned.generate_pairs([100], windows=4, spinup_days=0.05, fine=(64, 24, 32))
    net, _ = learned.train(pairs, (32, 12, 16), epochs=5, lr=1e-3)
    ev = learned.evaluate(net, 999, 0.05, 0.1, fine=(64, 24, 32))
    for name in ("coarse", "coarse+closure"):
        assert set(ev[name]["probe_error"]) == {"n", "v_r", "|B|"}
        assert all(np.isfinite(v) for v in ev[name]["probe_error"].values())
        assert ev[name]["coarse_steps"] > 0
    assert isinstance(ev["fallback_to_fine"], bool)
    net.close()
