"""Failure detection on the device without a fault: the bounded mbarrier wait
that every kernel uses gives up, the status reaches the host as
CM_ERR_TIMEOUT, tensor memory is released, and the context keeps working."""
import numpy as np
import pytest

import oracle
import paper_2505_22089_b300 as cm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_the_context_survives():
    for polls in (1, 1024, 1 << 14):
        with pytest.raises(cm.CMError) as e:
            cm.check(cm.lib().cm_selftest_wait(polls, cm._stream(None)))
        assert e.value.status == cm.CM_ERR_TIMEOUT
    # tensor memory was freed and the context is usable: a tcgen05 kernel runs and is exact
    rng = np.random.default_rng(1)
    desc = rng.integers(0, 256, (600, 128)).astype(np.uint8)
    best, d1, d2, rows = cm.nn_pairs(torch.from_numpy(desc).cuda(), [300, 300], [(0, 1)])
    o = oracle.brute_nn(desc[:300], desc[300:])
    assert np.array_equal(best.cpu().numpy(), o["best_j"])
