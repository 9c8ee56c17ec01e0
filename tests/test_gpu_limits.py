"""GPU parity at the size limits: images of 65,535 descriptors (the most a
16-bit database index addresses; ragged against every tile size), in the
FP32 and BF16 forms and K = 16, L = 8; the exhaustive matcher and VLAD on
the same images.  Checked against the oracle like the other parity tests."""
import numpy as np
import pytest

import oracle
import paper_2505_22089_b300 as cm
import synth
from gpu_common import compare_hash, compare_match, gpu_match, oparams
from oracle import vlad as ovlad

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N_MAX = 65535


@pytest.fixture(scope="module")
def big_pair():
    wl = synth.pair2k(n=N_MAX, shared=20000)
    return wl, wl.generate()


@pytest.mark.parametrize("kw", [dict(rerank="fp32"), dict(rerank="bf16"), dict(rerank="int", K=16, L=8)])
def test_cascade_matching_at_the_largest_image(big_pair, kw):
    wl, desc = big_pair
    p = cm.Params.make(**kw)
    index = cm.Index.build(p, wl.n_desc, torch.from_numpy(desc).cuda())
    pairs = [[0, 1], [1, 0]]
    plan, res = gpu_match(index, pairs, topk=False)
    oix = oracle.Index(desc, wl.n_desc, oparams(p))
    affected, n_diff, n_marg, n_bits = compare_hash(index, oix, [0, 1], p)
    assert n_diff <= 1e-4 * n_bits
    rows, excl, jac = compare_match(plan, res, oix, pairs, p, affected, check_topk=False)
    assert rows + excl == 2 * N_MAX
    assert excl <= 0.02 * (rows + excl) + 10 and jac >= 0.999, (rows, excl, jac)


def test_exhaustive_nn_at_the_largest_image(big_pair):
    wl, desc = big_pair
    best, d1, d2, rows = cm.nn_pairs(torch.from_numpy(desc).cuda(), wl.n_desc, [(0, 1)])
    best, d1, d2 = best.cpu().numpy(), d1.cpu().numpy(), d2.cpu().numpy()
    assert len(best) == N_MAX
    # sampled queries (first, last and random rows) against the brute force over all of J
    rng = np.random.default_rng(3)
    q = np.unique(np.concatenate([np.arange(64), np.arange(N_MAX - 64, N_MAX), rng.integers(0, N_MAX, 128)]))
    o = oracle.brute_nn(desc[q], desc[N_MAX:])
    assert np.array_equal(best[q], o["best_j"])
    assert np.array_equal(d1[q], o["d1sq"].astype(np.int64))
    assert np.array_equal(d2[q], o["d2sq"].astype(np.int64))


def test_vlad_at_the_largest_image(big_pair):
    wl, desc = big_pair
    rng = np.random.default_rng(4)
    cb = desc[rng.choice(len(desc), 256, replace=False)].copy()
    v, a = cm.vlad_encode(torch.from_numpy(desc).cuda(), wl.n_desc, torch.from_numpy(cb).cuda(), want_assign=True)
    want, wa = ovlad.encode(desc[:N_MAX], [N_MAX], cb)
    assert np.array_equal(a.cpu().numpy()[:N_MAX], wa)
    assert np.abs(v.cpu().numpy()[0] - want[0]).max() <= 2e-6
