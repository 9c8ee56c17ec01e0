"""GPU parity of the exhaustive nearest-neighbour matcher (cm_nn_pairs, the
quality ceiling of Sec. 2.3.1 with every database point a candidate) with the
oracle's brute force: q1, q2 and their squared distances bit for bit and the
exact ratio test, over pairs with empty, one-row and two-row database images,
ragged tiles and chunks, duplicated database rows (ties to the smaller j),
rows at the largest squared norms and two ratio thresholds."""
import numpy as np
import pytest

import oracle
import paper_2505_22089_b300 as cm
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _check(desc, nd, pairs, ratio=(4, 5)):
    off = np.concatenate([[0], np.cumsum(nd)])
    best, d1, d2, rows = cm.nn_pairs(torch.from_numpy(desc).cuda(), nd, pairs, ratio)
    torch.cuda.synchronize()
    best, d1, d2 = best.cpu().numpy(), d1.cpu().numpy(), d2.cpu().numpy()
    for k, (i, j) in enumerate(pairs):
        o = oracle.brute_nn(desc[off[i]:off[i + 1]], desc[off[j]:off[j + 1]], *ratio)
        r0, r1 = rows[k], rows[k + 1]
        assert np.array_equal(best[r0:r1], o["best_j"]), (k, i, j)
        assert np.array_equal(d1[r0:r1], o["d1sq"].astype(np.int64)), (k, i, j)
        assert np.array_equal(d2[r0:r1], o["d2sq"].astype(np.int64)), (k, i, j)
    return best


@pytest.mark.parametrize("ratio", [(4, 5), (1, 2)])
def test_exhaustive_nn_equals_brute_force(ratio):
    rng = np.random.default_rng(1)
    nd = np.array([0, 1, 2, 300, 257, 700, 513], dtype=np.int64)
    desc = rng.integers(0, 256, (int(nd.sum()), 128)).astype(np.uint8)
    off = np.concatenate([[0], np.cumsum(nd)])
    # shared rows with noise so that some queries pass the ratio test
    desc[off[5]:off[5] + 200] = np.clip(desc[off[3]:off[3] + 200].astype(int) + rng.integers(-6, 7, (200, 128)), 0, 255)
    pairs = [(3, 5), (5, 3), (4, 6), (6, 4), (3, 0), (3, 1), (3, 2), (0, 3), (1, 3), (2, 1), (5, 6)]
    best = _check(desc, nd, pairs, ratio)
    assert (best >= 0).sum() > 100


def test_duplicated_database_rows_tie_to_the_smaller_index():
    rng = np.random.default_rng(2)
    nd = np.array([200, 300], dtype=np.int64)
    desc = rng.integers(0, 256, (500, 128)).astype(np.uint8)
    desc[200 + 150:200 + 300] = desc[200:200 + 150]          # J holds every row twice
    desc[:100] = desc[200:300]                                # exact copies: d1 = d2 = 0, no match
    best = _check(desc, nd, [(0, 1)])
    assert (best[:100] == -1).all()


def test_extreme_magnitudes_stay_exact():
    # rows near the largest squared norm (128 * 255^2 < 2^23), all-255 and
    # all-zero rows: d^2 and the ratio test must still be exact
    rng = np.random.default_rng(3)
    nd = np.array([300, 400, 257], dtype=np.int64)
    desc = rng.integers(240, 256, (957, 128)).astype(np.uint8)
    desc[[0, 300, 700]] = 255
    desc[[1, 301, 956]] = 0
    desc[2, :64] = 255
    desc[2, 64:] = 0
    desc[302, 64:] = 255
    desc[302, :64] = 0
    desc[303] = 254
    desc[350:360] = np.clip(desc[10:20].astype(int) + 1, 0, 255)
    _check(desc, nd, [(0, 1), (1, 0), (2, 0), (1, 2)])
    _check(desc, nd, [(0, 1)], ratio=(1, 2))


def test_a_synthetic_pair_and_a_strip():
    wl = synth.pair2k(n=2000, shared=800)
    desc = wl.generate()
    best = _check(desc, wl.n_desc, [(0, 1), (1, 0)])
    assert (best[:2000] >= 0).sum() > 500
    wl = synth.strip30(n_images=4, n=1200)
    desc = wl.generate()
    _check(desc, wl.n_desc, [tuple(p) for p in wl.pairs])


def test_bad_arguments():
    d = torch.zeros((10, 128), dtype=torch.uint8, device="cuda")
    with pytest.raises(cm.CMError) as e:
        cm.nn_pairs(d, [5, 5], [(0, 2)])                      # image out of range
    assert e.value.status == cm.CM_ERR_INVALID
    with pytest.raises(cm.CMError) as e:
        cm.nn_pairs(d, [5, 5], [(0, 1)], ratio=(5, 4))        # ratio above 1
    assert e.value.status == cm.CM_ERR_INVALID
    best, _, _, rows = cm.nn_pairs(d, [5, 5], [])
    assert best.numel() == 0 and list(rows) == [0]
