"""The library's SAO local constraint (cm_sao_filter, C++ on the host) against
the oracle, score for score and decision for decision: random sub-pixel
keypoints, sixteenth-pixel lattices with many distance and direction ties,
many-to-one matches, clustered and collinear layouts, every neighbour count
from 1 to 32 and the degenerate sizes 0..3.  Then the chain SAO -> RANSAC of
the ready-made verifier on planted outliers."""
import numpy as np
import pytest

import paper_2505_22089_b300 as cm
from oracle import sao


def _ids(n):
    return (np.arange(n, dtype=np.uint32) << 16) | np.arange(n, dtype=np.uint32)


def _check(ki, kj, mt, k, tau=0.875):
    s_o, keep_o = sao.sao_filter(ki, kj, mt, k, tau)
    s_c, keep_c, n = cm.sao_filter(ki, kj, mt, k, tau)
    assert s_c.dtype == np.float32 and s_c.shape == s_o.shape
    bad = np.nonzero(s_c != s_o)[0]
    assert bad.size == 0, (k, bad[:10], s_c[bad[:10]], s_o[bad[:10]])
    assert np.array_equal(keep_c, keep_o)
    assert n == int(keep_o.sum())
    return s_c


def _planted(rng, n, share, noise=1.0, quant=None):
    A = np.array([[0.93, -0.21, 140.0], [0.24, 0.97, -60.0]])
    ki = rng.uniform(0, 4000, (n, 2))
    kj = ki @ A[:, :2].T + A[:, 2] + rng.normal(0, noise, (n, 2))
    out = rng.random(n) < share
    kj[out] = rng.uniform(0, 4000, (int(out.sum()), 2))
    if quant:
        ki, kj = np.round(ki * quant) / quant, np.round(kj * quant) / quant
    return ki.astype(np.float32), kj.astype(np.float32), out


@pytest.mark.parametrize("k", [1, 2, 4, 8, 16, 32])
def test_random_keypoints(k):
    rng = np.random.default_rng(100 + k)
    n = 700 if k <= 8 else 40 if k == 32 else 160     # the oracle's rotation search grows as k^4
    ki, kj, _ = _planted(rng, n, 0.4)
    _check(ki, kj, _ids(n), k)


def test_lattice_ties():
    """Integer and sixteenth-pixel lattices: many equal distances (ties by
    index) and neighbours on one ray from the centre (ties by index)."""
    rng = np.random.default_rng(5)
    g = np.stack(np.meshgrid(np.arange(20), np.arange(15)), -1).reshape(-1, 2).astype(np.float32) * 8
    perm = rng.permutation(len(g))
    ki = g[perm]
    kj = np.stack([-g[:, 1], g[:, 0]], 1)[perm] * 2 + 64      # exact rotation by 90 and scale 2
    for k in (4, 8, 12):
        s = _check(ki, kj, _ids(len(g)), k)
        assert (s == 0).all()
    kj2 = kj.copy()
    kj2[rng.choice(len(g), 60, replace=False)] = rng.integers(0, 64, (60, 2)) * 4.0
    for k in (6, 8):
        _check(ki, kj2, _ids(len(g)), k)
    ki3, kj3, _ = _planted(rng, 900, 0.3, quant=16)
    _check(ki3, kj3, _ids(900), 8)


def test_many_to_one_and_duplicates():
    rng = np.random.default_rng(6)
    ni, nj = 400, 150
    ki = rng.uniform(0, 1000, (ni, 2)).astype(np.float32)
    kj = rng.uniform(0, 1000, (nj, 2)).astype(np.float32)
    ki[50:60] = ki[40]                                     # coincident query keypoints
    q = np.sort(rng.choice(ni, 300, replace=False)).astype(np.uint32)
    j = rng.integers(0, nj, 300).astype(np.uint32)          # many queries share a database keypoint
    mt = (q << 16) | j
    for k in (3, 8):
        _check(ki, kj, mt, k)


def test_layouts():
    rng = np.random.default_rng(7)
    # clustered: a few tight clusters far apart (most grid cells empty)
    c = rng.uniform(0, 5000, (6, 2))
    ki = (c[rng.integers(0, 6, 500)] + rng.normal(0, 3, (500, 2))).astype(np.float32)
    kj = (ki * 1.1 + rng.normal(0, 0.5, (500, 2))).astype(np.float32)
    _check(ki, kj, _ids(500), 8)
    # collinear query keypoints (zero-height bounding box), a thin strip on the other side
    t = np.sort(rng.uniform(0, 3000, 300)).astype(np.float32)
    ki = np.stack([t, np.full(300, 7.0, np.float32)], 1)
    kj = np.stack([t * 0.5, rng.uniform(0, 1e-3, 300)], 1).astype(np.float32)
    _check(ki, kj, _ids(300), 8)
    # a dense cluster plus a few far points: the far points search many rings
    ki = np.concatenate([rng.normal(2000, 5, (590, 2)), rng.uniform(0, 4000, (10, 2))]).astype(np.float32)
    kj = np.concatenate([rng.normal(900, 8, (590, 2)), rng.uniform(0, 4000, (10, 2))]).astype(np.float32)
    _check(ki, kj, _ids(600), 8)
    # every keypoint the same point
    z = np.full((40, 2), 3.5, np.float32)
    s = _check(z, z, _ids(40), 8)
    assert (s == 0).all()
    # large coordinates and a wide aspect ratio
    ki = np.stack([rng.uniform(0, 1e6, 300), rng.uniform(0, 10, 300)], 1).astype(np.float32)
    kj = (ki + 5).astype(np.float32)
    _check(ki, kj, _ids(300), 8)


def test_degenerate_sizes_and_thresholds():
    rng = np.random.default_rng(8)
    for n in (0, 1, 2, 3, 4, 9):
        ki = rng.uniform(0, 100, (max(n, 1), 2)).astype(np.float32)
        kj = rng.uniform(0, 100, (max(n, 1), 2)).astype(np.float32)
        _check(ki, kj, _ids(n), 8)
    ki, kj, _ = _planted(rng, 300, 0.5)
    for tau in (0.0, 0.25, 0.5, 0.875, 1.0):
        _check(ki, kj, _ids(300), 8, tau)


def test_bad_arguments():
    z = np.zeros((4, 2), np.float32)
    for k, tau in ((0, 0.5), (33, 0.5), (8, -0.1), (8, float("nan"))):
        with pytest.raises(cm.CMError) as e:
            cm.sao_filter(z, z, _ids(4), k, tau)
        assert e.value.status == cm.CM_ERR_INVALID


def test_filter_removes_planted_outliers_before_ransac():
    """Local constraint then RANSAC, as the verifier chains them: most random
    outliers go and almost every inlier stays, so that on the kept matches
    (inlier share ~0.85 instead of 0.4) 20 RANSAC samples find the model
    (failure probability ~(1 - 0.85^3)^20 < 1e-8)."""
    rng = np.random.default_rng(9)
    ki, kj, out = _planted(rng, 2000, 0.6)
    _, keep, n = cm.sao_filter(ki, kj, _ids(2000), 8, 0.875)
    assert keep[out].mean() < 0.15            # outliers dropped
    assert keep[~out].mean() > 0.9            # inliers kept
    kept = _ids(2000)[keep]
    share = (~out & keep).sum() / keep.sum()
    assert share > 0.8
    _, mask_k, n_k = cm.verify_affine(ki, kj, kept, thresh_px=4.0, max_iters=20, seed=3)
    assert n_k >= int((~out & keep).sum()) - 5
    assert not (mask_k & out[keep]).any() or (mask_k & out[keep]).sum() <= 2
