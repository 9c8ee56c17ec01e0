"""Host-side geometric verification (cm_verify_affine, the RANSAC global
constraint of Sec. 2.3.2), pinned against planted affine maps: exact data must
give the exact map and every match as an inlier; planted outliers displaced far
beyond the threshold must be rejected exactly; degenerate inputs give no model."""
import numpy as np
import pytest

import paper_2505_22089_b300 as cm
import synth


def _ids(n):
    return (np.arange(n, dtype=np.uint32) << 16) | np.arange(n, dtype=np.uint32)


def _planted(seed, n, A, outlier_share, noise=0.5, far=40.0):
    rng = np.random.Generator(np.random.PCG64(seed))
    ki = rng.uniform(0, 4000, (n, 2))
    kj = ki @ A[:, :2].T + A[:, 2] + rng.normal(0, noise, (n, 2))
    out = rng.random(n) < outlier_share
    # outliers: displaced by at least `far` pixels from where the map puts them
    ang = rng.uniform(0, 2 * np.pi, out.sum())
    rad = far + rng.uniform(0, 500, out.sum())
    kj[out] = ki[out] @ A[:, :2].T + A[:, 2] + np.stack([rad * np.cos(ang), rad * np.sin(ang)], 1)
    return ki.astype(np.float32), kj.astype(np.float32), out


def test_exact_affine_is_recovered_with_all_inliers():
    A = np.array([[0.8, -0.35, 120.0], [0.3, 0.95, -40.0]])
    ki, kj, _ = _planted(1, 300, A, 0.0, noise=0.0)
    Af, mask, n = cm.verify_affine(ki, kj, _ids(300), thresh_px=1.0)
    assert n == 300 and mask.all()
    assert np.allclose(Af, A, atol=1e-3)


@pytest.mark.parametrize("share", [0.2, 0.5, 0.8])
def test_planted_outliers_are_rejected_exactly(share):
    A = np.array([[1.1, 0.2, -300.0], [-0.15, 0.9, 75.0]])
    ki, kj, out = _planted(2, 1000, A, share)
    Af, mask, n = cm.verify_affine(ki, kj, _ids(1000), thresh_px=3.0, max_iters=5000, seed=3)
    # inliers carry 0.5 px noise (residual > 3 px has probability ~1e-8), outliers sit >= 40 px away
    assert np.array_equal(mask, ~out)
    assert n == int((~out).sum())
    assert np.allclose(Af[:, :2], A[:, :2], atol=2e-3)
    assert np.allclose(Af[:, 2], A[:, 2], atol=2.0)


def test_degenerate_inputs():
    ki = np.zeros((4, 2), np.float32)
    kj = np.zeros((4, 2), np.float32)
    # fewer than three matches: no model
    _, mask, n = cm.verify_affine(ki, kj, _ids(2))
    assert n == 0 and not mask.any()
    # collinear query keypoints: every minimal sample is singular
    t = np.linspace(0, 100, 50, dtype=np.float32)
    ki = np.stack([t, 2 * t + 1], 1)
    _, mask, n = cm.verify_affine(ki, ki.copy(), _ids(50))
    assert n == 0 and not mask.any()
    # no matches at all
    _, mask, n = cm.verify_affine(ki, ki, np.zeros(0, np.uint32))
    assert n == 0 and mask.size == 0


def test_seeded_and_deterministic():
    A = np.array([[0.9, 0.1, 10.0], [-0.1, 0.9, 20.0]])
    ki, kj, _ = _planted(4, 400, A, 0.6)
    r1 = cm.verify_affine(ki, kj, _ids(400), seed=11)
    r2 = cm.verify_affine(ki, kj, _ids(400), seed=11)
    assert np.array_equal(r1[0], r2[0]) and np.array_equal(r1[1], r2[1]) and r1[2] == r2[2]


def test_bad_arguments():
    ki = np.zeros((4, 2), np.float32)
    with pytest.raises(cm.CMError) as e:
        cm.verify_affine(ki, ki, _ids(4), thresh_px=0.0)
    assert e.value.status == cm.CM_ERR_INVALID
    with pytest.raises(cm.CMError):
        cm.verify_affine(ki, ki, _ids(4), max_iters=0)


def test_synthetic_views_share_an_affine_map():
    # The generator's keypoints are affine images of planar world points, so
    # the descriptors of shared tracks are exact correspondences (+0.5 px noise).
    wl = synth.scaled("grid500", gx=3, gy=3, nmin=1500, nmax=1500)
    desc, kp, track = wl.generate(want_kp=True, want_track=True)
    off = wl.row_off
    i, j = int(wl.pairs[0][0]), int(wl.pairs[0][1])
    ti, tj = track[off[i]:off[i + 1]], track[off[j]:off[j + 1]]
    common, qi, qj = np.intersect1d(ti, tj, return_indices=True)
    common_ok = common >= 0
    qi, qj = qi[common_ok], qj[common_ok]
    assert len(qi) > 50
    m = (qi.astype(np.uint32) << 16) | qj.astype(np.uint32)
    _, mask, n = cm.verify_affine(kp[off[i]:off[i + 1]], kp[off[j]:off[j + 1]], m, thresh_px=3.0)
    # both keypoints carry 0.5 px noise: a residual beyond 3 px has probability ~exp(-9)
    assert n >= len(qi) - 3
