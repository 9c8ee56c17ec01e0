"""Pins of the VLAD oracle (Sec. 2.1) against facts that do not come from its
code: nearest codewords from scipy's distance matrix, closed forms for one
descriptor and for descriptors sitting on codewords, the additivity of raw
residuals over a split image, invariance to descriptor order, unit norm."""
import numpy as np
import pytest

from oracle import vlad

cdist = pytest.importorskip("scipy.spatial.distance").cdist


def _data(seed, n, C):
    rng = np.random.default_rng(seed)
    X = rng.integers(0, 256, (n, 128)).astype(np.uint8)
    Cb = rng.integers(0, 256, (C, 128)).astype(np.uint8)
    return rng, X, Cb


def test_assignment_equals_the_distance_matrix_argmin():
    _, X, Cb = _data(1, 900, 64)
    d = cdist(X.astype(np.float64), Cb.astype(np.float64), "sqeuclidean")
    assert np.array_equal(vlad.assign(X, Cb), np.argmin(d, axis=1))


def test_assignment_ties_go_to_the_smaller_codeword():
    Cb = np.zeros((4, 128), np.uint8)
    Cb[1, 0] = 2          # codewords 1 and 3 are both at distance 1 from x
    Cb[3, 1] = 2
    Cb[0, :] = 200        # far
    Cb[2, :] = 100        # far
    x = np.zeros((1, 128), np.uint8)
    x[0, 0] = 1
    x[0, 1] = 1
    assert vlad.assign(x, Cb)[0] == 1


def test_single_descriptor_closed_form():
    rng, X, Cb = _data(2, 1, 16)
    c = int(np.argmin(((X[0].astype(np.int64) - Cb.astype(np.int64)) ** 2).sum(1)))
    r = X[0].astype(np.float64) - Cb[c]
    s = np.sign(r) * np.sqrt(np.abs(r))
    want = np.zeros((16, 128))
    want[c] = s / np.linalg.norm(s)
    out, a = vlad.encode(X, [1], Cb)
    assert a[0] == c
    assert np.allclose(out[0], want.reshape(-1), rtol=0, atol=1e-15)


def test_descriptors_on_codewords_give_zero():
    _, _, Cb = _data(3, 1, 32)
    X = Cb[[0, 5, 5, 31]]
    out, a = vlad.encode(X, [4], Cb)
    assert list(a) == [0, 5, 5, 31]
    assert (out == 0).all()


def test_raw_residuals_add_over_a_split_and_ignore_order():
    rng, X, Cb = _data(4, 500, 32)
    whole = vlad.raw_vlad(X, Cb)
    assert np.array_equal(whole, vlad.raw_vlad(X[:200], Cb) + vlad.raw_vlad(X[200:], Cb))
    perm = rng.permutation(500)
    assert np.array_equal(whole, vlad.raw_vlad(X[perm], Cb))
    # per codeword: sum of members minus count times the codeword
    a = vlad.assign(X, Cb)
    c = int(np.bincount(a).argmax())
    assert np.array_equal(whole[c], X[a == c].astype(np.int64).sum(0) - (a == c).sum() * Cb[c].astype(np.int64))


def test_encoding_is_unit_norm_per_image_and_images_are_independent():
    _, X, Cb = _data(5, 700, 64)
    nd = [300, 0, 400]
    out, a = vlad.encode(X, nd, Cb)
    assert np.isclose(np.linalg.norm(out[0]), 1.0) and np.isclose(np.linalg.norm(out[2]), 1.0)
    assert (out[1] == 0).all()                                     # an empty image
    alone, _ = vlad.encode(X[300:], [400], Cb)
    assert np.array_equal(out[2], alone[0])
