"""Pins of the oracle's buckets, candidate ranking, rerank and ratio test
(Sec. 2.3.1 steps (1)-(4)) against brute force and invariants."""
import numpy as np
import pytest

import oracle
import synth


def _bits(code):
    return np.unpackbits(np.ascontiguousarray(code).view(np.uint8), axis=-1, bitorder="little")


def _dist2(a, b):
    a = a.astype(np.int64)
    b = b.astype(np.int64)
    return (a * a).sum(1)[:, None] + (b * b).sum(1)[None, :] - 2 * a @ b.T


@pytest.fixture(scope="module")
def small_pair():
    w = synth.pair2k(n=400, shared=160)
    d = w.generate()
    p = oracle.Params()
    idx = oracle.Index(d, w.n_desc, p, threads=2)
    return idx, idx.image(0), idx.image(1), p


def test_buckets_partition_and_order(small_pair):
    _, I, _, p = small_pair
    B = 1 << p.m
    for t in range(p.L):
        off, ids = I.off[t], I.idx[t]
        assert off[0] == 0 and off[-1] == I.n and np.all(np.diff(off) >= 0)
        assert np.array_equal(np.sort(ids), np.arange(I.n))
        for b in range(B):
            run = ids[off[b]:off[b + 1]]
            assert np.all(I.keys[run, t] == b)
            assert np.all(np.diff(run) > 0)          # ascending index inside a bucket


def test_candidates_and_topk_equal_brute_force(small_pair):
    # Brute force: C(q) = every database point sharing at least one of the L
    # keys with q (set semantics), ranked by (Hamming, index), first K kept.
    _, I, J, p = small_pair
    r = oracle.match_pair(I, J, p, topk=True)
    bi, bj = _bits(I.code), _bits(J.code)
    for q in range(I.n):
        share = (J.keys == I.keys[q][None, :]).any(1)
        C = np.nonzero(share)[0]
        assert r["ncand"][q] == len(C)
        h = (bj[C] != bi[q][None, :]).sum(1)
        order = np.lexsort((C, h))
        want = list(C[order][:p.K]) + [-1] * max(0, p.K - len(C))
        assert list(r["topk"][q]) == want


def test_one_bucket_all_candidates_is_exhaustive_nn():
    # With m = 0 every point shares the single bucket and with K = N_J every
    # candidate is reranked, so the cascade is exhaustive L2 NN + ratio test.
    w = synth.pair2k(n=64, shared=20)
    d = w.generate()
    p = oracle.Params(m=0, K=64)
    idx = oracle.Index(d, w.n_desc, p, threads=1)
    I, J = idx.image(0), idx.image(1)
    r = oracle.match_pair(I, J, p)
    bf = oracle.brute_nn(I.desc, J.desc, p.ratio_num, p.ratio_den)
    # independent numpy brute force with (d^2, index) ordering
    D2 = _dist2(I.desc, J.desc)
    order = np.lexsort((np.broadcast_to(np.arange(J.n), D2.shape), D2), axis=1)
    d1 = D2[np.arange(I.n), order[:, 0]]
    d2 = D2[np.arange(I.n), order[:, 1]]
    want = np.where(25 * d1 < 16 * d2, order[:, 0], -1)
    for res in (r, bf):
        assert np.array_equal(res["best_j"], want)
        assert np.array_equal(res["d1sq"].astype(np.int64), d1)
        assert np.array_equal(res["d2sq"].astype(np.int64), d2)


def test_distances_are_exact_integers(small_pair):
    _, I, J, p = small_pair
    r = oracle.match_pair(I, J, p, topk=True)
    D2 = _dist2(I.desc, J.desc)
    for q in range(I.n):
        kept = [j for j in r["topk"][q] if j >= 0]
        if len(kept) >= 1:
            ds = sorted((D2[q, j], j) for j in kept)
            assert r["d1sq"][q] == ds[0][0]
            if len(kept) >= 2:
                assert r["d2sq"][q] == ds[1][0]
                passes = 25 * ds[0][0] < 16 * ds[1][0]
                assert (r["best_j"][q] == ds[0][1]) == passes
            else:
                assert r["d2sq"][q] == 0xFFFFFFFF and r["best_j"][q] == -1
        else:
            assert r["best_j"][q] == -1 and r["d1sq"][q] == 0xFFFFFFFF


def test_ratio_test_monotone_in_threshold(small_pair):
    idx, I, J, _ = small_pair
    prev = None
    for num in range(0, 11):
        p = oracle.Params(ratio_num=num, ratio_den=10)
        r = oracle.match_pair(I, J, p)
        m = set(np.nonzero(r["best_j"] >= 0)[0])
        if num == 0:
            assert not m
        if prev is not None:
            assert prev <= m
        prev = m
    # t_r = 1 keeps exactly the queries whose nearest is strictly closer than the second
    p = oracle.Params(ratio_num=1, ratio_den=1)
    r = oracle.match_pair(I, J, p)
    strict = (r["d1sq"] < r["d2sq"]) & (r["d2sq"] != 0xFFFFFFFF)
    assert np.array_equal(r["best_j"] >= 0, strict)


def test_exact_planted_copies_always_match():
    # Noise-free copies have Hamming 0 and identical keys, so they are always
    # candidates, always ranked first and pass the ratio test (d1 = 0 < t_r d2).
    rng = np.random.default_rng(5)
    w = synth.pair2k(n=300, shared=0)
    A = w.generate()[:300]
    B = w.generate()[300:].copy()
    src = rng.choice(300, 120, replace=False)
    slots = rng.choice(300, 120, replace=False)
    B[slots] = A[src]
    assert len(np.unique(np.concatenate([A, B]), axis=0)) == 600 - 120
    p = oracle.Params()
    idx = oracle.Index(np.concatenate([B, A]), [300, 300], p, threads=1)
    r = oracle.match_pair(idx.image(0), idx.image(1), p)
    assert np.array_equal(r["best_j"][slots], src)
    assert np.all(r["d1sq"][slots] == 0)


def test_fewer_than_two_candidates_never_match():
    # A query alone in its buckets has |C| < 2: no ratio test, no match.
    w = synth.pair2k(n=200, shared=0)
    d = w.generate()
    p = oracle.Params(L=1, m=8)
    idx = oracle.Index(d, w.n_desc, p, threads=1)
    r = oracle.match_pair(idx.image(0), idx.image(1), p)
    few = r["ncand"] < 2
    assert few.any()
    assert np.all(r["best_j"][few] == -1)
    assert np.all(r["d2sq"][few] == 0xFFFFFFFF)
