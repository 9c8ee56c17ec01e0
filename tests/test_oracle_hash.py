"""Pins of the oracle's weight generator, centring and hashing (Sec. 2.3.1 steps (1)-(2)).

Each test checks the oracle against something other than itself: a published
test vector, a closed form of random-hyperplane LSH, a constructed special
case with a known answer, or a distribution law."""
import math

import numpy as np
import pytest
from scipy import stats

import oracle

P_DEFAULT = oracle.Params()


def test_splitmix64_published_vector():
    # First output of splitmix64 seeded with 0, as published with the generator
    # (Steele, Lea & Flood 2014; Vigna's reference C code).
    assert oracle.splitmix64_first(0) == 0xE220A8397B1DCDAF


def test_weights_are_standard_normal():
    W = oracle.weights(P_DEFAULT).astype(np.float64).ravel()
    assert W.shape == (128 * 176,)
    assert abs(W.mean()) < 4.0 / math.sqrt(W.size)
    assert abs(W.var() - 1.0) < 4.0 * math.sqrt(2.0 / W.size)
    assert stats.kstest(W, "norm").pvalue > 1e-3


def test_weights_box_muller_pairs_have_exponential_radius():
    # For a Box-Muller pair, (z0^2 + z1^2) / 2 = -ln(u1) is Exp(1) distributed,
    # and z0, z1 are uncorrelated.
    W = oracle.weights(oracle.Params(seed=7)).astype(np.float64).ravel()
    z0, z1 = W[0::2], W[1::2]
    r = (z0 * z0 + z1 * z1) / 2.0
    assert stats.kstest(r, "expon").pvalue > 1e-3
    assert abs(np.corrcoef(z0, z1)[0, 1]) < 4.0 / math.sqrt(z0.size)


def test_weights_depend_on_seed_and_are_deterministic():
    a = oracle.weights(oracle.Params(seed=1))
    b = oracle.weights(oracle.Params(seed=1))
    c = oracle.weights(oracle.Params(seed=2))
    assert np.array_equal(a, b) and not np.array_equal(a, c)


def test_bit_layout_with_selector_weights():
    # W[k][h] = 1 iff k == h mod 128 makes projection h equal to x~[h mod 128],
    # so key bit b of table t must be [x~[8t+b] > 0] and code bit b must be
    # [x~[(48+b) mod 128] > 0] (readings R1, R4).
    p = oracle.Params()
    W = np.zeros((128, p.P), dtype=np.float32)
    for h in range(p.P):
        W[h % 128, h] = 1.0
    rng = np.random.default_rng(0)
    xc = rng.standard_normal((64, 128))
    keys, code, marg = oracle.hash_centred(xc, W, p)
    for i in range(64):
        for t in range(p.L):
            want = sum(1 << b for b in range(p.m) if xc[i, p.m * t + b] > 0)
            assert keys[i, t] == want
        for b in range(p.nbits):
            bit = (int(code[i, b // 32]) >> (b % 32)) & 1
            assert bit == int(xc[i, (p.L * p.m + b) % 128] > 0)


def test_zero_vector_gives_zero_bits_and_marginal_flags():
    # A descriptor equal to the mean has x~ = 0: every projection is exactly 0,
    # so every bit is 0 under the strict rule (R4); with ||x~|| = 0 the strict
    # marginal test |s| < 1e-4 ||x~|| (R9) flags nothing.
    p = P_DEFAULT
    base = np.random.default_rng(1).integers(20, 200, size=128)
    delta = np.random.default_rng(2).integers(0, 20, size=128)
    desc = np.stack([base - delta, base, base + delta]).astype(np.uint8)   # mean == base exactly
    sums = oracle.col_sums(desc)
    assert np.array_equal(sums, 3 * base.astype(np.uint64))
    mu = oracle.mean_from_sums(sums, 3)
    keys, code, marg = oracle.hash_desc(desc, mu, oracle.weights(p), p)
    assert np.all(keys[1] == 0) and np.all(code[1] == 0) and np.all(marg[1] == 0)
    # rows 0 and 2 are reflections through the mean: complementary codes
    ok = marg[0] == 0
    bits0 = np.unpackbits(code[0].view(np.uint8), bitorder="little")
    bits2 = np.unpackbits(code[2].view(np.uint8), bitorder="little")
    fine_ok = ok[p.L * p.m:]
    assert np.all(bits0[fine_ok] != bits2[fine_ok])


def test_reflection_complements_every_bit():
    p = P_DEFAULT
    W = oracle.weights(p)
    xc = np.random.default_rng(3).standard_normal((200, 128))
    k1, c1, m1 = oracle.hash_centred(xc, W, p)
    k2, c2, m2 = oracle.hash_centred(-xc, W, p)
    # s -> -s flips every bit whose projection is not exactly 0; with Gaussian
    # vectors no projection is exactly 0.  The marginal share is ~2*phi(0)*1e-4.
    assert np.array_equal(m1, m2) and m1.mean() < 5e-4
    assert np.all(c1 ^ c2 == 0xFFFFFFFF)
    assert np.all(k1 ^ k2 == 0xFF)


@pytest.mark.parametrize("theta", [math.pi / 8, math.pi / 4, math.pi / 2, 3 * math.pi / 4])
def test_hamming_closed_form_theta_over_pi(theta):
    # Random hyperplanes: Pr[a code bit differs] = theta / pi, and the L
    # coarse keys of two vectors agree with probability (1 - theta/pi)^m.
    p = oracle.Params(seed=11)
    W = oracle.weights(p)
    rng = np.random.default_rng(int(theta * 1000))
    n = 3000
    x = rng.standard_normal((n, 128))
    x /= np.linalg.norm(x, axis=1, keepdims=True)
    r = rng.standard_normal((n, 128))
    r -= (r * x).sum(1, keepdims=True) * x
    r /= np.linalg.norm(r, axis=1, keepdims=True)
    y = math.cos(theta) * x + math.sin(theta) * r
    kx, cx, _ = oracle.hash_centred(x, W, p, marginal=False)
    ky, cy, _ = oracle.hash_centred(y, W, p, marginal=False)
    h = np.unpackbits((cx ^ cy).view(np.uint8), axis=1).sum(1)
    frac = h.mean() / p.nbits
    assert abs(frac - theta / math.pi) < 0.01
    agree = (kx == ky).mean()
    assert abs(agree - (1 - theta / math.pi) ** p.m) < 0.02


def test_hash_of_raw_descriptor_equals_hash_of_centred_vector():
    p = P_DEFAULT
    W = oracle.weights(p)
    desc = np.random.default_rng(4).integers(0, 256, size=(50, 128)).astype(np.uint8)
    sums = oracle.col_sums(desc)
    assert np.array_equal(sums, desc.astype(np.uint64).sum(0))
    mu = oracle.mean_from_sums(sums, 50)
    k1, c1, m1 = oracle.hash_desc(desc, mu, W, p)
    k2, c2, m2 = oracle.hash_centred(desc.astype(np.float64) - mu, W, p)
    assert np.array_equal(k1, k2) and np.array_equal(c1, c2) and np.array_equal(m1, m2)
