"""GPU parity of VLAD encoding (cm_vlad_encode, Sec. 2.1) with the oracle:
codeword assignments bit for bit (exact integer distances on the tensor
cores, ties to the smaller codeword), the normalised vectors to FP32
rounding; codebook sizes 1..256 including ones that are not multiples of 16,
duplicate codewords (exact ties), empty images, ragged last tiles, and a
large case checked on sampled rows."""
import numpy as np
import pytest

import paper_2505_22089_b300 as cm
import synth
from oracle import vlad as ovlad

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ATOL = 2e-6   # components of a unit vector: FP32 square roots and scaling against FP64


def _codebook(desc, C, seed):
    rng = np.random.default_rng(seed)
    return desc[rng.choice(len(desc), C, replace=False)].copy()


def _run(desc, nd, cb):
    v, a = cm.vlad_encode(torch.from_numpy(desc).cuda(), nd, torch.from_numpy(cb).cuda(), want_assign=True)
    torch.cuda.synchronize()
    return v.cpu().numpy(), a.cpu().numpy()


@pytest.mark.parametrize("C", [1, 16, 40, 64, 128, 200, 256])
def test_vlad_equals_the_oracle(C):
    wl = synth.strip30(n_images=5, n=1500)
    desc = wl.generate()
    nd = wl.n_desc.copy()
    nd[2] = 0                      # an empty image (its rows move to the next one)
    nd[3] += wl.n_desc[2]
    cb = _codebook(desc, C, C)
    v, a = _run(desc, nd, cb)
    want, wa = ovlad.encode(desc, nd, cb)
    assert np.array_equal(a, wa)
    assert np.abs(v - want).max() <= ATOL
    assert (v[2] == 0).all()


def test_duplicate_codewords_and_ragged_tiles():
    rng = np.random.default_rng(3)
    desc = rng.integers(0, 256, (1000 + 77, 128)).astype(np.uint8)
    cb = _codebook(desc, 48, 4)
    cb[30] = cb[7]                 # exact ties: the smaller index wins
    cb[47] = cb[0]
    desc[:50] = cb[7]              # rows sitting on the duplicated codeword
    nd = [129, 1, 0, 947]
    v, a = _run(desc, nd, cb)
    want, wa = ovlad.encode(desc, nd, cb)
    assert np.array_equal(a, wa)
    assert (a[:50] == 7).all() and not (a == 30).any() and not (a == 47).any()
    assert np.abs(v - want).max() <= ATOL


def test_large_case_on_sampled_rows():
    wl = synth.scaled("grid500", gx=5, gy=4, nmin=8000, nmax=20000)
    desc = wl.generate()
    cb = _codebook(desc, 256, 9)
    v, a = _run(desc, wl.n_desc, cb)
    rng = np.random.default_rng(10)
    rows = rng.choice(len(desc), 20000, replace=False)
    assert np.array_equal(a[rows], ovlad.assign(desc[rows], cb))
    # two whole images against the oracle, and unit norm for all
    off = wl.row_off
    for i in (0, wl.n_images - 1):
        want, _ = ovlad.encode(desc[off[i]:off[i + 1]], [wl.n_desc[i]], cb)
        assert np.abs(v[i] - want[0]).max() <= ATOL
    assert np.allclose(np.linalg.norm(v, axis=1), 1.0, atol=1e-5)


def test_bad_arguments():
    d = torch.zeros((10, 128), dtype=torch.uint8, device="cuda")
    for C in (0, 257):
        cb = torch.zeros((max(C, 1), 128), dtype=torch.uint8, device="cuda")
        with pytest.raises(cm.CMError) as e:
            cm.check(cm.lib().cm_vlad_encode(cm._ptr(d), np.array([0, 10], np.int64).ctypes.data, 1, cm._ptr(cb), C,
                                             cm._ptr(d), 1 << 20, None, cm._ptr(d), cm._stream(None)))
        assert e.value.status == cm.CM_ERR_INVALID
    cb = torch.zeros((4, 128), dtype=torch.uint8, device="cuda")
    w = torch.empty(1024, dtype=torch.uint8, device="cuda")
    out = torch.empty((1, 512), dtype=torch.float32, device="cuda")
    with pytest.raises(cm.CMError) as e:   # workspace too small
        cm.check(cm.lib().cm_vlad_encode(cm._ptr(d), np.array([0, 10], np.int64).ctypes.data, 1, cm._ptr(cb), 4,
                                         cm._ptr(w), 16, None, cm._ptr(out), cm._stream(None)))
    assert e.value.status == cm.CM_ERR_BUDGET
    with pytest.raises(cm.CMError) as e:   # offsets must start at 0
        cm.check(cm.lib().cm_vlad_encode(cm._ptr(d), np.array([1, 10], np.int64).ctypes.data, 1, cm._ptr(cb), 4,
                                         cm._ptr(w), 1024, None, cm._ptr(out), cm._stream(None)))
    assert e.value.status == cm.CM_ERR_INVALID
