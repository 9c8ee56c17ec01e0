"""Host-side checks of the C-ABI library (no GPU needed): it loads, exports
every declared symbol, validates arguments, and its host-only calls (weights,
GPS, schedule blocks) agree exactly with the oracle."""
import os
import re

import numpy as np
import pytest

import oracle
from oracle import gps as ogps
import paper_2505_22089_b300 as cm
import synth

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "cashmatch.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cm_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    lib = cm.lib()
    names = declared_functions()
    assert len(names) >= 25
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(cm.EXPORTS) == names
    assert "sm_103a" in cm.version()


def test_params_validation():
    lib = cm.lib()
    p = cm.Params()
    assert lib.cm_params_default(p) == cm.CM_OK
    assert (p.L, p.m, p.n_bits, p.K, p.ratio_num, p.ratio_den) == (6, 8, 128, 8, 4, 5)
    for bad in (dict(L=0), dict(L=9), dict(m=9), dict(K=3), dict(K=32), dict(ratio=(1, 0)), dict(ratio=(-1, 2)),
                dict(query_tile=100), dict(query_tile=32), dict(query_tile=8192, algo="tile"), dict(algo=5), dict(n_bits=64), dict(rerank=7)):
        q = cm.Params.make(**bad)
        assert lib.cm_params_check(q) == cm.CM_ERR_INVALID
        assert lib.cm_last_error()


@pytest.mark.parametrize("kw", [dict(), dict(seed=1), dict(L=1, m=0), dict(L=8, m=8), dict(L=3, m=5)])
def test_weights_bitwise_equal_oracle(kw):
    p = cm.Params.make(**kw)
    op = oracle.Params(L=p.L, m=p.m, seed=p.seed)
    W = cm.make_weights(p)
    Wo = oracle.weights(op)
    assert W.shape == Wo.shape == (128, p.P)
    assert np.array_equal(W.view(np.uint32), Wo.view(np.uint32))


def test_gps_matches_oracle_on_synthetic_graphs():
    # Image ids are shuffled as a retrieval front end would leave them; GPS must
    # bring the band back close to the layout's natural order.
    import random
    for wl in (synth.strip30(), synth.grid500(gx=10, gy=8), synth.oblique200()):
        n = wl.n_images
        ids = list(range(n))
        random.Random(n).shuffle(ids)
        natural = [tuple(e) for e in wl.pairs.tolist()]
        edges = [(ids[a], ids[b]) for a, b in natural]
        a = cm.gps_order(n, edges)
        b = ogps.gps_order(n, edges)
        assert a == b
        bw = ogps.bandwidth(a, edges)
        assert bw <= 0.5 * ogps.bandwidth(list(range(n)), edges)
        assert bw <= 1.5 * ogps.bandwidth(list(range(n)), natural)


@pytest.mark.parametrize("budget_imgs,blk", [(10 ** 4, 400), (60, 20), (14, 5), (5, 2), (2, 1)])
def test_schedule_matches_oracle(budget_imgs, blk):
    wl = synth.grid500(gx=12, gy=9, nmin=500, nmax=3000)
    p = cm.Params.make()
    nb = [cm.image_bytes(p, n) for n in wl.n_desc]
    budget = int(budget_imgs * max(nb))
    got = cm.schedule_blocks(wl.pairs, wl.n_desc, p, budget, blk)
    want = ogps.schedule([tuple(x) for x in wl.pairs.tolist()], nb, budget, blk)
    assert got.rows == want
    assert got.iterations == (max(r["iteration"] for r in want) + 1 if want else 0)


def test_schedule_errors():
    p = cm.Params.make()
    nb = cm.image_bytes(p, 1000)
    with pytest.raises(cm.CMError) as e:
        cm.schedule_blocks([(0, 0)], [1000, 1000], p, 10 * nb, 4)
    assert e.value.status == cm.CM_ERR_INVALID
    with pytest.raises(cm.CMError) as e:
        cm.schedule_blocks([(0, 5)], [1000, 1000], p, 10 * nb, 4)
    assert e.value.status == cm.CM_ERR_INVALID
    with pytest.raises(cm.CMError) as e:
        cm.schedule_blocks([(0, 1)], [1000, 1000], p, nb, 4)
    assert e.value.status == cm.CM_ERR_BUDGET
    with pytest.raises(cm.CMError) as e:
        cm.image_bytes(p, 70000)
    assert e.value.status == cm.CM_ERR_INVALID


def test_image_bytes_layout():
    p = cm.Params.make()
    b0 = cm.image_bytes(p, 0)
    b = cm.image_bytes(p, 20000)
    # 128 desc + 8 key + 16 code + 6*16 sorted codes + 6*2 indices + 4 norm bytes per descriptor
    assert b - b0 >= 264 * 20000
    assert b - b0 < 264 * 20000 + 4096
    assert cm.image_bytes(cm.Params.make(rerank="int"), 20000) == b


def test_host_argument_checks_of_the_later_entry_points():
    lib = cm.lib()
    # rejected before any device work, so these run without a GPU
    assert lib.cm_selftest_wait(0, None) == cm.CM_ERR_INVALID
    assert lib.cm_selftest_wait((1 << 24) + 1, None) == cm.CM_ERR_INVALID
    off = np.array([1, 5], dtype=np.int64)
    assert lib.cm_vlad_encode(None, off.ctypes.data, 1, None, 4, None, 0, None, None, None) == cm.CM_ERR_INVALID
    assert lib.cm_nn_pairs(None, off.ctypes.data, 1, None, 0, 5, 4, None, 0, None, None, None, None) == cm.CM_ERR_INVALID
    b = cm.ctypes.c_uint64()
    assert lib.cm_vlad_workspace_bytes(3, 100, cm.ctypes.byref(b)) == cm.CM_OK and b.value % 256 == 0
    off3 = np.array([0, 300, 700, 700], dtype=np.int64)
    pr3 = np.array([[0, 1], [1, 0], [2, 0]], dtype=np.int32)   # database images 1 (400 rows) and 0 (300 rows)
    assert lib.cm_nn_workspace_bytes(off3.ctypes.data, 3, pr3.ctypes.data, 3, cm.ctypes.byref(b)) == cm.CM_OK
    assert b.value % 256 == 0 and b.value >= 4 * 256 * 144 * 2   # two 256-row tiles (K = 144) per database image
    assert lib.cm_nn_workspace_bytes(off3.ctypes.data, 3, pr3.ctypes.data, -1, cm.ctypes.byref(b)) == cm.CM_ERR_INVALID
    bad = np.array([[0, 5]], dtype=np.int32)
    assert lib.cm_nn_workspace_bytes(off3.ctypes.data, 3, bad.ctypes.data, 1, cm.ctypes.byref(b)) == cm.CM_ERR_INVALID


def test_images_above_65535_descriptors_are_rejected():
    lib = cm.lib()
    p = cm.Params.make()
    b = cm.ctypes.c_uint64()
    assert lib.cm_image_bytes(cm.ctypes.byref(p), 65535, cm.ctypes.byref(b)) == cm.CM_OK
    assert lib.cm_image_bytes(cm.ctypes.byref(p), 65536, cm.ctypes.byref(b)) == cm.CM_ERR_INVALID
    nd = np.array([10, 65536], dtype=np.int32)
    assert lib.cm_index_bytes(cm.ctypes.byref(p), 2, nd.ctypes.data, 0, cm.ctypes.byref(b)) == cm.CM_ERR_INVALID
    off = np.array([0, 10, 10 + 65536], dtype=np.int64)
    pr = np.array([[0, 1]], dtype=np.int32)
    fake = cm.ctypes.c_void_p(1 << 20)   # never dereferenced: the sizes are rejected first
    assert lib.cm_nn_pairs(fake, off.ctypes.data, 2, pr.ctypes.data, 1, 4, 5, fake, 1 << 30, fake, None, None,
                           None) == cm.CM_ERR_INVALID
    assert b"65535" in lib.cm_last_error()


def test_noalloc_rejects_unsupported_forms_before_touching_the_gpu():
    """The allocation-free entry point checks its parameters on the host: the
    tensor-core projection and scan and the tensor-core reranks are refused
    with CM_ERR_INVALID, images over 8,192 rows with CM_ERR_BUDGET."""
    import ctypes
    lib = cm.lib()
    sums = np.ones(128, np.uint64)
    fake = ctypes.c_void_p(1 << 20)    # never dereferenced: every case fails on the host first
    for kw, n_i, want in ((dict(projection="tc"), 10, cm.CM_ERR_INVALID),
                          (dict(projection="ffma", algo="tc"), 10, cm.CM_ERR_INVALID),
                          (dict(projection="ffma", rerank="bf16"), 10, cm.CM_ERR_INVALID),
                          (dict(projection="ffma"), 8193, cm.CM_ERR_BUDGET)):
        p = cm.Params.make(**kw)
        st = lib.cm_match_pair_noalloc(ctypes.byref(p), fake, n_i, fake, 10, sums.ctypes.data, 100, fake, None, None,
                                       None)
        assert st == want, (kw, st)
        assert lib.cm_last_error()


def test_auto_mapping_follows_the_plan_size():
    """AUTO sizes a plan as the bucket-major matcher's (pair order + per-query
    key lists) from 256 pairs on, and as the tile form's below; the
    tensor-core reranks keep their hand-over under either."""
    for rerank in ("fp32", "bf16", "fp8"):
        auto, bucket, tile = (cm.Params.make(rerank=rerank, algo=a) for a in ("auto", "bucket", "tile"))
        for n_pairs in (1, 255, 256, 4000):
            rows = 2000 * n_pairs
            want = bucket if n_pairs >= 256 else tile
            assert cm.plan_bytes(auto, n_pairs, rows, 2000) == cm.plan_bytes(want, n_pairs, rows, 2000)
        extra = cm.plan_bytes(bucket, 300, 600000, 2000) - cm.plan_bytes(tile, 300, 600000, 2000)
        assert extra >= 600000 * 8 * 4 + 300 * 4   # key lists and the pair order
