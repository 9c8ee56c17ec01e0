"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.  Tolerances: key/code bits exact except marginal bits
(|s| < 1e-4 ||x~||, counted, < 0.01 % of bits); bucket tables, top-K lists,
squared distances and match decisions exact on every query that no differing
bit touches; match-set agreement >= 99.9 %."""
import numpy as np
import pytest

import oracle
import paper_2505_22089_b300 as cm
import synth
from gpu_common import compare_hash, compare_match, gpu_match, oparams

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _run(wl, p: cm.Params, pairs=None, desc=None, check_topk=True, threads=None):
    desc = wl.generate() if desc is None else desc
    pairs = wl.pairs if pairs is None else pairs
    index = cm.Index.build(p, wl.n_desc, torch.from_numpy(desc).cuda())
    plan, res = gpu_match(index, pairs)
    oix = oracle.Index(desc, wl.n_desc, oparams(p), threads=threads)
    imgs = sorted(set(np.asarray(pairs).reshape(-1).tolist()))
    affected, n_diff, n_marg, n_bits = compare_hash(index, oix, imgs, p)
    assert n_marg <= 1e-4 * n_bits + 10
    rows, excl, jac = compare_match(plan, res, oix, pairs, p, affected, check_topk)
    # differing bits are rare (FP32 vs FP64 projections); the queries they can
    # touch are excluded from the exact checks and bounded here
    assert n_diff <= 1e-4 * n_bits, (n_diff, n_bits)
    # a differing bit of a database point can reach every query that shares one
    # of its buckets and ranks it near the K-th place (a few % at small N)
    assert excl <= 0.02 * (rows + excl) + 10, (excl, rows, n_diff)
    assert jac >= 0.999, (jac, excl, n_diff)
    print("parity: rows exact %d, excluded %d, differing bits %d of %d, jaccard %.6f" % (rows, excl, n_diff,
                                                                                         n_bits, jac))
    return res, rows, excl, n_diff


def test_pair2k_paper_defaults():
    res, rows, excl, n_diff = _run(synth.pair2k(), cm.Params.make())
    assert rows + excl == 2000
    # 800 of the query image's descriptors have a sigma-8 copy in the database image
    assert 500 < (res["best_j"] >= 0).sum() < 1000


@pytest.mark.parametrize("algo", ["tile", "warp"])
@pytest.mark.parametrize("tile", [64, 256, 640, 2048])
def test_pair2k_query_tiles_with_ragged_tail(tile, algo):
    _run(synth.pair2k(), cm.Params.make(query_tile=tile, algo=algo))


@pytest.mark.parametrize("algo", ["bucket", "tile", "warp", "tc"])
def test_pair2k_integer_rerank(algo):
    _run(synth.pair2k(), cm.Params.make(rerank="int", algo=algo))


@pytest.mark.parametrize("algo", ["bucket", "tile", "warp", "tc"])
def test_strip30_full_block(algo):
    # 30 images x 8,000 descriptors, 120 ordered pairs: one MBR block
    _run(synth.strip30(), cm.Params.make(algo=algo), threads=16)


@pytest.mark.parametrize("projection", ["tc", "ffma"])
@pytest.mark.parametrize("kw", [dict(), dict(L=8, m=8), dict(L=1, m=0), dict(L=3, m=5)])
def test_projection_forms(projection, kw):
    # tensor-core (BF16x3, FP32 accumulate) and CUDA-core FP32 projections: every
    # bit that differs from the FP64 oracle must be marginal
    _run(synth.pair2k(n=3000, shared=1000), cm.Params.make(projection=projection, **kw))


@pytest.mark.parametrize("algo", ["bucket", "tile", "warp", "tc"])
def test_uneven_sizes_including_tiny_images(algo):
    wl = synth.grid500(gx=5, gy=4, nmin=1, nmax=5000)
    wl.images["n"][[0, 7]] = [1, 63]
    _run(wl, cm.Params.make(query_tile=512, algo=algo))


@pytest.mark.parametrize("kw", [dict(K=2), dict(K=4), dict(K=16), dict(m=4), dict(m=0, K=16), dict(L=1),
                                dict(L=8), dict(L=8, m=6), dict(ratio=(0, 1)), dict(ratio=(1, 2)),
                                dict(ratio=(1, 1)), dict(seed=12345)])
@pytest.mark.parametrize("algo", ["bucket", "tile", "warp", "tc"])
def test_parameter_variants(kw, algo):
    if algo == "tc" and kw.get("K") == 2:
        pytest.skip("the tensor-core scan keeps K >= 4")
    wl = synth.pair2k(n=1500, shared=600)
    _run(wl, cm.Params.make(algo=algo, **kw))


@pytest.mark.parametrize("algo", ["bucket", "tile", "warp", "tc"])
def test_one_bucket_full_rerank_is_exhaustive_nn(algo):
    # m = 0 and K >= N_J: every database point is reranked, so the GPU result
    # equals exhaustive L2 nearest neighbours with the ratio test.
    wl = synth.pair2k(n=16, shared=6)
    desc = wl.generate()
    p = cm.Params.make(m=0, K=16, algo=algo)
    index = cm.Index.build(p, wl.n_desc, torch.from_numpy(desc).cuda())
    plan, res = gpu_match(index, wl.pairs)
    bf = oracle.brute_nn(desc[:16], desc[16:], 4, 5)
    assert np.array_equal(res["best_j"], bf["best_j"])
    assert np.array_equal(res["d1sq"], bf["d1sq"]) and np.array_equal(res["d2sq"], bf["d2sq"])


def test_empty_and_single_descriptor_images():
    wl = synth.pair2k(n=300, shared=100)
    desc = wl.generate()
    # images: 0 (300), 1 (300), 2 (empty), 3 (one descriptor)
    n_desc = np.array([300, 300, 0, 1], dtype=np.int32)
    all_desc = np.concatenate([desc, desc[:1]])
    p = cm.Params.make()
    index = cm.Index.build(p, n_desc, torch.from_numpy(all_desc).cuda())
    pairs = np.array([[0, 2], [2, 0], [0, 3], [3, 0], [0, 1]], dtype=np.int32)
    plan, res = gpu_match(index, pairs)
    assert plan.rows == 300 + 0 + 300 + 1 + 300
    r = plan.row_off
    assert np.all(res["best_j"][r[0]:r[1]] == -1) and np.all(res["d1sq"][r[0]:r[1]] == 0xFFFFFFFF)
    assert np.all(res["best_j"][r[2]:r[3]] == -1) and np.all(res["d2sq"][r[2]:r[3]] == 0xFFFFFFFF)
    oix = oracle.Index(all_desc, n_desc, oparams(p))
    o = oracle.match_pair(oix.image(3), oix.image(0), oparams(p), topk=True)
    assert np.array_equal(res["best_j"][r[3]:r[4]], o["best_j"])
    assert np.array_equal(res["d1sq"][r[3]:r[4]], o["d1sq"])


def test_plan_and_index_errors():
    wl = synth.pair2k(n=200, shared=50)
    desc = wl.generate()
    p = cm.Params.make()
    index = cm.Index.build(p, wl.n_desc, torch.from_numpy(desc).cuda())
    for bad, status in (([[0, 0]], cm.CM_ERR_INVALID), ([[0, 2]], cm.CM_ERR_INVALID), ([[-1, 1]], cm.CM_ERR_INVALID)):
        with pytest.raises(cm.CMError) as e:
            cm.MatchPlan(index, bad)
        assert e.value.status == status
    index.evict([1])
    with pytest.raises(cm.CMError) as e:
        cm.MatchPlan(index, [[0, 1]])
    assert e.value.status == cm.CM_ERR_STATE
    with pytest.raises(cm.CMError) as e:
        index.evict([1])
    assert e.value.status == cm.CM_ERR_STATE
    with pytest.raises(cm.CMError) as e:
        cm.Index.build(p, wl.n_desc, torch.from_numpy(desc).cuda(), arena_bytes=1 << 16)
    assert e.value.status == cm.CM_ERR_BUDGET


def test_load_evict_rehash_cycle():
    # Block-row style residency: images come and go; results match the oracle
    # computed with the same global centring mean.
    wl = synth.strip30(n_images=8, n=1200)
    desc = wl.generate()
    p = cm.Params.make()
    off = wl.row_off
    oix = oracle.Index(desc, wl.n_desc, oparams(p))
    # room for 70 % of the images plus one window's plan (its pair table and per-query lists)
    plan_room = cm.plan_bytes(p, 12, 12 * 1200, 1200)
    index = cm.Index(p, wl.n_desc, arena_bytes=int(cm.index_bytes(p, wl.n_desc) * 0.7) + plan_room)
    index.set_mean(oix.sums, int(off[-1]))
    dev = torch.from_numpy(desc).cuda()
    rows_seen = 0
    for window in ([0, 1, 2, 3], [2, 3, 4, 5], [4, 5, 6, 7]):
        new = [w for w in window if w not in (getattr(index, "_res", set()))]
        index.load(new, [dev[off[w]:off[w + 1]] for w in new], cm.MEM_DEVICE)
        index._res = set(window)
        pairs = [(a, b) for a in window for b in window if a != b]
        plan, res = gpu_match(index, pairs)
        affected, *_ = compare_hash(index, oix, window, p)
        rows, excl, jac = compare_match(plan, res, oix, pairs, p, affected)
        rows_seen += rows
        index.evict(window[:2])
    assert rows_seen > 0
    # rehash recomputes the mean over the resident images only
    index.rehash()
    torch.cuda.synchronize()


def test_plan_rerun_is_deterministic():
    wl = synth.pair2k()
    desc = wl.generate()
    p = cm.Params.make()
    index = cm.Index.build(p, wl.n_desc, torch.from_numpy(desc).cuda())
    plan = cm.MatchPlan(index, [[0, 1], [1, 0]])
    outs = []
    for _ in range(3):
        out = plan.alloc_out(topk=True)
        plan.run(out)
        index.rehash()
        torch.cuda.synchronize()
        outs.append({k: v.cpu().numpy() for k, v in out.items() if k != "stats"})
    for o in outs[1:]:
        for k in o:
            assert np.array_equal(o[k], outs[0][k])


@pytest.mark.parametrize("rerank", ["fp32", "bf16"])
def test_marked_run_times_the_lookup_launch(rerank):
    # cm_match_plan_run_marked records the caller's event between the lookup
    # and the rerank launch; the results are those of cm_match_plan_run
    wl = synth.strip30(n_images=4, n=3000)
    index = cm.Index.build(cm.Params.make(rerank=rerank), wl.n_desc, torch.from_numpy(wl.generate()).cuda())
    plan = cm.MatchPlan(index, wl.pairs)
    a, b = plan.alloc_out(), plan.alloc_out()
    plan.run(a)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ev[0].record()
    plan.run(b, scan_done=ev[1])
    ev[2].record()
    torch.cuda.synchronize()
    for k in ("best_j", "d1sq", "d2sq"):
        assert torch.equal(a[k], b[k])
    t_scan, t_all = ev[0].elapsed_time(ev[1]), ev[0].elapsed_time(ev[2])
    assert 0 < t_scan <= t_all


@pytest.mark.parametrize("K", [2, 4, 8, 16])
def test_bf16_tensor_core_rerank_is_exact(K):
    # BF16 holds uint8 exactly and the FP32 accumulation of integer products is
    # exact, so the tcgen05 rerank must equal the oracle bit for bit
    _run(synth.pair2k(n=1500, shared=600), cm.Params.make(rerank="bf16", K=K))


def test_bf16_tensor_core_rerank_full_strip():
    _run(synth.strip30(), cm.Params.make(rerank="bf16"), threads=16)


def test_bf16_form_equals_fp32_form_on_a_grid():
    # BF16 products of uint8 and their FP32 sums are exact, so the tensor-core
    # rerank must decide every query as the CUDA-core FP32 form does.  A grid
    # of 20,000-descriptor images gives every CTA hundreds of sub-tiles, so the
    # stage and accumulator rings wrap many times (the small cases above give
    # a CTA one sub-tile or none)
    wl = synth.scaled("grid5000", gx=8, gy=5)
    desc = torch.from_numpy(wl.generate()).cuda()
    res = {}
    for form in ("fp32", "bf16", "bf16"):
        index = cm.Index.build(cm.Params.make(rerank=form), wl.n_desc, desc)
        plan = cm.MatchPlan(index, wl.pairs)
        out = plan.alloc_out()
        plan.run(out)
        torch.cuda.synchronize()
        got = tuple(out[k].cpu().numpy() for k in ("best_j", "d1sq", "d2sq"))
        if form in res:   # a rerun gives the same bits
            assert all(np.array_equal(a, b) for a, b in zip(got, res[form]))
        res[form] = got
        del plan, index, out
    for a, b in zip(res["bf16"], res["fp32"]):
        assert np.array_equal(a, b)
    assert (res["bf16"][0] >= 0).sum() > 0.1 * len(res["bf16"][0])


@pytest.mark.parametrize("K", [2, 4, 8, 16])
def test_fp8_tensor_core_rerank(K):
    # E4M3 distances pick q1, q2, which are re-scored exactly: top-K lists are
    # exact, re-scored distances are exact wherever the decision agrees, and the
    # decisions agree with the oracle on >= 99.5 % of queries
    wl = synth.strip30(n_images=6, n=4000)
    desc = wl.generate()
    p = cm.Params.make(rerank="fp8", K=K)
    index = cm.Index.build(p, wl.n_desc, torch.from_numpy(desc).cuda())
    plan, res = gpu_match(index, wl.pairs)
    oix = oracle.Index(desc, wl.n_desc, oparams(p))
    affected, *_ = compare_hash(index, oix, range(wl.n_images), p)
    same = total = 0
    for k, (i, j) in enumerate(wl.pairs):
        r0, r1 = plan.row_off[k], plan.row_off[k + 1]
        o = oracle.match_pair(oix.image(i), oix.image(j), oparams(p), topk=True)
        from gpu_common import affected_queries
        ok = ~affected_queries(p, oix, int(i), int(j), affected, o["topk"])
        assert np.array_equal(res["topk"][r0:r1][ok], o["topk"][ok])
        g = res["best_j"][r0:r1]
        agree = (g == o["best_j"]) & ok
        same += int(agree.sum())
        total += int(ok.sum())
        both = agree & (g >= 0)
        assert np.array_equal(res["d1sq"][r0:r1][both], o["d1sq"][both])
    assert same / total >= 0.995, same / total
    print("fp8 K=%d decision agreement %.5f, top-2 re-score swaps %d" % (K, same / total, res["stats"][2]))


def test_tensor_core_scan_pair2k_defaults():
    res, rows, excl, n_diff = _run(synth.pair2k(), cm.Params.make(algo="tc"))
    assert rows + excl == 2000


@pytest.mark.parametrize("rerank", ["bf16", "fp32"])
def test_tensor_core_scan_big_buckets(rerank):
    # m = 2: four buckets of ~1,000 points per table, so a bucket spans several
    # 128-row query tiles and 128-column database chunks
    _run(synth.pair2k(n=4000, shared=1500), cm.Params.make(algo="tc", m=2, rerank=rerank))


@pytest.mark.parametrize("K", [4, 8, 16])
def test_tensor_core_scan_equals_tile_scan(K):
    # the two scans rank the same candidates by the same exact keys
    wl = synth.strip30(n_images=6, n=3000)
    desc = wl.generate()
    outs = []
    for algo in ("tile", "tc"):
        p = cm.Params.make(algo=algo, K=K, rerank="int")
        index = cm.Index.build(p, wl.n_desc, torch.from_numpy(desc).cuda())
        plan, res = gpu_match(index, wl.pairs)
        outs.append(res)
    for key in ("best_j", "d1sq", "d2sq", "topk"):
        assert np.array_equal(outs[0][key], outs[1][key]), key


@pytest.mark.parametrize("rerank", ["int", "bf16"])
def test_bucket_major_equals_tile_form_on_a_grid(rerank):
    """The bucket-major matcher (units of 32 queries of one bucket, database runs
    staged in chunks of 64 by bulk copies) against the tile form on uneven
    images with long runs: top-K lists, distances and decisions bit for bit."""
    wl = synth.scaled("grid500", gx=5, gy=4, nmin=2000, nmax=12000)
    desc = wl.generate()
    res = {}
    for algo in ("bucket", "tile"):
        p = cm.Params.make(rerank=rerank, algo=algo)
        index = cm.Index.build(p, wl.n_desc, torch.from_numpy(desc).cuda())
        plan, got = gpu_match(index, wl.pairs)
        res[algo] = got
        del plan, index
    for k in ("best_j", "d1sq", "d2sq", "topk"):
        assert np.array_equal(res["bucket"][k], res["tile"][k]), k
    assert (res["bucket"]["best_j"] >= 0).sum() > 0.1 * len(res["bucket"]["best_j"])
