"""GPU tests of the block machinery around the fused match launch: compaction
into per-pair match lists (Algorithm 1's initial matches), the captured block
sequence (one CUDA graph) and the block-row pipeline with CPU verification
overlapped (Sec. 2.3.2).  Each result is compared with the plain plan-run
path, which the parity tests compare with the FP64 oracle."""
import numpy as np
import pytest

import paper_2505_22089_b300 as cm
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _index(wl, p, desc):
    return cm.Index.build(p, wl.n_desc, torch.from_numpy(desc).cuda())


def _direct(index, pairs):
    plan = cm.MatchPlan(index, pairs)
    out = plan.alloc_out()
    plan.run(out)
    torch.cuda.synchronize()
    return plan, out["best_j"].cpu().numpy()


def _lists(plan, best):
    """Per-pair match lists (query << 16 | j) from best_j, in query order."""
    res = []
    for k in range(len(plan.pairs)):
        b = best[plan.row_off[k]:plan.row_off[k + 1]]
        q = np.nonzero(b >= 0)[0]
        res.append(((q.astype(np.int64) << 16) | b[q].astype(np.int64)).astype(np.uint32))
    return res


def test_compaction_lists_counts_offsets():
    wl = synth.strip30(n_images=6, n=3000)
    desc = wl.generate()
    index = _index(wl, cm.Params.make(), desc)
    plan, best = _direct(index, wl.pairs)
    want = _lists(plan, best)
    counts, offsets, total, matches = plan.compact(torch.from_numpy(best).cuda())
    torch.cuda.synchronize()
    c, o, t, mt = (x.cpu().numpy() for x in (counts, offsets, total, matches))
    assert np.array_equal(c, [len(w) for w in want])
    assert np.array_equal(o, np.concatenate([[0], np.cumsum(c)[:-1]]))
    assert t[0] == sum(len(w) for w in want)
    for k, w in enumerate(want):
        assert np.array_equal(mt[o[k]:o[k] + c[k]].view(np.uint32), w)


def test_compaction_capacity_truncates_but_counts_stay_exact():
    wl = synth.pair2k()
    desc = wl.generate()
    index = _index(wl, cm.Params.make(), desc)
    plan, best = _direct(index, [[0, 1], [1, 0]])
    want = np.concatenate(_lists(plan, best))
    cap = len(want) // 2
    counts, offsets, total, matches = plan.compact(torch.from_numpy(best).cuda(), capacity=cap)
    torch.cuda.synchronize()
    assert int(total.cpu()[0]) == len(want)
    assert np.array_equal(matches.cpu().numpy()[:cap].view(np.uint32), want[:cap])


def test_compaction_empty_pairs():
    wl = synth.pair2k(n=200, shared=50)
    desc = wl.generate()
    n_desc = np.array([200, 200, 0], np.int32)
    index = cm.Index.build(cm.Params.make(), n_desc, torch.from_numpy(desc).cuda())
    plan, best = _direct(index, [[2, 0], [0, 2], [0, 1]])
    counts, offsets, total, _ = plan.compact(torch.from_numpy(np.concatenate([best, [-1]]).astype(np.int32)).cuda())
    torch.cuda.synchronize()
    c = counts.cpu().numpy()
    assert c[0] == 0 and c[1] == 0 and c[2] == (best[200:] >= 0).sum()


@pytest.mark.parametrize("rerank", ["fp32", "bf16"])
def test_captured_sequence_replays_the_block_rows(rerank):
    wl = synth.strip30(n_images=10, n=2500)
    desc = wl.generate()
    p = cm.Params.make(rerank=rerank)
    index = _index(wl, p, desc)
    rows = [wl.pairs[:15], wl.pairs[15:28], wl.pairs[28:]]
    plans = [cm.MatchPlan(index, r) for r in rows]
    outs = [pl.alloc_out(topk=True) for pl in plans]
    comps = [cm.compact_out(pl) for pl in plans]
    seq = cm.Sequence(index, plans, outs, comps, rehash=True)
    assert seq.kernels >= 3 * 4   # rehash kernels + per row one match launch and three compaction kernels
    ref_plan, ref_best = _direct(index, wl.pairs)
    for rep in range(2):
        for o in outs:
            o["best_j"].fill_(-7)
        seq.launch()
        torch.cuda.synchronize()
        got = np.concatenate([o["best_j"].cpu().numpy() for o in outs])
        assert np.array_equal(got, ref_best), rep
        for pl, o, c in zip(plans, outs, comps):
            want = _lists(pl, o["best_j"].cpu().numpy())
            off = c["offsets"].cpu().numpy()
            mt = c["matches"].cpu().numpy().view(np.uint32)
            for k, w in enumerate(want):
                assert np.array_equal(mt[off[k]:off[k] + len(w)], w)
    # a residency change invalidates the graph
    index.evict([9])
    with pytest.raises(cm.CMError) as e:
        seq.launch()
    assert e.value.status == cm.CM_ERR_STATE
    seq.close()


def test_sequence_rejects_the_default_stream_and_foreign_plans():
    wl = synth.pair2k(n=300, shared=100)
    desc = wl.generate()
    a = _index(wl, cm.Params.make(), desc)
    b = _index(wl, cm.Params.make(), desc)
    pb = cm.MatchPlan(b, [[0, 1]])
    with pytest.raises(cm.CMError) as e:
        cm.Sequence(a, [pb], [pb.alloc_out()])
    assert e.value.status == cm.CM_ERR_STATE
    pa = cm.MatchPlan(a, [[0, 1]])
    with pytest.raises(cm.CMError) as e:
        cm.Sequence(a, [pa], [pa.alloc_out()], stream=0)
    assert e.value.status == cm.CM_ERR_INVALID


def _grid_case(max_block=8):
    wl = synth.scaled("grid500", gx=6, gy=4, nmin=1500, nmax=4000)
    desc, kp = wl.generate(want_kp=True)
    off = wl.row_off
    p = cm.Params.make()
    sched = cm.schedule_blocks(wl.pairs, wl.n_desc, p, budget=1 << 34, max_images_per_block=max_block)
    host = [torch.from_numpy(desc[off[i]:off[i + 1]]).pin_memory() for i in range(wl.n_images)]
    kps = [kp[off[i]:off[i + 1]] for i in range(wl.n_images)]
    return wl, desc, p, sched, host, kps


def _pipeline_index(wl, p, desc):
    sums = desc.astype(np.uint64).sum(0)
    index = cm.Index(p, wl.n_desc)
    index.set_mean(sums, int(wl.total_desc))
    return index


def test_pipeline_equals_direct_matching():
    wl, desc, p, sched, host, _ = _grid_case()
    assert len(sched.rows) > 2
    got = {}

    def collect(row, pair_id, ij, matches):
        got[pair_id] = (row, ij, matches)
        return 0

    index = _pipeline_index(wl, p, desc)
    stats, _ = cm.run_schedule(index, sched, host, verify=collect, workers=3)
    assert sorted(got) == list(range(len(wl.pairs)))
    direct = _index(wl, p, desc)
    plan, best = _direct(direct, wl.pairs)
    want = _lists(plan, best)
    for k, (i, j) in enumerate(wl.pairs):
        assert got[k][1] == (i, j)
        assert np.array_equal(got[k][2], want[k]), k
    assert stats["rows"] == len(sched.rows)
    assert stats["pairs"] == len(wl.pairs)
    assert stats["matches"] == sum(len(w) for w in want)
    loads = sum(len(r["load"]) for r in sched.rows)
    assert loads >= wl.n_images
    assert stats["h2d_bytes"] == 128 * sum(int(wl.n_desc[i]) for r in sched.rows for i in r["load"])
    assert stats["d2h_bytes"] == 4 * stats["matches"] + 8 * sum(len(r["pairs"]) + 1 for r in sched.rows
                                                                if r["pairs"])
    # everything the pipeline loaded is released at the end: a second run works
    stats2, _ = cm.run_schedule(index, sched, host, verify=None, workers=1)
    assert stats2["matches"] == stats["matches"]


def test_pipeline_affine_verification_finds_the_shared_tracks():
    wl, desc, p, sched, host, kps = _grid_case()
    index = _pipeline_index(wl, p, desc)
    stats, inliers = cm.run_schedule(index, sched, host, verify="affine", keypoints=kps, thresh_px=4.0, workers=4)
    assert np.all(inliers >= 0)
    direct = _index(wl, p, desc)
    plan, best = _direct(direct, wl.pairs)
    n_match = np.array([len(w) for w in _lists(plan, best)])
    # overlapping views share tracks: most initial matches are geometric inliers
    share = inliers.sum() / max(1, n_match.sum())
    assert share > 0.8, share
    assert stats["verify_ms"] > 0


def test_pipeline_sao_then_affine_equals_the_host_calls():
    """The verifier with the SAO local constraint: per pair, the kept count is
    cm_sao_filter's on the pair's initial matches and the inlier count is
    cm_verify_affine's on the kept ones (same seed per pair)."""
    wl, desc, p, sched, host, kps = _grid_case()
    index = _pipeline_index(wl, p, desc)
    kept = np.full(len(wl.pairs), -1, dtype=np.int64)
    seed = 7
    stats, inliers = cm.run_schedule(index, sched, host, verify="affine", keypoints=kps, thresh_px=4.0, workers=4,
                                     seed=seed, sao_k=8, sao_max_score=0.875, sao_kept=kept)
    direct = _index(wl, p, desc)
    plan, best = _direct(direct, wl.pairs)
    lists = _lists(plan, best)
    for k, (i, j) in enumerate(wl.pairs):
        _, keep, nk = cm.sao_filter(kps[i], kps[j], lists[k], 8, 0.875)
        assert kept[k] == nk, k
        _, _, n_in = cm.verify_affine(kps[i], kps[j], lists[k][keep], thresh_px=4.0, max_iters=500,
                                      seed=seed ^ k)
        assert inliers[k] == n_in, k
    assert 0 < kept.sum() <= stats["matches"]


def test_pipeline_callback_abort_and_recovery():
    wl, desc, p, sched, host, _ = _grid_case()
    index = _pipeline_index(wl, p, desc)
    with pytest.raises(cm.CMError) as e:
        cm.run_schedule(index, sched, host, verify=lambda *a: 1, workers=2)
    assert e.value.status == cm.CM_ERR_STATE
    stats, _ = cm.run_schedule(index, sched, host, verify=None, workers=2)
    assert stats["pairs"] == len(wl.pairs)


@pytest.mark.parametrize("rerank", ["int", "bf16"])
def test_autotune_keeps_the_decisions(rerank):
    wl = synth.strip30(n_images=8, n=3000)
    desc = wl.generate()
    p = cm.Params.make(rerank=rerank)
    index = _index(wl, p, desc)
    _, before = _direct(index, wl.pairs)
    r = index.autotune(wl.pairs[:12])
    assert r["trials"] >= 3 and r["query_tile"] % 64 == 0 and r["K"] == 8
    assert (r["query_tile"] == 0) == (r["algo"] == "bucket")
    if rerank == "bf16":
        assert r["algo"] in ("bucket", "tile")
    _, after = _direct(index, wl.pairs)   # a plan made after tuning uses the chosen tile and mapping
    assert np.array_equal(before, after)


def test_autotune_chooses_K_under_an_agreement_floor():
    wl = synth.strip30(n_images=8, n=3000)
    desc = wl.generate()
    index = _index(wl, cm.Params.make(rerank="int"), desc)
    r = index.autotune(wl.pairs[:12], Ks=[4, 8, 16], min_agreement=0.99)
    assert r["K"] in (4, 8, 16) and r["agreement"] >= 0.99
    assert index.p.K == r["K"]
    plan, best = _direct(index, wl.pairs[:12])
    assert plan.K == r["K"]
    # a floor of 1.0 leaves only K values whose decisions equal the largest K's
    r2 = index.autotune(wl.pairs[:12], Ks=[4, 8, 16], min_agreement=1.0)
    assert r2["agreement"] == 1.0


@pytest.mark.parametrize("strategy,rerank", [("per_pair", "fp32"), ("pair_blocks", "fp32"), ("load_free_list", "fp32"),
                                             ("graph_partition", "fp32"), ("graph_partition", "fp8"),
                                             ("pair_blocks", "bf16")])
def test_other_schedule_strategies_give_the_same_matches(strategy, rerank):
    """Caller-built rows (cm_schedule_from_rows) through the pipeline: rows
    that reload an image the previous row frees, rows without loads, many
    small rows, and the tensor-core forms whose plans carry large hand-overs,
    all in an arena of exactly cm_schedule_arena_bytes; the match lists equal
    direct matching."""
    from paper_2505_22089_b300 import strategies as st
    wl, desc, _, _, host, _ = _grid_case()
    p = cm.Params.make(rerank=rerank)
    ib = np.array([cm.image_bytes(p, int(n)) for n in wl.n_desc], dtype=np.int64)
    budget = int(ib.sum() // 3)
    order = st.connection_order(wl.pairs, wl.n_images, cm.gps_order)
    rows = {"per_pair": lambda: st.per_pair(wl.pairs),
            "pair_blocks": lambda: st.pair_blocks(wl.pairs, ib, budget),
            "load_free_list": lambda: st.load_free_list(wl.pairs, ib, budget, order),
            "graph_partition": lambda: st.graph_partition(wl.pairs, ib, budget, order,
                                                          max(1, int(budget // 2 // ib.max())))}[strategy]()
    sched = cm.schedule_from_rows(rows, wl.pairs, wl.n_images)
    sums = desc.astype(np.uint64).sum(0)
    index = cm.Index(p, wl.n_desc, arena_bytes=cm.schedule_arena_bytes(sched, p, wl.n_desc))
    index.set_mean(sums, int(wl.total_desc))
    got = {}

    def collect(row, pair_id, ij, matches):
        got[pair_id] = matches
        return 0

    stats, _ = cm.run_schedule(index, sched, host, verify=collect, workers=2)
    direct = _index(wl, p, desc)
    plan, best = _direct(direct, wl.pairs)
    want = _lists(plan, best)
    assert sorted(got) == list(range(len(wl.pairs)))
    for k in range(len(wl.pairs)):
        assert np.array_equal(got[k], want[k]), k
    assert stats["rows"] == len(rows)


def test_pipeline_with_the_gpu_sao_constraint():
    """SAO on the GPU inside the pipeline: verification receives exactly the
    matches the host form keeps from the unfiltered lists."""
    wl, desc, p, sched, host, kps = _grid_case()
    index = _pipeline_index(wl, p, desc)
    kp_all = np.concatenate(kps).astype(np.float32)
    kp_dev = torch.from_numpy(kp_all).cuda()
    off_dev = torch.from_numpy(wl.row_off.astype(np.int64)).cuda()
    got = {}

    def collect(row, pair_id, ij, matches):
        got[pair_id] = matches
        return 0

    stats, _ = cm.run_schedule(index, sched, host, verify=collect, workers=3, gpu_sao_k=8, sao_max_score=0.875,
                               kp_dev=kp_dev, kp_off_dev=off_dev)
    direct = _index(wl, p, desc)
    plan, best = _direct(direct, wl.pairs)
    want = _lists(plan, best)
    kept = 0
    for k, (i, j) in enumerate(wl.pairs):
        _, keep, n = cm.sao_filter(kps[i], kps[j], want[k], 8, 0.875)
        assert np.array_equal(got[k], want[k][keep]), k
        kept += n
    assert stats["matches"] == kept
