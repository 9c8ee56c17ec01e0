"""GPU parity of the block machinery against the FP64 oracle: the per-pair
match lists that leave the block-row pipeline (cm_run_schedule, Algorithm 1:
load, match, compaction, free, with the next row's copies prefetched into
arena space freed by earlier rows) and a captured block sequence replayed as
one CUDA graph (rehash, then per row the fused match launch and compaction)
are compared list by list with oracle.Index.match on the same descriptors.

The oracle computes its own centring sums from the raw rows (the library's
sums are only compared with them).  Queries that a differing marginal code
bit can touch are excluded from the exact checks, as in the other parity
tests; the FP32 and BF16 forms must then equal the oracle exactly, the FP8
form on >= 99.5 % of decisions."""
import numpy as np
import pytest

import oracle
import paper_2505_22089_b300 as cm
import synth
from gpu_common import affected_queries, compare_hash, oparams

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _grid(gx=6, gy=4):
    wl = synth.scaled("grid500", gx=gx, gy=gy, nmin=1500, nmax=4000)
    return wl, wl.generate()


def _decode(lst, n_i):
    """Per-query best_j from a match list (query << 16 | j, query order)."""
    best = np.full(n_i, -1, dtype=np.int32)
    lst = np.asarray(lst, dtype=np.uint32)
    q = (lst >> 16).astype(np.int64)
    assert np.all(np.diff(q) > 0), "a match list is not in strictly increasing query order"
    best[q] = (lst & 0xFFFF).astype(np.int32)
    return best


def _compare_lists(lists, pairs, oix, p, affected, form):
    """lists[k]: pair k's match list.  Returns (queries compared, excluded,
    decision agreement, match-set Jaccard) and asserts the form's bar."""
    op = oparams(p)
    same = total = excl = inter = union = 0
    for k, (i, j) in enumerate(np.asarray(pairs).reshape(-1, 2)):
        I = oix.image(int(i))
        o = oracle.match_pair(I, oix.image(int(j)), op, topk=True)
        ok = ~affected_queries(p, oix, int(i), int(j), affected, o["topk"])
        g = _decode(lists[k], I.n)
        if form != "fp8":
            assert np.array_equal(g[ok], o["best_j"][ok]), "pair %d (%d,%d): match list differs" % (k, i, j)
        same += int(((g == o["best_j"]) & ok).sum())
        total += int(ok.sum())
        excl += int((~ok).sum())
        gm = set(zip(np.nonzero(g >= 0)[0].tolist(), g[g >= 0].tolist()))
        om = set(zip(np.nonzero(o["best_j"] >= 0)[0].tolist(), o["best_j"][o["best_j"] >= 0].tolist()))
        inter += len(gm & om)
        union += len(gm | om)
    agree = same / max(total, 1)
    jac = inter / union if union else 1.0
    if form == "fp8":
        assert agree >= 0.995, agree
        assert jac >= 0.99, jac
    else:
        assert agree == 1.0
        assert jac >= 0.999, jac
    assert excl <= 0.02 * (total + excl) + 10, (excl, total)
    return total, excl, agree, jac


@pytest.mark.parametrize("form,centre", [("fp32", "mean_host"), ("bf16", "mean_host"), ("fp8", "mean_host"),
                                         ("bf16", "pipeline")])
def test_pipeline_match_lists_equal_the_oracle(form, centre):
    wl, desc = _grid()
    off = wl.row_off
    p = cm.Params.make(rerank=form)
    ib = sum(cm.image_bytes(p, int(n)) for n in wl.n_desc)
    # a third of the images' bytes: rows load and free in turn over several MBR iterations
    sched = cm.schedule_blocks(wl.pairs, wl.n_desc, p, budget=ib // 3, max_images_per_block=4)
    assert len(sched.rows) >= 3 and sched.iterations >= 2
    arena = cm.schedule_arena_bytes(sched, p, wl.n_desc)
    assert arena < ib, "the arena must be smaller than all images together, so freed space is reused"
    host = [torch.from_numpy(desc[off[i]:off[i + 1]]).pin_memory() for i in range(wl.n_images)]
    index = cm.Index(p, wl.n_desc, arena_bytes=arena)
    oix = oracle.Index(desc, wl.n_desc, oparams(p))          # the oracle's own sums
    if centre == "mean_host":
        index.mean_host(host)                               # the library's own centring sums, from host rows
        sums, n_total = index.col_sums()
        assert n_total == wl.total_desc and np.array_equal(sums, oix.sums)
    got = {}

    def collect(row, pair_id, ij, matches):
        got[pair_id] = matches
        return 0

    # centre == "pipeline": the run computes the mean itself (row 0's images summed in their slots)
    stats, _ = cm.run_schedule(index, sched, host, verify=collect, workers=2, centre=centre == "pipeline")
    if centre == "pipeline":
        sums, n_total = index.col_sums()
        assert n_total == wl.total_desc and np.array_equal(sums, oix.sums)
        assert stats["h2d_bytes"] == 128 * (wl.total_desc + sum(int(wl.n_desc[i]) for r in sched.rows[1:]
                                                                for i in r["load"]))
    assert sorted(got) == list(range(len(wl.pairs)))
    assert stats["rows"] == len(sched.rows) and stats["prefetched_rows"] >= 1, stats
    # the marginal-bit exclusions come from the same kernels on a resident index with the same mean
    direct = cm.Index.build(p, wl.n_desc, torch.from_numpy(desc).cuda())
    affected, n_diff, _, n_bits = compare_hash(direct, oix, range(wl.n_images), p)
    assert n_diff <= 1e-4 * n_bits
    total, excl, agree, jac = _compare_lists([got[k] for k in range(len(wl.pairs))], wl.pairs, oix, p, affected,
                                             form)
    assert stats["matches"] == sum(len(v) for v in got.values())
    print("pipeline %s: %d rows (%d prefetched), queries exact %d, excluded %d, agreement %.6f, jaccard %.6f"
          % (form, stats["rows"], stats["prefetched_rows"], total, excl, agree, jac))


@pytest.mark.parametrize("form", ["bf16", "fp8"])
def test_captured_sequence_lists_equal_the_oracle(form):
    """Residency with reuse of freed space, then a graph of rehash + 3 rows:
    the rehash re-centres on the resident images, so the oracle takes its own
    sums over those images' rows."""
    wl, desc = _grid(gx=5, gy=4)
    off = wl.row_off
    p = cm.Params.make(rerank=form)
    n = wl.n_images
    first, later = list(range(0, 12)), list(range(12, n))
    dropped = first[:6]
    # arena: room for the fixed tables, the first 12 images and the plans, not for all images at once
    ib = [cm.image_bytes(p, int(x)) for x in wl.n_desc]
    need = max(sum(ib[i] for i in first), sum(ib[i] for i in first if i not in dropped) + sum(ib[i] for i in later))
    arena = cm.index_bytes(p, [0] * n) + need + need // 4 + cm.default_headroom(p, wl.n_desc)
    assert sum(ib) > need + need // 4, "the later images fit only into the space the evicted ones free"
    index = cm.Index(p, wl.n_desc, arena_bytes=arena)
    index.set_mean(desc.astype(np.uint64).sum(0), int(wl.total_desc))
    index.load(first, [desc[off[i]:off[i + 1]] for i in first], cm.MEM_HOST)
    index.evict(dropped)
    index.load(later, [desc[off[i]:off[i + 1]] for i in later], cm.MEM_HOST)   # into the freed space
    resident = sorted(set(first) - set(dropped) | set(later))
    pr = [(int(i), int(j)) for i, j in wl.pairs if int(i) in resident and int(j) in resident]
    assert len(pr) >= 12
    rows = [pr[: len(pr) // 3], pr[len(pr) // 3: 2 * len(pr) // 3], pr[2 * len(pr) // 3:]]
    plans = [cm.MatchPlan(index, r) for r in rows]
    outs = [pl.alloc_out(d12=False) for pl in plans]
    comps = [cm.compact_out(pl) for pl in plans]
    seq = cm.Sequence(index, plans, outs, comps, rehash=True)
    rrows = np.concatenate([desc[off[i]:off[i + 1]] for i in resident])
    oix = oracle.Index(desc, wl.n_desc, oparams(p), sums=oracle.col_sums(rrows), n_total=len(rrows))
    for rep in range(2):
        for c in comps:
            c["matches"].fill_(-7)
        seq.launch()
        torch.cuda.synchronize()
        sums, n_total = index.col_sums()
        assert n_total == len(rrows) and np.array_equal(sums, oix.sums)
        if rep == 0:
            affected, n_diff, _, n_bits = compare_hash(index, oix, resident, p)
            assert n_diff <= 1e-4 * n_bits
        lists = []
        for pl, c in zip(plans, comps):
            cnt = c["counts"].cpu().numpy()
            o = c["offsets"].cpu().numpy()
            mt = c["matches"].cpu().numpy().view(np.uint32)
            lists += [mt[o[k]:o[k] + cnt[k]] for k in range(len(pl.pairs))]
        total, excl, agree, jac = _compare_lists(lists, pr, oix, p, affected, form)
        print("sequence %s replay %d: queries exact %d, excluded %d, agreement %.6f, jaccard %.6f"
              % (form, rep, total, excl, agree, jac))
    seq.close()


def test_match_pairs_async_equals_the_oracle():
    """cm_match_pairs with a caller workspace (no arena space taken), sized by
    cm_index_workspace_bytes for a schedule row, run on a side stream."""
    wl, desc = _grid(gx=4, gy=3)
    p = cm.Params.make()
    index = cm.Index.build(p, wl.n_desc, torch.from_numpy(desc).cuda())
    sched = cm.schedule_blocks(wl.pairs, wl.n_desc, p, budget=1 << 34, max_images_per_block=3)
    oix = oracle.Index(desc, wl.n_desc, oparams(p))
    affected, *_ = compare_hash(index, oix, range(wl.n_images), p)
    ws_max = index.workspace_bytes(sched, -1)
    s = torch.cuda.Stream()
    for r, row in enumerate(sched.rows):
        if not row["pairs"]:
            continue
        rp = wl.pairs[np.asarray(row["pairs"], dtype=np.int64)]
        need = index.workspace_bytes(sched, r)
        assert need == index.match_pairs_bytes(rp) and need <= ws_max
        work = torch.empty(need + 256, dtype=torch.uint8, device="cuda")
        rows_n = int(wl.n_desc[rp[:, 0]].sum())
        best = torch.full((rows_n,), -7, dtype=torch.int32, device="cuda")
        d1 = torch.empty(rows_n, dtype=torch.int32, device="cuda")
        d2 = torch.empty(rows_n, dtype=torch.int32, device="cuda")
        s.wait_stream(torch.cuda.current_stream())
        index.match_pairs(rp, work, best, d1, d2, stream=s)
        s.synchronize()
        b = best.cpu().numpy()
        ro = np.concatenate([[0], np.cumsum(wl.n_desc[rp[:, 0]])])
        lists = []
        for k in range(len(rp)):
            bk = b[ro[k]:ro[k + 1]]
            q = np.nonzero(bk >= 0)[0]
            lists.append(((q.astype(np.int64) << 16) | bk[q].astype(np.int64)).astype(np.uint32))
        _compare_lists(lists, rp, oix, p, affected, "fp32")
    small = torch.empty(256 + 64, dtype=torch.uint8, device="cuda")
    rp = wl.pairs[:4]
    out = torch.empty(int(wl.n_desc[rp[:, 0]].sum()), dtype=torch.int32, device="cuda")
    with pytest.raises(cm.CMError) as e:
        index.match_pairs(rp, small, out)
    assert e.value.status == cm.CM_ERR_BUDGET
