"""cm_match_pair_noalloc: matching for callers that may not allocate GPU memory.

Such callers (code inside another framework's memory budget, plug-ins of a
process that owns the device, real-time paths where an allocation could block
or fail) pass only inputs and outputs; the library's scratch is a fixed 5 MiB
device array shared by every call.  The calls below run back to back, a small
image pair after the largest one the array holds, so a call that read what
the previous call left in the array would show.  Each result is compared with
the index path under the same projection and thread mapping, and with the
FP64 oracle.  This file is collected last so that a run stopping at the first
failure has already run every other test."""
import numpy as np
import pytest

import oracle
import paper_2505_22089_b300 as cm
import synth
from gpu_common import affected_queries, compare_hash, oparams

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _workload():
    wl = synth.strip30(n_images=5, n=3000)
    wl.images["n"][3] = 8192                      # the largest image the scratch holds
    wl.images["n"][4] = 0                         # an empty database image
    return wl, wl.generate()


def _index_path(p, wl, dev, pairs):
    index = cm.Index.build(p, wl.n_desc, dev)
    plan = cm.MatchPlan(index, pairs)
    out = plan.alloc_out()
    plan.run(out)
    torch.cuda.synchronize()
    res = {k: out[k].cpu().numpy().view(np.uint32 if k != "best_j" else np.int32) for k in ("best_j", "d1sq", "d2sq")}
    return index, res, plan.row_off


@pytest.mark.parametrize("algo", ["tile", "warp"])
@pytest.mark.parametrize("rerank", ["fp32", "int"])
def test_noalloc_equals_index_path_and_oracle_on_calls_in_a_row(rerank, algo):
    wl, desc = _workload()
    dev = torch.from_numpy(desc).cuda()
    off = wl.row_off
    p = cm.Params.make(rerank=rerank, projection="ffma", algo=algo)
    calls = [(0, 1), (3, 2), (0, 1), (2, 4)]      # a smaller pair after the largest; an empty database image
    uniq = sorted(set(calls))
    index, ref, row_off = _index_path(p, wl, dev, uniq)
    sums, n_total = index.col_sums()
    oix = oracle.Index(desc, wl.n_desc, oparams(p))
    assert np.array_equal(sums, oix.sums)
    affected, *_ = compare_hash(index, oix, range(wl.n_images), p)
    for i, j in calls:
        n_i = int(wl.n_desc[i])
        best = torch.full((n_i,), -7, dtype=torch.int32, device="cuda")
        d1 = torch.zeros(n_i, dtype=torch.int32, device="cuda")
        d2 = torch.zeros(n_i, dtype=torch.int32, device="cuda")
        cm.match_pair_noalloc(p, dev[off[i]:off[i + 1]], dev[off[j]:off[j + 1]], sums, n_total, best, d1, d2)
        torch.cuda.synchronize()
        k = uniq.index((i, j))
        r0, r1 = row_off[k], row_off[k + 1]
        g_best = best.cpu().numpy()
        assert np.array_equal(g_best, ref["best_j"][r0:r1])
        assert np.array_equal(d1.cpu().numpy().view(np.uint32), ref["d1sq"][r0:r1])
        assert np.array_equal(d2.cpu().numpy().view(np.uint32), ref["d2sq"][r0:r1])
        o = oracle.match_pair(oix.image(i), oix.image(j), oparams(p), topk=True)
        ok = ~affected_queries(p, oix, i, j, affected, o["topk"])
        assert np.array_equal(g_best[ok], o["best_j"][ok])
        assert np.array_equal(d1.cpu().numpy().view(np.uint32)[ok], o["d1sq"][ok])
        if wl.n_desc[j] == 0:
            assert (g_best == -1).all()
        else:
            assert (g_best >= 0).sum() > 0


def test_noalloc_rejects_what_it_cannot_do():
    wl = synth.pair2k(n=100, shared=10)
    dev = torch.from_numpy(wl.generate()).cuda()
    big = torch.zeros((8193, 128), dtype=torch.uint8, device="cuda")
    out = torch.empty(8193, dtype=torch.int32, device="cuda")
    p = cm.Params.make(projection="ffma")
    with pytest.raises(cm.CMError) as e:
        cm.match_pair_noalloc(p, big, dev[:100], np.ones(128, np.uint64), 100, out)
    assert e.value.status == cm.CM_ERR_BUDGET and "8192" in str(e.value)
    for bad in (cm.Params.make(projection="tc"), cm.Params.make(projection="ffma", algo="tc"),
                cm.Params.make(projection="ffma", rerank="bf16")):
        with pytest.raises(cm.CMError) as e:
            cm.match_pair_noalloc(bad, dev[:100], dev[100:], np.ones(128, np.uint64), 100, out)
        assert e.value.status == cm.CM_ERR_INVALID
    with pytest.raises(ValueError):
        cm.match_pair_noalloc(p, dev[:100], dev[100:], np.ones(128, np.uint64), 100, out[:50])
