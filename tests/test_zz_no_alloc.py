"""cm_match_pair_noalloc: matching for callers that may not allocate GPU memory.

Such callers (code inside another framework's memory budget, plug-ins of a
process that owns the device, real-time paths where an allocation could block
or fail) pass only inputs and outputs; the library's scratch is a fixed 5 MiB
device array.  This file is collected last so that a run stopping at the
first failure has already run every other test."""
import numpy as np
import pytest

import paper_2505_22089_b300 as cm
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _reference(p, wl, dev, pairs):
    index = cm.Index.build(p, wl.n_desc, dev)
    plan = cm.MatchPlan(index, pairs)
    out = plan.alloc_out()
    plan.run(out)
    torch.cuda.synchronize()
    sums, n_total = index.col_sums()
    res = {k: out[k].cpu().numpy().view(np.uint32 if k != "best_j" else np.int32) for k in ("best_j", "d1sq", "d2sq")}
    return res, plan.row_off, sums, n_total


@pytest.mark.parametrize("rerank", ["fp32", "int"])
def test_noalloc_equals_index_path_on_two_calls_in_a_row(rerank):
    wl = synth.strip30(n_images=4, n=3000)
    wl.images["n"][3] = 8192                      # the largest image the scratch holds
    desc = wl.generate()
    dev = torch.from_numpy(desc).cuda()
    off = wl.row_off
    p = cm.Params.make(rerank=rerank)
    pairs = [(0, 1), (3, 2)]
    ref, row_off, sums, n_total = _reference(p, wl, dev, pairs)
    for k, (i, j) in enumerate(pairs):            # two calls in a row share the scratch
        n_i = int(wl.n_desc[i])
        best = torch.full((n_i,), -7, dtype=torch.int32, device="cuda")
        d1 = torch.zeros(n_i, dtype=torch.int32, device="cuda")
        d2 = torch.zeros(n_i, dtype=torch.int32, device="cuda")
        cm.match_pair_noalloc(p, dev[off[i]:off[i + 1]], dev[off[j]:off[j + 1]], sums, n_total, best, d1, d2)
        torch.cuda.synchronize()
        r0, r1 = row_off[k], row_off[k + 1]
        assert np.array_equal(best.cpu().numpy(), ref["best_j"][r0:r1])
        assert np.array_equal(d1.cpu().numpy().view(np.uint32), ref["d1sq"][r0:r1])
        assert np.array_equal(d2.cpu().numpy().view(np.uint32), ref["d2sq"][r0:r1])
        assert (best >= 0).sum().item() > 0


def test_noalloc_rejects_images_over_the_limit():
    wl = synth.pair2k(n=100, shared=10)
    dev = torch.from_numpy(wl.generate()).cuda()
    big = torch.zeros((8193, 128), dtype=torch.uint8, device="cuda")
    out = torch.empty(8193, dtype=torch.int32, device="cuda")
    p = cm.Params.make()
    with pytest.raises(cm.CMError) as e:
        cm.match_pair_noalloc(p, big, dev[:100], np.ones(128, np.uint64), 100, out)
    assert e.value.status == cm.CM_ERR_BUDGET and "8192" in str(e.value)
