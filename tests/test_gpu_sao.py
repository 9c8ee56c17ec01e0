"""GPU parity of the SAO local constraint over a plan's matches
(cm_match_plan_sao) with the host form cm_sao_filter, which the CPU tests pin
bit for bit to the oracle, and directly with the oracle on a small pair:
scores and decisions bit for bit, for several neighbour counts, many matches
(several tiles and chunks), lattice keypoints with exact distance ties (the
FP64 fallback), planted outliers, and in-place operation."""
import numpy as np
import pytest

import paper_2505_22089_b300 as cm
import synth
from oracle import sao as osao

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _case(wl, kp=None):
    desc, kp0 = wl.generate(want_kp=True)
    kp = kp0 if kp is None else kp
    index = cm.Index.build(cm.Params.make(), wl.n_desc, torch.from_numpy(desc).cuda())
    plan = cm.MatchPlan(index, wl.pairs)
    out = plan.alloc_out()
    plan.run(out)
    torch.cuda.synchronize()
    kp_dev = torch.from_numpy(np.ascontiguousarray(kp, dtype=np.float32)).cuda()
    off_dev = torch.from_numpy(wl.row_off.astype(np.int64)).cuda()
    return index, plan, out["best_j"], kp, kp_dev, off_dev


def _lists(plan, best):
    b = best.cpu().numpy()
    res = []
    for k in range(len(plan.pairs)):
        s = b[plan.row_off[k]:plan.row_off[k + 1]]
        q = np.nonzero(s >= 0)[0]
        res.append(((q.astype(np.uint32) << 16) | s[q].astype(np.uint32), q))
    return res


def _check(wl, plan, best, kp, kp_dev, off_dev, k, tau=0.875, in_place=False):
    before = _lists(plan, best)
    if in_place:
        work = best.clone()
        b = cm.ctypes.c_uint64()
        cm.check(cm.lib().cm_match_plan_sao_bytes(plan.h, cm.ctypes.byref(b)))
        ws = torch.empty(int(b.value) + 256, dtype=torch.uint8, device="cuda")
        wb = (ws.data_ptr() + 255) // 256 * 256
        score = torch.empty(best.numel(), dtype=torch.float32, device="cuda")
        cm.check(cm.lib().cm_match_plan_sao(plan.h, cm._ptr(work), cm._ptr(work), cm._ptr(kp_dev), cm._ptr(off_dev), k,
                                            tau, cm._ptr(score), cm.ctypes.c_void_p(wb), int(b.value),
                                            cm._stream(None)))
        out = work
    else:
        out, score = plan.sao(best, kp_dev, off_dev, k, tau, want_score=True)
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    sc = score.cpu().numpy()
    off = wl.row_off
    kept_total = 0
    for kk, (i, j) in enumerate(np.asarray(plan.pairs)):
        mt, q = before[kk]
        s_h, keep_h, n_h = cm.sao_filter(kp[off[i]:off[i + 1]], kp[off[j]:off[j + 1]], mt, k, tau)
        r0 = plan.row_off[kk]
        assert np.array_equal(sc[r0 + q], s_h), (kk, np.nonzero(sc[r0 + q] != s_h)[0][:5])
        assert np.array_equal(o[r0 + q] >= 0, keep_h), kk
        kept_total += n_h
    assert int((o >= 0).sum()) == kept_total
    return kept_total, sum(len(m) for m, _ in before)


@pytest.mark.parametrize("k", [1, 4, 8, 16])
def test_gpu_sao_equals_the_host_form(k):
    wl = synth.strip30(n_images=5, n=2500)
    _, plan, best, kp, kp_dev, off_dev = _case(wl)
    kept, total = _check(wl, plan, best, kp, kp_dev, off_dev, k)
    assert total > 1000


def test_gpu_sao_many_matches_lattice_ties_and_outliers():
    wl = synth.pair2k(n=5000, shared=3500)
    desc, kp = wl.generate(want_kp=True)
    # keypoints on a coarse lattice: exact distance ties everywhere (the FP64 fallback path)
    kp = (np.round(kp / 8.0) * 8.0).astype(np.float32)
    # planted outliers: a fifth of image 1's keypoints moved far away
    rng = np.random.default_rng(5)
    off = wl.row_off
    mv = off[1] + rng.choice(wl.n_desc[1], wl.n_desc[1] // 5, replace=False)
    kp[mv] = rng.uniform(0, 8000, (len(mv), 2)).astype(np.float32)
    _, plan, best, kp, kp_dev, off_dev = _case(wl, kp)
    kept, total = _check(wl, plan, best, kp, kp_dev, off_dev, 8)
    assert total > 2500 and kept < total
    kept2, _ = _check(wl, plan, best, kp, kp_dev, off_dev, 8, in_place=True)
    assert kept2 == kept


def test_gpu_sao_equals_the_oracle_on_a_small_pair():
    wl = synth.pair2k(n=800, shared=500)
    _, plan, best, kp, kp_dev, off_dev = _case(wl)
    mt, q = _lists(plan, best)[0]
    out, score = plan.sao(best, kp_dev, off_dev, 8, 0.875, want_score=True)
    torch.cuda.synchronize()
    off = wl.row_off
    s_o, keep_o = osao.sao_filter(kp[off[0]:off[1]], kp[off[1]:off[2]], mt, 8, 0.875)
    assert np.array_equal(score.cpu().numpy()[q], s_o)
    assert np.array_equal(out.cpu().numpy()[q] >= 0, keep_o)


def test_gpu_sao_arguments():
    wl = synth.pair2k(n=300, shared=100)
    _, plan, best, kp, kp_dev, off_dev = _case(wl)
    for k in (0, 17):
        with pytest.raises(cm.CMError) as e:
            plan.sao(best, kp_dev, off_dev, k)
        assert e.value.status == cm.CM_ERR_INVALID
