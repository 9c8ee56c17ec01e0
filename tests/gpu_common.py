"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI
and the FP64 oracle on the same seeded inputs, then compare."""
from __future__ import annotations

import numpy as np

import oracle
import paper_2505_22089_b300 as cm

U32_MAX = 0xFFFFFFFF


def oparams(p: cm.Params) -> oracle.Params:
    return oracle.Params(L=p.L, m=p.m, nbits=p.n_bits, K=p.K, ratio_num=p.ratio_num, ratio_den=p.ratio_den,
                         seed=p.seed)


def gpu_match(index: cm.Index, pairs, topk: bool = True):
    import torch
    plan = cm.MatchPlan(index, pairs)
    out = plan.alloc_out(topk=topk)
    plan.run(out)
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    for k in ("d1sq", "d2sq"):
        res[k] = res[k].view(np.uint32)
    if topk:
        res["topk"] = res["topk"][: plan.rows * plan.K].reshape(-1, plan.K)
    return plan, res


def bit_diff(gv: dict, oi: oracle.HashedImage, p: cm.Params):
    """Differing key/code bits between the GPU and the oracle for one image,
    and whether each differing bit is marginal (|s| < 1e-4 ||x~||)."""
    n = oi.n
    L, m = p.L, p.m
    diff = np.zeros((n, L * m + 128), dtype=bool)
    for t in range(L):
        x = gv["keys"][:, t] ^ oi.keys[:, t]
        for b in range(m):
            diff[:, t * m + b] = (x >> b) & 1
    cb = np.unpackbits((gv["code"] ^ oi.code).view(np.uint8), axis=1, bitorder="little").astype(bool)
    diff[:, L * m:] = cb
    return diff


def compare_hash(index: cm.Index, oix: oracle.Index, images, p: cm.Params):
    """Checks keys, codes and bucket tables of `images`.  Returns
    (affected descriptors per image, n differing bits, n marginal bits, n bits).
    Affected entries: image -> (indices, differing code bits, GPU keys)."""
    affected = {}
    n_diff = n_marg = n_bits = 0
    for i in images:
        gv = index.image_view(i)
        oi = oix.image(i, marginal=True)
        d = bit_diff(gv, oi, p)
        n_diff += int(d.sum())
        n_marg += int(oi.marginal.sum())
        n_bits += d.size
        assert not np.any(d & (oi.marginal == 0)), "a non-marginal bit differs in image %d" % i
        idx = np.nonzero(d.any(1))[0]
        affected[i] = (idx, d[idx, p.L * p.m:].sum(1), gv["keys"][idx])
        # bucket tables: exact when the image's keys agree
        if not d[:, : p.L * p.m].any():
            assert np.array_equal(gv["off"].astype(np.int64), oi.off.astype(np.int64))
            assert np.array_equal(gv["sidx"].astype(np.int64), oi.idx.astype(np.int64))
        # sorted codes are the image's own codes in bucket order
        for t in range(p.L):
            assert np.array_equal(gv["scode"][t], gv["code"][gv["sidx"][t].astype(np.int64)])
    return affected, n_diff, n_marg, n_bits


def _ham(a, b):
    return np.unpackbits((a ^ b).view(np.uint8), axis=-1).sum(-1)


def affected_queries(p, oix: oracle.Index, i: int, j: int, affected: dict, o_topk: np.ndarray) -> np.ndarray:
    """Queries of pair (i, j) excluded from the exact checks.

    A query is excluded when one of its own bits differs, or when a database
    point j* with d* differing code bits (or differing keys) could reach its
    top-K under either hash: j* shares a bucket with the query under the
    oracle's or the GPU's keys and its oracle Hamming distance is within d* of
    the query's K-th ranked candidate (or the list is not full)."""
    I, J = oix.image(i), oix.image(j)
    bad = np.zeros(I.n, dtype=bool)
    own = affected.get(i)
    if own is not None:
        bad[own[0]] = True
    aj = affected.get(j)
    if aj is None or not len(aj[0]):
        return bad
    K = p.K
    full = o_topk[:, K - 1] >= 0
    kth = np.full(I.n, 10 ** 6, dtype=np.int64)
    if full.any():
        kj = o_topk[full, K - 1]
        kth[full] = _ham(I.code[full], J.code[kj])
    for js, dcode, gkeys in zip(*aj):
        share = np.zeros(I.n, dtype=bool)
        for t in range(p.L):
            share |= (I.keys[:, t] == J.keys[js, t]) | (I.keys[:, t] == gkeys[t])
        h = _ham(I.code, J.code[js][None, :])
        bad |= share & (h <= kth + int(dcode) + 1)
    return bad


def compare_match(plan, res, oix: oracle.Index, pairs, p: cm.Params, affected: dict, check_topk: bool = True):
    """Exact comparison of per-query outputs on unaffected queries; returns
    (rows compared, rows excluded, Jaccard agreement of match sets)."""
    op = oparams(p)
    rows = excl = 0
    inter = union = 0
    for k, (i, j) in enumerate(np.asarray(pairs).reshape(-1, 2)):
        r0, r1 = plan.row_off[k], plan.row_off[k + 1]
        o = oracle.match_pair(oix.image(i), oix.image(j), op, topk=True)
        bad = affected_queries(p, oix, i, j, affected, o["topk"])
        ok = ~bad
        g_best = res["best_j"][r0:r1]
        assert np.array_equal(g_best[ok], o["best_j"][ok]), "pair %d (%d,%d): best_j differs" % (k, i, j)
        assert np.array_equal(res["d1sq"][r0:r1][ok], o["d1sq"][ok]), "pair %d: d1sq differs" % k
        assert np.array_equal(res["d2sq"][r0:r1][ok], o["d2sq"][ok]), "pair %d: d2sq differs" % k
        if check_topk and "topk" in res:
            assert np.array_equal(res["topk"][r0:r1][ok], o["topk"][ok]), "pair %d: top-K lists differ" % k
        rows += int(ok.sum())
        excl += int(bad.sum())
        gm = set(zip(np.nonzero(g_best >= 0)[0].tolist(), g_best[g_best >= 0].tolist()))
        om = set(zip(np.nonzero(o["best_j"] >= 0)[0].tolist(), o["best_j"][o["best_j"] >= 0].tolist()))
        inter += len(gm & om)
        union += len(gm | om)
    return rows, excl, (inter / union if union else 1.0)
