#!/usr/bin/env python3
"""Throughput of cascade-hashing feature matching on one B300: pairs matched/s.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload grid5000]
                    [--rerank bf16|fp8|fp32|int] [--impl ours|reference]

A step is one pass of the whole hot path over the workload's MBR block rows:
centring statistics, projection to bucket keys and codes, bucket
construction, then per block row one persistent fused match launch (lookup,
Hamming top-K, rerank, ratio test) and the compaction of its decisions into
per-pair match lists.  `value` replays that step as one captured CUDA graph
with the descriptors already resident in HBM (headline rerank form; the other
forms are timed the same way under "forms").  `e2e` runs the public pipeline
call with the descriptors in pinned host memory: H2D, matching and the D2H of
the match lists are inside its timed region.  "pipeline_verified" repeats it
with outlier removal overlapped with the GPU rows: affine RANSAC alone on the
host cores, the SAO local constraint ahead of it on the host, and SAO on the
GPU (per block row, before the matches reach the host) ahead of it.

The workloads are synthetic stand-ins for the paper's UAV datasets (see
synth/).  `--impl reference` times the FP64 CPU oracle on the host cores on a
bounded sample of the same workload.  Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "pairs matched/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
SM_COUNT = 148


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="grid5000", choices=sorted(synth.WORKLOADS))
    ap.add_argument("--rerank", default="bf16", choices=["fp32", "int", "bf16", "fp8"], help="headline form")
    ap.add_argument("--forms", default="all", choices=["all", "one"], help="also time the other rerank forms")
    ap.add_argument("--vlad-codewords", type=int, default=128,
                    help="codebook size of the VLAD encoding timed beside the matching (0: skip)")
    ap.add_argument("--K", type=int, default=8)
    ap.add_argument("--tune-pairs", type=int, default=1800,
                    help="pairs of the first block row the autotuner times (0: no tuning); the bucket-major "
                         "form runs one pair per CTA, so a fair sample holds a few pairs per CTA")
    ap.add_argument("--verify-workers", type=int, default=-1,
                    help="CPU threads of the overlapped RANSAC run (-1: all host cores, 0: skip)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--algo", default="auto", choices=["auto", "bucket", "tile", "warp", "tc"],
                    help="match kernel thread mapping")
    ap.add_argument("--projection", default="tc", choices=["tc", "ffma"], help="hash projection: tensor cores or FP32 FFMA")
    ap.add_argument("--block-images", type=int, default=400, help="Size_blk: images per schedule chunk")
    ap.add_argument("--budget-gb", type=float, default=150.0, help="HBM budget of the MBR schedule")
    ap.add_argument("--plain-pairs", type=int, default=200, help="pairs timed in the plain per-pair form")
    ap.add_argument("--oracle-pairs", type=int, default=12,
                    help="pairs per step of the reference arm's oracle sample")
    ap.add_argument("--oracle-frac", type=float, default=0.02,
                    help="share of the pairs the FP64 oracle checks in full (at least --oracle-min-pairs); 0: skip")
    ap.add_argument("--oracle-min-pairs", type=int, default=1000)
    ap.add_argument("--configs", default="all", choices=["all", "none"],
                    help="also measure the four smaller workloads (pair2k, strip30, grid500, oblique200)")
    ap.add_argument("--config-oracle-pairs", type=int, default=300,
                    help="pairs the oracle checks in full per smaller workload (all pairs when fewer)")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--nn-pairs", type=int, default=64,
                    help="sampled pairs matched exhaustively on the tensor cores (recall ceiling, L/K sweep); 0: skip")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--strategy-runs", type=int, default=1, choices=[0, 1],
                    help="0: count the schedule strategies without running them (shorter profiling runs)")
    ap.add_argument("--grid", default=None, help="GXxGY: a smaller grid of the same per-image shape (profiling)")
    ap.add_argument("--multi", default="shard", choices=["shard", "replicas"],
                    help="N > 1: one job sharded over the ranks (strong scaling), or an independent job per rank")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t0 = time.time()
            while not self.rows and time.time() - t0 < 5.0 and self.proc.poll() is None:
                time.sleep(0.05)
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(r[1]) for r in self.rows if len(r) > 8 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 8 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for k, n in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


# DRAM traffic of the lookup kernel k_match_bm, from ncu (dram__bytes_read.sum +
# dram__bytes_write.sum) on a small case of the same per-image shape: the 200-image grid of the
# grid5000 workload, one block row of 2,104 pairs, mean of 3 launches.  A pair's traffic (its two
# images' tables, its lists and hand-over) does not depend on how many pairs share the launch, so
# the figure is stated per pair and scaled by the pairs of a launch.  It is reported only for the
# form it was taken on and only while the kernel's sources are unchanged (their SHA-256 below);
# otherwise the roofline's "traffic" is null.
KMATCH_TRAFFIC = {"workload": "grid5000", "rerank": "bf16", "K": 8, "bytes_per_pair": 13073947,
                  "sources_sha256": "5e9009d04827065cee63da5d098b700e8afe64ad5b36801e6454bb70dee12408"}
KMATCH_SOURCES = ["paper_2505_22089_b300/csrc/cm_match_bm.cu", "paper_2505_22089_b300/csrc/cm_internal.h",
                  "paper_2505_22089_b300/csrc/cm_ratio.cuh", "paper_2505_22089_b300/csrc/cm_tc.cuh"]


def kmatch_sources_sha256() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KMATCH_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def kmatch_traffic(args, pairs_per_launch):
    t = KMATCH_TRAFFIC
    if (t["bytes_per_pair"] is None or args.workload != t["workload"] or args.rerank != t["rerank"]
            or args.K != t["K"] or kmatch_sources_sha256() != t["sources_sha256"]):
        return None
    return t["bytes_per_pair"] * pairs_per_launch


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2032.0}, "fallback"


def bucket_evaluations(index, wl, pairs):
    """Candidate evaluations the lookup makes: sum over pairs, tables and
    buckets of n_I(t,b) * n_J(t,b) (a query meets every point of its bucket)."""
    import paper_2505_22089_b300 as cm
    L, B = index.p.L, 1 << index.p.m
    cnt = {}
    for i in sorted(set(pairs.reshape(-1).tolist())):
        import ctypes
        ptrs = [ctypes.c_void_p() for _ in range(5)]
        cm.check(cm.lib().cm_index_image_view(index.h, int(i), *[ctypes.byref(x) for x in ptrs]))
        off = cm.device_to_numpy(ptrs[4].value, (L, B + 1), np.uint32).astype(np.int64)
        cnt[i] = np.diff(off, axis=1)
    return int(sum((cnt[int(i)] * cnt[int(j)]).sum() for i, j in pairs))


def make_workload(args):
    kw = dict(getattr(args, "workload_kw", None) or {})   # image sizes of a small test job
    if args.grid:
        gx, gy = (int(v) for v in args.grid.lower().split("x"))
        return synth.WORKLOADS[args.workload](gx=gx, gy=gy, **kw)
    return synth.WORKLOADS[args.workload](**kw) if kw else synth.workload(args.workload)


def _sync_ms(ms, world, dev):
    """Max over ranks of a per-rank time (weak scaling: the job ends with the slowest rank)."""
    if world <= 1:
        return ms
    import torch
    t = torch.tensor([ms], device=dev)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


U32_MAX = 0xFFFFFFFF


def pick_sample(pairs, frac, min_pairs, seed=0):
    """A seeded sample of pair ids for the full oracle check (frac of the pairs,
    at least min_pairs), the images it names, and every pair both of whose
    images are among them (their near-threshold queries are checked too)."""
    P = len(pairs)
    n = min(P, max(int(min_pairs), int(np.ceil(frac * P))))
    sel = np.sort(np.random.default_rng(seed).choice(P, n, replace=False)) if n else np.zeros(0, np.int64)
    imgs = np.unique(pairs[sel]) if n else np.zeros(0, np.int64)
    elig = np.nonzero(np.isin(pairs[:, 0], imgs) & np.isin(pairs[:, 1], imgs))[0]
    return sel, imgs, elig


def gpu_outputs(plans, outs, rows, sel, elig, ratio, index, imgs, extra=()):
    """Host copies of what the oracle check needs from one pass's device
    outputs (outs with best_j, d1sq, d2sq): every row of the sampled pairs (and
    of `extra` pairs), the near-threshold rows of the eligible pairs
    (|sqrt(d1/d2) - t_r| < 1e-3 by the GPU's own distances), and the keys and
    codes of the sampled images."""
    import torch
    where = {}
    for r, rr in enumerate(rows):
        for q, k in enumerate(rr):
            where[int(k)] = (r, q)

    def rows_of(k):
        r, q = where[k]
        a, b = plans[r].row_off[q], plans[r].row_off[q + 1]
        o = outs[r]
        return (o["best_j"][a:b].cpu().numpy(), o["d1sq"][a:b].cpu().numpy().view(np.uint32),
                o["d2sq"][a:b].cpu().numpy().view(np.uint32))

    full = {int(k): rows_of(int(k)) for k in set(sel.tolist()) | set(int(x) for x in extra)}
    t = ratio[0] / ratio[1]
    elig_set = set(elig.tolist())
    near = {}
    for r, (pl, o) in enumerate(zip(plans, outs)):
        if not pl.rows or not elig_set:
            continue
        d1 = (o["d1sq"][:pl.rows].to(torch.int64) & U32_MAX).double()
        d2 = (o["d2sq"][:pl.rows].to(torch.int64) & U32_MAX).double()
        m = (d2 < float(U32_MAX)) & (d2 > 0) & ((torch.sqrt(d1 / d2.clamp(min=1.0)) - t).abs() < 1e-3)
        idx = torch.nonzero(m).flatten()
        del d1, d2, m
        if not idx.numel():
            continue
        b = o["best_j"][idx].cpu().numpy()
        e1 = o["d1sq"][idx].cpu().numpy().view(np.uint32)
        e2 = o["d2sq"][idx].cpu().numpy().view(np.uint32)
        idx = idx.cpu().numpy()
        q = np.searchsorted(pl.row_off, idx, side="right") - 1
        for qq in np.unique(q):
            k = int(rows[r][qq])
            if k not in elig_set:
                continue
            sel_q = q == qq
            near[k] = (idx[sel_q] - pl.row_off[qq], b[sel_q], e1[sel_q], e2[sel_q])
    bits = {int(i): index.image_bits(int(i)) for i in imgs}
    return {"full": full, "near": near, "bits": bits}


def _oparams(p):
    import oracle
    return oracle.Params(L=p.L, m=p.m, nbits=p.n_bits, K=p.K, ratio_num=p.ratio_num, ratio_den=p.ratio_den,
                         seed=p.seed)


def _match_set(best):
    q = np.nonzero(best >= 0)[0]
    return set(zip(q.tolist(), best[q].tolist()))


def oracle_check(wl, desc, p, pairs, sel, imgs, elig, got, gpu_sums, form, marginal_images=32, one_core=True,
                 cache=None):
    """The FP64 oracle against the GPU's outputs, with the oracle's own
    centring sums: (1) the sums themselves; (2) every key / code bit of the
    sampled images (differing bits must be marginal: |s| < 1e-4 |x - mu|;
    the marginal share is counted on a subset of them); (3) every query of the
    sampled pairs: decision, match-set Jaccard, exact d^2; (4) every
    near-threshold query of the pairs whose two images the sample hashed, one
    query at a time.  Also times the oracle as it stands (all host cores, and
    one core) for the CPU baseline."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    cores = os.cpu_count() or 1
    op = _oparams(p)
    if cache is not None and cache.get("key") == (op, tuple(sel.tolist())):
        oix, res, t_sums, t_match = cache["val"]                  # the same workload checked for another form
    else:
        t0 = time.perf_counter()
        oix = oracle.Index(desc, wl.n_desc, op, threads=cores)     # its own sums over every row
        t_sums = time.perf_counter() - t0
        t0 = time.perf_counter()
        res = oix.match(pairs[sel])                               # hashes the sampled images, then matches
        t_match = time.perf_counter() - t0
        if cache is not None:
            cache["key"], cache["val"] = (op, tuple(sel.tolist())), (oix, res, t_sums, t_match)
    out = {"form": form, "oracle_sums_equal_gpu": bool(np.array_equal(oix.sums, gpu_sums)),
           "oracle_sums": "computed by the oracle from the raw rows (not the GPU's)"}
    # (2) bits
    n_bits = n_diff = n_diff_nonmarg = 0
    L, m = p.L, p.m
    diff_imgs = []
    for i in imgs:
        gk, gc = got["bits"][int(i)]
        oi = oix.image(int(i))
        kd = np.unpackbits((gk ^ oi.keys).reshape(-1, L, 1), axis=2, bitorder="little")[:, :, :m].reshape(len(gk), -1)
        cd = np.unpackbits((gc ^ oi.code).view(np.uint8), axis=1, bitorder="little")
        d = np.concatenate([kd, cd], axis=1).astype(bool)
        n_bits += d.size
        if d.any():
            n_diff += int(d.sum())
            diff_imgs.append((int(i), d))
    def marginal_of(i):
        return oracle.hash_image(oix.image_desc(int(i)), oix.mu, oix.W, op, marginal=True).marginal

    with ThreadPoolExecutor(cores) as ex:                         # differing bits must be marginal ones
        for (i, d), mg in zip(diff_imgs, ex.map(marginal_of, [i for i, _ in diff_imgs])):
            n_diff_nonmarg += int((d & (mg == 0)).sum())
        n_mb = n_marg = 0
        for mg in ex.map(marginal_of, list(imgs[:marginal_images])):
            n_marg += int(mg.sum())
            n_mb += int(mg.size)
    out["bits"] = {"images": int(len(imgs)), "bits": n_bits, "differing": n_diff,
                   "differing_share": n_diff / max(n_bits, 1), "differing_not_marginal": n_diff_nonmarg,
                   "marginal_share": n_marg / max(n_mb, 1), "marginal_counted_on_images": int(min(len(imgs),
                                                                                           marginal_images)),
                   "marginal": "|s| < 1e-4 |x - mu| (FP64); must stay under 0.01 % of bits"}
    # (3) sampled pairs in full
    same = total = inter = union = ng = no = 0
    d_cmp = d_err = d2_diff = 0
    for k, o in zip(sel, res):
        g, g1, g2 = got["full"][int(k)]
        same += int((g == o["best_j"]).sum())
        total += len(g)
        gm, om = _match_set(g), _match_set(o["best_j"])
        inter += len(gm & om)
        union += len(gm | om)
        ng += len(gm)
        no += len(om)
        both = (g == o["best_j"]) & (g >= 0)
        d_cmp += int(both.sum())
        d_err = max(d_err, float(np.max(np.abs(g1[both].astype(np.float64) - o["d1sq"][both]) /
                                         np.maximum(o["d1sq"][both], 1), initial=0.0)))
        d2_diff += int((g2[both] != o["d2sq"][both]).sum())
    out["sample"] = {"pairs": int(len(sel)), "of_pairs": int(len(pairs)), "share": len(sel) / max(len(pairs), 1),
                     "seed": 0, "queries": total, "per_query_agreement": same / max(total, 1),
                     "match_set_jaccard": inter / union if union else 1.0, "gpu_matches": ng, "oracle_matches": no,
                     "d1_max_rel_err": d_err, "d_compared": d_cmp, "d2_differs": d2_diff,
                     "d_note": "queries whose decision agrees with a match: d1^2 (the match's exact squared "
                               "distance) against the oracle's; d2_differs counts those whose second candidate "
                               "differs (a marginal code bit moved it in or out of the top K)"}
    # (4) near-threshold queries, one by one
    jobs = [(k, v) for k, v in got["near"].items()]

    def check_near(job):
        k, (qs, b, e1, e2) = job
        i, j = (int(x) for x in pairs[k])
        I, J = oix.image(i), oix.image(j)
        agree = dd = 0
        for q, bb, a1, a2 in zip(qs, b, e1, e2):
            o = oracle.match_pair(I, J, op, q0=int(q), q1=int(q) + 1)
            agree += int(o["best_j"][0] == bb)
            dd += int(o["d1sq"][0] == a1 and o["d2sq"][0] == a2)
        return agree, dd, len(qs)

    t0 = time.perf_counter()
    with ThreadPoolExecutor(cores) as ex:
        rr = list(ex.map(check_near, jobs))
    a = sum(x[0] for x in rr)
    dd = sum(x[1] for x in rr)
    nq = sum(x[2] for x in rr)
    out["near_threshold"] = {"definition": "|sqrt(d1/d2) - t_r| < 1e-3 by the GPU's d1, d2",
                             "pairs_scanned": int(len(elig)), "pairs_with_such_queries": len(jobs), "queries": nq,
                             "decision_agreement": a / max(nq, 1), "distances_equal": dd / max(nq, 1),
                             "oracle_s": round(time.perf_counter() - t0, 2)}
    per_pair = (t_match + t_sums * len(sel) / max(len(pairs), 1)) / max(len(sel), 1)
    out["oracle_time_s"] = {"sums_all_rows": round(t_sums, 2), "hash_and_match_sample": round(t_match, 2)}
    base = {"value": 1.0 / per_pair, "unit": "pairs/s", "cores": cores, "kind": "oracle",
            "sample": "%d of %d pairs (seeded), FP64 oracle as it stands on %d host threads: its own column sums "
                      "over all %d rows (time pro-rated per pair), hashing of the %d images the sample names, "
                      "matching" % (len(sel), len(pairs), cores, wl.total_desc, len(imgs))}
    if one_core and len(sel):
        k = int(sel[0])
        i, j = (int(x) for x in pairs[k])
        t0 = time.perf_counter()
        I1 = oracle.hash_image(oix.image_desc(i), oix.mu, oix.W, op)
        J1 = oracle.hash_image(oix.image_desc(j), oix.mu, oix.W, op)
        oracle.match_pair(I1, J1, op)
        t1c = time.perf_counter() - t0
        base["one_core"] = {"value": 1.0 / (t1c + t_sums * cores / max(len(pairs), 1)), "unit": "pairs/s",
                            "sample": "pair %d: hash both images + match on one thread; the sums pass pro-rated "
                                      "per pair at %d x its all-core time" % (k, cores)}
    return out, base


def device_forms(args, wl, desc_dev, rows, stream, dev, world, forms, check=None, extra=()):
    """Device-resident steps, one per rerank form: descriptors already in HBM;
    a step = the captured block sequence (rehash of every resident image, then
    per block row one fused match launch and its compaction) replayed as one
    CUDA graph.  The headline form (first) is also run once more per step
    without the graph with CUDA events around each match launch, which gives
    the k_match launch duration behind the roofline figure."""
    import torch
    import paper_2505_22089_b300 as cm
    pairs = wl.pairs
    res = {}
    ref_best = None
    headline = forms[0]
    for form in forms:
        p = cm.Params.make(rerank=form, algo=args.algo, projection=args.projection, K=args.K)
        sample = pairs[rows[0][:args.tune_pairs]] if args.tune_pairs > 0 else None
        # plans take the most any thread mapping the tuner may choose needs (the tile form's
        # hand-over to the tensor-core rerank is larger than the bucket-major form's key lists)
        tuned_algos = ("bucket", "tile") + (() if form in ("bf16", "fp8") else ("warp",))   # those the tuner tries
        mappings = [p] + ([cm.Params.make(rerank=form, algo=a, projection=args.projection, K=args.K)
                           for a in tuned_algos] if sample is not None and args.algo == "auto" else [])
        arena = (cm.index_bytes(p, wl.n_desc, inplace=True) + cm.PLAN_HEADROOM +
                 sum(max(cm.pairs_plan_bytes(q, wl.n_desc, pairs[r]) for q in mappings) for r in rows))
        if sample is not None:   # the tuner's plan and decision scratch
            arena += cm.pairs_plan_bytes(p, wl.n_desc, sample) + 4 * int(wl.n_desc[sample[:, 0]].sum()) + (1 << 20)
        tuned = None
        with torch.cuda.stream(stream):
            index = cm.Index.build(p, wl.n_desc, desc_dev, stream=stream, arena_bytes=arena)
            if sample is not None and args.algo == "auto":
                tuned = index.autotune(sample, stream=stream)   # work-item size and thread mapping
            plans = [cm.MatchPlan(index, pairs[r], stream=stream) for r in rows]
            outs = [pl.alloc_out(d12=False) for pl in plans]
            comps = [cm.compact_out(pl) for pl in plans]
        stream.synchronize()
        seq = cm.Sequence(index, plans, outs, comps, rehash=True, stream=stream)
        for _ in range(args.warmup):
            seq.launch(stream)
        stream.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(torch.cuda.current_device()) as clk:
            start.record(stream)
            for _ in range(args.steps):
                seq.launch(stream)
            stop.record(stream)
            stop.synchronize()
        torch.cuda.synchronize()
        ms = _sync_ms(start.elapsed_time(stop) / args.steps, world, dev)
        index.check(stream)
        r = {"ms_per_step": ms, "value": len(pairs) * world / (ms / 1e3), "graph_kernels": seq.kernels,
             "clocks": clk.summary(), "tuned": tuned}
        best = torch.cat([o["best_j"][:pl.rows] for pl, o in zip(plans, outs)])
        n_match = int(sum(int(c["total"].item()) for c in comps))
        r["matches"] = n_match
        assert n_match == int((best >= 0).sum().item())
        if form == "fp32":
            ref_best = best
        elif ref_best is not None:
            same = int((best == ref_best).sum().item())
            inter = int(((best == ref_best) & (best >= 0)).sum().item())
            union = int((best >= 0).sum().item()) + int((ref_best >= 0).sum().item()) - inter
            r["decision_agreement_vs_fp32"] = same / best.numel()
            r["match_jaccard_vs_fp32"] = inter / union if union else 1.0
        if form == headline:
            # the same launches without the graph, events around every match launch
            # (the middle event is recorded by the library after the lookup launch);
            # these outputs also carry d1^2, d2^2 and the counters of the last step
            outs_d = [dict(o, d1sq=torch.empty_like(o["best_j"]), d2sq=torch.empty_like(o["best_j"])) for o in outs]
            evs = [[[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in plans]
                   for _ in range(args.steps)]
            for s in range(args.steps):
                if s == args.steps - 1:
                    for o in outs_d:
                        o["stats"].zero_()
                index.rehash(stream)
                for k, (pl, o) in enumerate(zip(plans, outs_d)):
                    evs[s][k][0].record(stream)
                    pl.run(o, stream, scan_done=evs[s][k][1])
                    evs[s][k][2].record(stream)
            stream.synchronize()
            st = torch.stack([o["stats"] for o in outs_d]).sum(0).cpu().numpy()
            r["fp64_rechecks_per_step"] = int(st[0])
            r["fp8_top2_swaps_per_step"] = int(st[2])
            launch_ms = [e[k][0].elapsed_time(e[k][2]) for e in evs for k in range(len(plans))]
            scan_ms = [e[k][0].elapsed_time(e[k][1]) for e in evs for k in range(len(plans))]
            r["match_launch_ms"] = float(np.mean(launch_ms))
            r["scan_launch_ms"] = float(np.mean(scan_ms))
            r["match_ms_per_step"] = float(np.sum(launch_ms)) / args.steps
            r["evals_per_step"] = bucket_evaluations(index, wl, pairs)
            r["launches"] = len(plans)
            r["_p"] = cm.Params.from_buffer_copy(index.p)
            r["_sums"] = index.col_sums(stream)[0]
            if check is not None:
                sel, imgs, elig = check
                r["_got"] = gpu_outputs(plans, outs_d, rows, sel, elig, (p.ratio_num, p.ratio_den), index, imgs,
                                        extra)
            del outs_d
        res[form] = r
        seq.close()
        for pl in plans:
            pl.close()
        index.close()
        del seq, plans, outs, comps, index, best
        torch.cuda.empty_cache()
    return res


# The smaller workloads measured next to the headline one: (line, workload, rerank form, HBM budget in GB,
# Size_blk).  grid500 runs once as one block and once cut into blocks of at most 100 images.
CONFIG_RUNS = [("pair2k", "pair2k", "fp32", 150.0, 400), ("strip30", "strip30", "fp32", 150.0, 400),
               ("grid500", "grid500", "fp32", 40.0, 400), ("grid500_blk100", "grid500", "fp32", 40.0, 100),
               ("oblique200_bf16", "oblique200", "bf16", 150.0, 400),
               ("oblique200_fp8", "oblique200", "fp8", 150.0, 400)]


def config_lines(args, stream, dev):
    """Per workload: pairs/s of the device-resident step (one CUDA graph:
    rehash, per block row one match launch and its compaction, as for the
    headline workload), then the FP64 oracle (own sums) on every pair, or on
    a seeded sample of --config-oracle-pairs pairs plus the near-threshold
    queries of the pairs among the sampled images."""
    import torch
    import paper_2505_22089_b300 as cm
    out = {}
    descs, caches = {}, {}
    for key, wname, form, budget_gb, size_blk in CONFIG_RUNS:
        wl = synth.workload(wname)
        if wname not in descs:
            descs[wname] = wl.generate()
        desc = descs[wname]
        pairs = wl.pairs
        p = cm.Params.make(rerank=form)
        sched = cm.schedule_blocks(pairs, wl.n_desc, p, int(budget_gb * 2 ** 30), size_blk)
        rows = [np.asarray(r["pairs"], dtype=np.int64) for r in sched.rows if r["pairs"]]
        n_rows, n_iter = len(sched.rows), sched.iterations
        sched.close()
        desc_dev = torch.from_numpy(desc).to(dev)
        arena = (cm.index_bytes(p, wl.n_desc, inplace=True) + cm.PLAN_HEADROOM +
                 sum(cm.pairs_plan_bytes(p, wl.n_desc, pairs[r]) for r in rows))
        with torch.cuda.stream(stream):
            index = cm.Index.build(p, wl.n_desc, desc_dev, stream=stream, arena_bytes=arena)
            plans = [cm.MatchPlan(index, pairs[r], stream=stream) for r in rows]
            outs = [pl.alloc_out() for pl in plans]
            comps = [cm.compact_out(pl) for pl in plans]
        stream.synchronize()
        seq = cm.Sequence(index, plans, outs, comps, rehash=True, stream=stream)
        for _ in range(args.warmup):
            seq.launch(stream)
        start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(torch.cuda.current_device()) as clk:
            start.record(stream)
            for _ in range(args.steps):
                seq.launch(stream)
            stop.record(stream)
            stop.synchronize()
        ms = start.elapsed_time(stop) / args.steps
        for o in outs:
            o["stats"].zero_()
        seq.launch(stream)
        stream.synchronize()
        index.check(stream)
        st = torch.stack([o["stats"] for o in outs]).sum(0).cpu().numpy()
        P = len(pairs)
        n_s = min(P, args.config_oracle_pairs)
        sel, imgs, elig = pick_sample(pairs, n_s / P, n_s)
        got = gpu_outputs(plans, outs, rows, sel, elig, (p.ratio_num, p.ratio_den), index, imgs)
        sums = index.col_sums(stream)[0]
        seq.close()
        for pl in plans:
            pl.close()
        index.close()
        del seq, plans, outs, comps, index, desc_dev
        torch.cuda.empty_cache()
        chk, base = oracle_check(wl, desc, p, pairs, sel, imgs, elig, got, sums, form, one_core=False,
                                 cache=caches.setdefault(wname, {}))
        out[key] = {"workload": wname, "images": wl.n_images, "pairs": P, "descriptors": wl.total_desc,
                    "rerank": form, "budget_gb": budget_gb, "size_blk": size_blk, "block_rows": n_rows,
                    "gps_iterations": n_iter, "match_launches": len(rows), "ms_per_step": ms,
                    "value": P / (ms / 1e3), "unit": "pairs/s", "clocks": clk.summary(),
                    "fp64_rechecks_per_step": int(st[0]), "fp8_top2_swaps_per_step": int(st[2]),
                    "oracle": chk, "cpu_oracle_pairs_per_s": base["value"],
                    "step": "one CUDA graph: rehash + per block row match + compaction, descriptors resident"}
    return out


def vlad_encoding(args, wl, desc_dev, host, stream, world, dev):
    """VLAD encoding of every image of the workload (the retrieval front end,
    Sec. 2.1) with the descriptors resident: cm_vlad_encode timed with CUDA
    events over the steps, its two kernels' bounds stated, and the FP64 oracle
    timed on one image for the CPU figure."""
    import torch
    import paper_2505_22089_b300 as cm
    from oracle import vlad as ovlad
    C = args.vlad_codewords
    rng = np.random.default_rng(77)
    cb_host = host[np.sort(rng.choice(len(host), C, replace=False))].copy()   # stand-in for k-means centroids
    cb = torch.from_numpy(cb_host).to(dev)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            v, _ = cm.vlad_encode(desc_dev, wl.n_desc, cb, stream=stream, check_status=False)
        stream.synchronize()
        start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        start.record(stream)
        for _ in range(args.steps):
            v, _ = cm.vlad_encode(desc_dev, wl.n_desc, cb, stream=stream, check_status=False)
        stop.record(stream)
        stop.synchronize()
    ms = _sync_ms(start.elapsed_time(stop) / args.steps, world, dev)
    n = int(wl.total_desc)
    NC = (C + 15) // 16 * 16
    flops = 2.0 * 128 * NC * n
    hbm = 2 * (128 + 2) * n + 4 * C * 128 * wl.n_images      # both kernels read the rows and the assignments
    norms = v.norm(dim=1).cpu().numpy()
    t0 = time.perf_counter()
    i0 = int(np.argmax(wl.n_desc > 0))
    off = wl.row_off
    ovlad.encode(host[off[i0]:off[i0 + 1]], [wl.n_desc[i0]], cb_host)
    cpu_s = time.perf_counter() - t0
    return {"codewords": C, "images": wl.n_images, "descriptors": n, "ms_per_step": ms,
            "images_per_s": wl.n_images * world / (ms / 1e3), "descriptors_per_s": n * world / (ms / 1e3),
            "tensor_tflops_if_assign_alone": flops / (ms / 1e3) / 1e12,
            "hbm_gbs_if_streaming_alone": hbm / (ms / 1e3) / 1e9,
            "algorithmic": {"assign_flop": flops, "hbm_bytes": hbm},
            "unit_norm": bool(np.allclose(norms[wl.n_desc > 0], 1.0, atol=1e-5)),
            "cpu_oracle_images_per_s": 1.0 / cpu_s, "cpu_oracle_sample": "1 image of %d rows, FP64 numpy"
                                                                        % int(wl.n_desc[i0]),
            "codebook": "C rows sampled from the workload (seeded), a stand-in for k-means centroids"}


def pipeline_e2e(args, wl, host, kp, stream, world, dev):
    """End to end through the public calls, timed by the host clock around the
    whole job: the MBR schedule (cm_schedule_blocks, host), then
    cm_run_schedule with its own centring pass (exact column sums of the
    pinned host rows on the GPU: the first row's images go straight into
    their slots, every other image passes once through a staging block), and
    per block row: H2D of the row's new images, hashing, one fused match
    launch, compaction straight into pinned host memory, release of the freed
    images.  The index (its device arena and pinned result buffers) is set up
    once, outside the timed region, as a service would keep it."""
    import torch
    import paper_2505_22089_b300 as cm
    p = cm.Params.make(rerank=args.rerank, algo=args.algo, projection=args.projection, K=args.K)
    off = wl.row_off
    hl = [host[off[i]:off[i + 1]] for i in range(wl.n_images)]
    budget = int(args.budget_gb * 2 ** 30)
    sched = cm.schedule_blocks(wl.pairs, wl.n_desc, p, budget, args.block_images)
    index = cm.Index(p, wl.n_desc, arena_bytes=cm.schedule_arena_bytes(sched, p, wl.n_desc))
    sched.close()
    walls, parts, stats = [], [], None
    for s in range(args.e2e_steps + 1):
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sched = cm.schedule_blocks(wl.pairs, wl.n_desc, p, budget, args.block_images)
        t1 = time.perf_counter()
        stats, _ = cm.run_schedule(index, sched, hl, verify=None, workers=1, stream=stream, centre=True)
        sched.close()
        t2 = time.perf_counter()
        if s > 0:
            walls.append((t2 - t0) * 1e3)
            parts.append(((t1 - t0) * 1e3, stats["wall_ms"]))
    ms = _sync_ms(float(np.mean(walls)), world, dev)
    pm = np.mean(parts, axis=0)
    out = {"value": len(wl.pairs) * world / (ms / 1e3), "unit": "pairs/s", "ms_per_step": ms,
           "h2d_bytes_per_step": int(stats["h2d_bytes"]), "d2h_bytes_per_step": int(stats["d2h_bytes"]),
           "block_rows": stats["rows"], "kernels_per_step": int(stats["kernels"]),
           "prefetched_rows": int(stats["prefetched_rows"]),
           "parts_ms": {"schedule": round(float(pm[0]), 2), "pipeline_with_centring": round(float(pm[1]), 2)},
           "form": "host clock around cm_schedule_blocks + cm_run_schedule(centre=1): centring statistics from "
                   "the pinned host rows, H2D of each row's images, hashing, match, compaction into pinned host "
                   "memory; h2d counts every descriptor byte copied (the centring pass and the rows' loads)"}
    index.close()
    del index
    ver = None
    if kp is not None and args.verify_workers > 0:
        sched = cm.schedule_blocks(wl.pairs, wl.n_desc, p, int(args.budget_gb * 2 ** 30), args.block_images)
        index = cm.Index(p, wl.n_desc, arena_bytes=cm.schedule_arena_bytes(sched, p, wl.n_desc))
        index.mean_host(hl, stream)
        # outlier removal on the host workers, overlapped with the GPU rows:
        # RANSAC alone, then the SAO local constraint ahead of RANSAC (Sec. 2.3.3)
        kl = [kp[off[i]:off[i + 1]] for i in range(wl.n_images)]
        ver = {"overlap": "GPU rows overlap CPU verification when wall_ms < gpu_ms + verify_ms / workers"}
        kp_dev = torch.from_numpy(np.ascontiguousarray(kp, dtype=np.float32)).to(dev)
        kp_off_dev = torch.from_numpy(off.astype(np.int64)).to(dev)
        for mode, sao_k, gpu_sao_k in (("ransac", 0, 0), ("sao_ransac", 8, 0), ("gpu_sao_ransac", 0, 8)):
            kept = np.zeros(len(wl.pairs), dtype=np.int64)
            st, inl = cm.run_schedule(index, sched, hl, verify="affine", keypoints=kl, thresh_px=4.0,
                                      workers=args.verify_workers, stream=stream, sao_k=sao_k, sao_kept=kept,
                                      gpu_sao_k=gpu_sao_k, kp_dev=kp_dev, kp_off_dev=kp_off_dev)
            v = {k: (round(x, 2) if isinstance(x, float) else x) for k, x in st.items()}
            v["inliers"] = int(inl.sum())
            v["inlier_share"] = float(inl.sum() / max(1, st["matches"]))
            if sao_k:
                v["sao_kept"] = int(kept.sum())
                v["sao"] = {"k": sao_k, "max_score": 0.875, "where": "host worker threads"}
            if gpu_sao_k:
                v["sao"] = {"k": gpu_sao_k, "max_score": 0.875, "where": "GPU, per block row before compaction",
                            "note": "matches counts the kept ones"}
            ver[mode] = v
        del kp_dev, kp_off_dev
        index.close()
        sched.close()
    return out, ver


def strategy_rows(wl, p, budget, size_blk):
    """Row lists of the five strategies for one workload under one budget
    (MBR from cm_schedule_blocks, the others from the strategies module)."""
    import paper_2505_22089_b300 as cm
    from paper_2505_22089_b300 import strategies as st
    ib = np.array([cm.image_bytes(p, int(n)) for n in wl.n_desc], dtype=np.int64)
    order = st.connection_order(wl.pairs, wl.n_images, cm.gps_order)
    sched = cm.schedule_blocks(wl.pairs, wl.n_desc, p, int(budget), size_blk)
    mbr = [{"load": r["load"], "free": r["free"], "pairs": r["pairs"], "iteration": r["iteration"]}
           for r in sched.rows]
    sched.close()
    part = max(1, int(budget // 2 // ib.max()))
    return ib, {"per_pair": st.per_pair(wl.pairs), "pair_blocks": st.pair_blocks(wl.pairs, ib, budget),
                "load_free_list": st.load_free_list(wl.pairs, ib, budget, order),
                "graph_partition": st.graph_partition(wl.pairs, ib, budget, order, part), "mbr_blocks": mbr}


def schedule_comparison(args, wl, p, stream, world, dev):
    """Data schedules compared (Sec. 2.2 against the strategies of Sec. 4):
    one pair at a time, blocks of pairs in input order, a load/free list in
    connection order (one pair per row), graph partitions, and the MBR block
    rows.  (1) Counted on the host for the bench workload under its budget:
    image loads, H2D bytes, launches, peak resident bytes.  (2) Measured end to
    end through cm_run_schedule on the 200-image grid under a quarter of its
    bytes: wall time, GPU time (GPU busy = GPU / wall), H2D bytes, pairs/s."""
    import paper_2505_22089_b300 as cm
    from paper_2505_22089_b300 import strategies as st
    budget = int(args.budget_gb * 2 ** 30)
    ib, strat = strategy_rows(wl, p, budget, args.block_images)
    counts = {}
    for name, rows in strat.items():
        r = st.residency(rows, ib)
        r["h2d_bytes"] = int(128 * sum(int(wl.n_desc[x]) for row in rows for x in row["load"]))
        counts[name] = r
    if args.strategy_runs == 0:
        return {"budget_bytes": budget, "size_blk": args.block_images, "counted": counts, "measured": None}
    # measured on a smaller grid with a tight budget, so that every strategy has to choose
    sw = synth.scaled(args.workload, gx=20, gy=10) if args.workload == "grid5000" else wl
    host = sw.generate()
    off = sw.row_off
    hl = [host[off[i]:off[i + 1]] for i in range(sw.n_images)]
    sums = host.astype(np.uint64).sum(0)
    ib2 = np.array([cm.image_bytes(p, int(n)) for n in sw.n_desc], dtype=np.int64)
    budget2 = int(ib2.sum() // 4)
    _, strat2 = strategy_rows(sw, p, budget2, args.block_images)
    measured = {}
    for name, rows in strat2.items():
        sched = cm.schedule_from_rows(rows, sw.pairs, sw.n_images)
        index = cm.Index(p, sw.n_desc, arena_bytes=cm.schedule_arena_bytes(sched, p, sw.n_desc))
        index.set_mean(sums, int(sw.total_desc), stream)
        cm.run_schedule(index, sched, hl, verify=None, workers=1, stream=stream)   # warm-up
        stt, _ = cm.run_schedule(index, sched, hl, verify=None, workers=1, stream=stream)
        rr = st.residency(rows, ib2)
        measured[name] = {"pairs_per_s": len(sw.pairs) / (stt["wall_ms"] / 1e3), "wall_ms": round(stt["wall_ms"], 2),
                          "gpu_ms": round(stt["gpu_ms"], 2), "gpu_busy": stt["gpu_ms"] / stt["wall_ms"],
                          "pairs_per_gpu_s": len(sw.pairs) / (stt["gpu_ms"] / 1e3),
                          "h2d_bytes": int(stt["h2d_bytes"]), "rows": stt["rows"], "kernels": int(stt["kernels"]),
                          "peak_resident_bytes": rr["peak_resident_bytes"],
                          "memory_use": rr["peak_resident_bytes"] / budget2, "matches": int(stt["matches"])}
        index.close()
        sched.close()
    return {"budget_bytes": budget, "size_blk": args.block_images, "counted": counts,
            "measured": {"workload": "%s %dx%d grid, %d images, %d pairs" % (args.workload, 20, 10, sw.n_images,
                                                                              len(sw.pairs)),
                         "budget_bytes": budget2, "strategies": measured,
                         "note": "cm_run_schedule from pinned host rows, no verification; gpu_busy = GPU time "
                                 "of the rows (copies included) / wall time; pairs_per_gpu_s = pairs / GPU time"}}


class GpuShardEngine:
    """One rank's share of a sharded job on its GPU: the images it needs
    resident in HBM (used in place), one match plan per block row it holds.
    A step: exact column sums of its owned images (on the GPU), the caller's
    all-reduce, the mean from the reduced sums, hashing of its resident images,
    then each row's fused match launch and compaction."""

    def __init__(self, args, wl, p, part, dev):
        import torch
        import paper_2505_22089_b300 as cm
        self.cm, self.torch, self.dev = cm, torch, dev
        self.stream = torch.cuda.current_stream(dev)
        off = wl.row_off
        res = part["resident"]
        nd = wl.n_desc.astype(np.int64)
        total = int(nd[res].sum())
        host = torch.empty((max(total, 1), 128), dtype=torch.uint8, pin_memory=True)
        hv = host.numpy()
        at, self.views = 0, []
        for i in res:   # each image generated on its own (only this rank's share)
            n = int(nd[i])
            wl.generate(int(i), int(i) + 1, desc=hv[at:at + n] if n else np.empty((0, 128), np.uint8))
            at += n
        self.h2d_bytes = 128 * total
        self.host = host
        self.dbuf = host.to(dev)
        at = 0
        for i in res:
            n = int(nd[i])
            self.views.append(self.dbuf[at:at + n])
            at += n
        nd_res = np.zeros_like(wl.n_desc)
        nd_res[res] = wl.n_desc[res]
        rows = [r for r in part["rows"] if len(r)]
        arena = (cm.index_bytes(p, nd_res, inplace=True) + cm.PLAN_HEADROOM +
                 sum(cm.pairs_plan_bytes(p, wl.n_desc, wl.pairs[r]) for r in rows))
        self.index = cm.Index(p, wl.n_desc, arena_bytes=arena)
        self.index.set_mean(np.zeros(128, np.uint64), 1)   # a placeholder: every step sets the real mean
        self.index.load(res, self.views, cm.MEM_DEVICE_INPLACE)
        self.rows = rows
        self.plans = [cm.MatchPlan(self.index, wl.pairs[r]) for r in rows]
        self.outs = [pl.alloc_out(d12=False) for pl in self.plans]
        self.comps = [cm.compact_out(pl) for pl in self.plans]
        self.owned = part["owned"]
        self.sums = torch.zeros(128, dtype=torch.int64, device=dev)
        self.kernels = 0

    def local_sums(self):
        self.index.col_sums_of(self.owned, self.sums)
        return self.sums

    def apply_mean(self, sums, n_total):
        self.index.set_mean_device(sums, n_total)

    def match(self):
        import ctypes
        cm = self.cm
        self.index.hash()
        for pl, o, c in zip(self.plans, self.outs, self.comps):
            pl.run(o)
            cm.check(cm.lib().cm_match_plan_compact(pl.h, cm._ptr(o["best_j"]), cm._ptr(c["counts"]),
                                                    cm._ptr(c["offsets"]), cm._ptr(c["total"]), cm._ptr(c["matches"]),
                                                    ctypes.c_uint64(c["capacity"]), cm._stream(None)))

    def timer(self):
        torch = self.torch
        start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

        class T:
            def __enter__(s):
                start.record()
                return s

            def __exit__(s, *a):
                stop.record()
                stop.synchronize()
                s.ms = start.elapsed_time(stop)
        return T()

    def sync(self):
        self.torch.cuda.synchronize(self.dev)
        self.index.check()

    def upload(self):
        """The e2e step's input: this rank's descriptor rows from pinned host memory."""
        self.dbuf.copy_(self.host, non_blocking=True)

    def download(self):
        """The e2e step's result: the compacted match lists, to host memory; returns bytes."""
        n = 0
        for c in self.comps:
            tot = int(c["total"].item())
            n += 4 * tot + 8 * c["offsets"].numel()
            c["offsets"].cpu()
            c["matches"][:tot].cpu()
        return n

    def launches(self, p):
        hash_k = (3 if p.projection == 0 else 2) + (1 if p.rerank in (1, 2) else 0)
        match_k = 2 if p.rerank in (1, 2) else 1
        return 2 + hash_k + len(self.plans) * (match_k + 3)

    def results(self):
        """(pair ids, row offsets, best_j on the host) per plan, and the matches counted on the GPU."""
        out = []
        n = 0
        for r, pl, o, c in zip(self.rows, self.plans, self.outs, self.comps):
            out.append((r, pl.row_off, o["best_j"][:pl.rows].cpu().numpy()))
            n += int(c["total"].item())
        return out, n

    def scalar(self, v):
        return self.torch.tensor([float(v)], dtype=self.torch.float64, device=self.dev)


def run_sharded(args, rank, world, make_engine):
    """One job sharded over the ranks (the partition of the multi-GPU plan):
    every rank computes the same MBR schedule, takes its contiguous share of
    the block rows' pairs, makes resident only the images it needs, and per
    step contributes the column sums of the images it owns to the one
    all-reduce (128 exact integers) before hashing and matching.  Timing:
    the engine's clock over the timed steps, max over ranks.  The ranks'
    decision checksums and match counts add up to a single run's."""
    import torch
    import torch.distributed as dist
    import paper_2505_22089_b300 as cm
    from paper_2505_22089_b300 import shard
    wl = make_workload(args)
    p = cm.Params.make(rerank=args.rerank, algo=args.algo, projection=args.projection, K=args.K)
    sched = cm.schedule_blocks(wl.pairs, wl.n_desc, p, int(args.budget_gb * 2 ** 30), args.block_images)
    rows = [np.asarray(r["pairs"], dtype=np.int64) for r in sched.rows if r["pairs"]]
    sched.close()
    part = shard.plan(rows, wl.pairs, wl.n_images, rank, world, wl.n_desc)
    eng = make_engine(args, wl, p, part)

    def step():
        s = eng.local_sums()
        dist.all_reduce(s, op=dist.ReduceOp.SUM)
        eng.apply_mean(s, wl.total_desc)
        eng.match()

    for _ in range(args.warmup):
        step()
    eng.sync()
    dist.barrier()
    with eng.timer() as tm:
        for _ in range(args.steps):
            step()
    eng.sync()
    t = eng.scalar(tm.ms / args.steps)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms = float(t.item())
    # end to end: per step the rank's rows from pinned host memory, the step, the match lists back
    walls, d2h = [], 0
    for _ in range(args.e2e_steps):
        dist.barrier()
        t0 = time.perf_counter()
        eng.upload()
        step()
        d2h = eng.download()
        eng.sync()
        walls.append((time.perf_counter() - t0) * 1e3)
    e2e = None
    if walls:
        te = eng.scalar(float(np.mean(walls)))
        dist.all_reduce(te, op=dist.ReduceOp.MAX)
        e2e_ms = float(te.item())
    res, n_match = eng.results()
    csum = sum(shard.checksum(ids, ro, b) for ids, ro, b in res) % shard._M61
    parts = [None] * world
    dist.all_gather_object(parts, (int(csum), int(n_match), int(sum(len(r) for r in part["rows"])),
                                   int(getattr(eng, "h2d_bytes", 0)), int(d2h), int(eng.launches(p))))
    if rank != 0:
        return None
    if walls:
        e2e = {"value": len(wl.pairs) / (e2e_ms / 1e3), "unit": "pairs/s", "ms_per_step": e2e_ms,
               "h2d_bytes_per_step": int(sum(c[3] for c in parts)), "d2h_bytes_per_step": int(sum(c[4] for c in parts)),
               "form": "per rank: its resident images' rows from pinned host memory, the step, the match lists "
                       "and their offsets back to host memory; host clock, max over ranks"}
    return {"metric": METRIC, "value": len(wl.pairs) / (ms / 1e3), "unit": "pairs/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "u8/" + args.rerank,
            "data": "synthetic (seeded track model, %s)" % args.workload,
            "config": {"workload": args.workload, "images": wl.n_images, "pairs": len(wl.pairs),
                       "parallelism": "pairs of the block rows cut into %d contiguous ranges" % world,
                       "rerank": args.rerank, "L": p.L, "m": p.m, "K": p.K,
                       "step": "per rank: column sums of owned images, one all-reduce of 128 integers, mean, "
                               "hashing of resident images, per block row match + compaction",
                       "l2": "inputs larger than L2"},
            "shards": [{"rank": r, "pairs": c[2], "matches": c[1]} for r, c in enumerate(parts)],
            "decision_checksum": int(sum(c[0] for c in parts) % shard._M61),
            "matches": int(sum(c[1] for c in parts)),
            "e2e": e2e, "gpu_launches": int(args.steps * sum(c[5] for c in parts))}


def timed_leg(legs, name, fn):
    t0 = time.time()
    r = fn()
    legs[name] = round(time.time() - t0, 1)
    return r


def run_ours(args, rank, world, local):
    import torch
    import paper_2505_22089_b300 as cm

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl = make_workload(args)
    if world > 1:
        wl.seed += 1000 * rank          # weak scaling: an independent job of the same shape per rank
    n_desc = wl.n_desc
    total = wl.total_desc
    pairs = wl.pairs
    t0 = time.time()
    host = torch.empty((total, 128), dtype=torch.uint8, pin_memory=True)
    kp = None
    if args.verify_workers > 0:
        _, kp = wl.generate(desc=host.numpy(), want_kp=True)
    else:
        wl.generate(desc=host.numpy())
    gen_s = time.time() - t0
    stream = torch.cuda.Stream(device=dev)
    p = cm.Params.make(rerank=args.rerank, algo=args.algo, projection=args.projection, K=args.K)
    sched = cm.schedule_blocks(pairs, n_desc, p, int(args.budget_gb * 2 ** 30), args.block_images)
    rows = [np.asarray(r["pairs"], dtype=np.int64) for r in sched.rows if r["pairs"]]
    n_iter = sched.iterations
    sched.close()

    # ---- device-resident steps (graph replay), every form
    forms = [args.rerank] + ([f for f in ("fp32", "int", "bf16", "fp8") if f != args.rerank]
                             if args.forms == "all" else [])
    # the oracle's sample (rank 0 at N=1) and the exhaustive-NN sample: their GPU rows are kept
    check = rank == 0 and world == 1 and args.oracle_frac > 0
    sample = pick_sample(pairs, args.oracle_frac, args.oracle_min_pairs) if check else None
    nn_sel = (np.sort(np.random.default_rng(123).choice(len(pairs), min(args.nn_pairs, len(pairs)), replace=False))
              if args.nn_pairs > 0 else np.zeros(0, np.int64))
    desc_dev = host.to(dev, non_blocking=False)
    legs = {"generate": round(gen_s, 1)}
    t_leg = time.time()
    fr = device_forms(args, wl, desc_dev, rows, stream, dev, world, forms,
                      check=sample if sample is not None else (np.zeros(0, np.int64),) * 3, extra=nn_sel)
    head = fr[args.rerank]
    got, sums = head.pop("_got"), head.pop("_sums")
    head_p = head.pop("_p")
    gpu_rows = {k: v[0] for k, v in got["full"].items()}
    legs["device_forms"], t_leg = round(time.time() - t_leg, 1), time.time()
    vl = vlad_encoding(args, wl, desc_dev, host.numpy(), stream, world, dev) if args.vlad_codewords > 0 else None
    legs["vlad"], t_leg = round(time.time() - t_leg, 1), time.time()
    ceiling = sweep = None
    if args.nn_pairs > 0:
        ceiling, sweep = exhaustive_leg(args, wl, desc_dev, host.numpy(), sums, pairs, nn_sel, gpu_rows, stream,
                                        world, dev, float(peaks()[0].get("bf16_tflops", 1800.0)))
        legs["exhaustive_and_sweep"] = round(time.time() - t_leg, 1)
    del desc_dev
    torch.cuda.empty_cache()
    ms = head["ms_per_step"]
    value = head["value"]

    # roofline: the lookup launch's candidate evaluations (128-bit Hamming distances) per second
    # against the measured peak of that operation on this GPU: cm_probe_int's carry-save distance
    # (3 POPC + 8 LOP3) per clock per SM, x SMs x the SM clock sampled during the timed steps
    pk, pk_kind = peaks()
    sm_mhz = float(head["clocks"].get("sm_mhz") or pk.get("sm_max_mhz", 2032.0))
    probe = {k: cm.probe_int(k, 8192) for k in ("popc", "lop3", "ham4", "ham3")}
    peak = probe["ham3"] * SM_COUNT * sm_mhz * 1e6
    evals = head["evals_per_step"]
    achieved = evals / head["launches"] / (head["scan_launch_ms"] / 1e3)
    roofline = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "T distances/s",
                "frac": achieved / peak, "traffic": kmatch_traffic(args, len(pairs) / head["launches"]),
                "traffic_kind": "ncu DRAM bytes per pair of k_match_bm on the 200-image grid x pairs per launch",
                "peak_kind": "measured live: cm_probe_int carry-save 128-bit distance %.3f per clock per SM x %d "
                             "SMs x %.0f MHz (SM clock sampled in the timed steps)" % (probe["ham3"], SM_COUNT, sm_mhz),
                "probe_per_clock_per_sm": {k: round(v, 3) for k, v in probe.items()},
                "kernel": "k_match_bm" if (head.get("tuned") or {}).get("algo", "bucket") == "bucket" else "k_match",
                "algo": (head.get("tuned") or {}).get("algo", args.algo),
                "evals_per_step": evals, "k_match_launch_ms": head["scan_launch_ms"],
                "match_launch_ms": head["match_launch_ms"],
                "rerank_launch_ms": head["match_launch_ms"] - head["scan_launch_ms"],
                "match_ms_per_step": head["match_ms_per_step"],
                "match_share_of_step": head["match_ms_per_step"] / ms}

    # ---- end to end through the pipeline call, then the same with CPU verification overlapped
    e2e, verified = (None, None)
    if args.e2e_steps > 0:
        t_leg = time.time()
        e2e, verified = pipeline_e2e(args, wl, host, kp, stream, world, dev)
        legs["e2e_and_verified"] = round(time.time() - t_leg, 1)

    # ---- plain per-pair form (no schedule): upload both images, hash, match, download, free
    t_leg = time.time()
    plain = plain_per_pair(args, wl, host, sums, stream, dev) if args.plain_pairs > 0 else None
    legs["plain"], t_leg = round(time.time() - t_leg, 1), time.time()

    # ---- the FP64 oracle on its sample (rank 0 at N=1): agreement, and the CPU baseline from its timing
    cpu = base = None
    if check:
        cpu, base = oracle_check(wl, host.numpy(), head_p, pairs, *sample, got, sums, args.rerank)
        legs["oracle_check"] = round(time.time() - t_leg, 1)
        cpu["fp64_rechecks_per_step"] = head["fp64_rechecks_per_step"]
        cpu["fp8_top2_swaps_per_step"] = head["fp8_top2_swaps_per_step"]
    del got

    forms_out = {}
    for f, r in fr.items():
        forms_out[f] = {k: (round(v, 6) if isinstance(v, float) else v) for k, v in r.items()
                        if k in ("value", "ms_per_step", "matches", "decision_agreement_vs_fp32",
                                 "match_jaccard_vs_fp32", "graph_kernels", "tuned")}
    res = {
        "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8/fp32" if args.rerank == "fp32" else "u8/" + args.rerank,
        "data": "synthetic (seeded track model, %s)" % args.workload,
        "config": {"workload": args.workload, "images": wl.n_images, "pairs": len(pairs),
                   "descriptors": total, "rerank": args.rerank, "algo": args.algo, "projection": args.projection,
                   "L": p.L, "m": p.m, "K": p.K, "ratio": "%d/%d" % (p.ratio_num, p.ratio_den),
                   "block_rows": len(rows), "gps_iterations": n_iter, "size_blk": args.block_images,
                   "budget_gb": args.budget_gb, "step": "one CUDA graph: rehash + per block row match + compaction",
                   "l2": "inputs (%.1f GB descriptors) larger than L2" % (total * 128 / 1e9),
                   "generate_s": round(gen_s, 1)},
        "e2e": e2e,
        "forms": forms_out,
        "plain_fp32_per_pair": plain,
        "pipeline_verified": verified,
        "schedules": timed_leg(legs, "schedules", lambda: schedule_comparison(args, wl, p, stream, world, dev)
                               if world == 1 else None),
        "configs": timed_leg(legs, "configs", lambda: config_lines(args, stream, dev)
                             if (world == 1 and args.configs == "all") else None),
        "leg_seconds": legs,
        "gpu_launches": args.steps * head["graph_kernels"],
        "roofline": roofline,
        "vlad": vl,
        "exhaustive_nn": ceiling,
        "quality_sweep": sweep,
        "clocks": head["clocks"],
    }
    if cpu is not None:
        if not args.no_cpu_baseline:
            res["cpu_baseline"] = base
        res["agreement"] = cpu
    return res, None


def plain_per_pair(args, wl, host, sums, stream, dev):
    """Sequential per-pair form (the paper's "no schedule" strategy, Sec. 2.2):
    per pair, a fresh two-image index in one fixed arena (upload both images
    from pinned host memory, hash, bucket), one match launch with FP32 rerank,
    download of the results, free."""
    import torch
    import paper_2505_22089_b300 as cm
    n = min(args.plain_pairs, len(wl.pairs))
    sel = np.linspace(0, len(wl.pairs) - 1, n).astype(np.int64)
    off = wl.row_off
    pf = cm.Params.make(rerank="fp32")
    nmax = int(wl.n_desc.max())
    arena = torch.empty(cm.index_bytes(pf, [nmax, nmax]) + (1 << 20), dtype=torch.uint8, device=dev)
    best = torch.empty(nmax, dtype=torch.int32, device=dev)
    best_h = torch.empty(nmax, dtype=torch.int32, pin_memory=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in sel:
        i, j = (int(x) for x in wl.pairs[k])
        ix = cm.Index(pf, [wl.n_desc[i], wl.n_desc[j]], arena=arena)
        ix.set_mean(sums, wl.total_desc, stream)
        ix.load([0, 1], [host[off[i]:off[i + 1]], host[off[j]:off[j + 1]]], cm.MEM_HOST, stream)
        pl = cm.MatchPlan(ix, [[0, 1]], stream=stream)
        pl.run({"best_j": best}, stream)
        with torch.cuda.stream(stream):
            best_h[: pl.rows].copy_(best[: pl.rows], non_blocking=True)
        stream.synchronize()
        pl.close()
        ix.close()
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": "pairs/s", "pairs_timed": int(n), "rerank": "fp32",
            "form": "per pair: upload 2 images (pinned host), hash, bucket, 1 match launch, download, free"}


def recall_precision(g, ex):
    shared = int(((g == ex) & (g >= 0)).sum())
    n_ex, n_g = int((ex >= 0).sum()), int((g >= 0).sum())
    return shared, n_ex, n_g


def exhaustive_leg(args, wl, desc_dev, host, sums, pairs, sel, gpu_rows, stream, world, dev, peak_tflops):
    """Quality ceiling and its cost: exhaustive nearest neighbours (cm_nn_pairs,
    tensor cores, exact) on a seeded sample of pairs, timed with CUDA events;
    the main run's cascade-hashing matches against them (recall = shared /
    exhaustive, precision = shared / cascade); then the L / K sweep."""
    import torch
    import paper_2505_22089_b300 as cm
    sp = pairs[sel]
    with torch.cuda.stream(stream):
        best, _, _, rows = cm.nn_pairs(desc_dev, wl.n_desc, sp, stream=stream)   # warm-up, status checked
        start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        start.record(stream)
        for _ in range(2):
            best, _, _, rows = cm.nn_pairs(desc_dev, wl.n_desc, sp, stream=stream, check_status=False)
        stop.record(stream)
        stop.synchronize()
    ms = start.elapsed_time(stop) / 2
    bj = best.cpu().numpy()
    exact = {int(k): bj[rows[q]:rows[q + 1]] for q, k in enumerate(sel)}
    shared = n_ex = n_g = 0
    for k in sel:
        s_, e_, g_ = recall_precision(gpu_rows[int(k)], exact[int(k)])
        shared, n_ex, n_g = shared + s_, n_ex + e_, n_g + g_
    nd = wl.n_desc.astype(np.int64)
    flop = 2.0 * 128 * float((nd[sp[:, 0]] * nd[sp[:, 1]]).sum())
    tf = flop / (ms / 1e3) / 1e12
    ceiling = {"pairs": int(len(sel)), "exhaustive_matches": n_ex, "cascade_matches": n_g,
               "recall": shared / n_ex if n_ex else 1.0, "precision": shared / n_g if n_g else 1.0,
               "exhaustive_ms": ms, "exhaustive_pairs_per_s": len(sel) * world / (ms / 1e3),
               "exhaustive_tflops": tf, "exhaustive_frac_of_bf16_peak": tf / peak_tflops,
               "note": "cm_nn_pairs: every database row a candidate, exact d^2 from BF16 tensor-core products, "
                       "exact ratio test 4/5; FLOP = 2 x 128 x n_i x n_j per pair"}
    sweep = quality_sweep(wl, host, sums, pairs, sel, exact, gpu_rows, args.K)
    return ceiling, sweep


def quality_sweep(wl, desc, sums, pairs, sel, exact, gpu_rows, main_K):
    """Recall / precision against exhaustive NN, and the candidate evaluations
    of the lookup, for L in {4, 6, 8} tables and K in {4, 8, 16} kept
    candidates, on the sampled pairs: an index over just their images, centred
    on the whole workload's mean like the main run (so L=6 reproduces the
    main run's matches at the main run's K, which is checked)."""
    import paper_2505_22089_b300 as cm
    off = wl.row_off
    imgs = sorted(set(int(x) for k in sel for x in pairs[k]))
    remap = {im: n for n, im in enumerate(imgs)}
    sub_nd = np.array([wl.n_desc[im] for im in imgs], dtype=np.int32)
    sub_pairs = np.array([[remap[int(pairs[k][0])], remap[int(pairs[k][1])]] for k in sel], dtype=np.int32)
    views = [np.ascontiguousarray(desc[off[im]:off[im + 1]]) for im in imgs]
    out = []
    import torch
    for L in (4, 6, 8):
        for K in (4, 8, 16):
            p = cm.Params.make(L=L, K=K)
            index = cm.Index(p, sub_nd)
            index.set_mean(sums, wl.total_desc)
            index.load(list(range(len(imgs))), views, cm.MEM_HOST)
            plan = cm.MatchPlan(index, sub_pairs)
            o = plan.alloc_out(d12=False)
            plan.run(o)
            torch.cuda.synchronize()
            bj = o["best_j"].cpu().numpy()
            shared = n_ex = n_g = 0
            same_as_main = True
            for q, k in enumerate(sel):
                mine = bj[plan.row_off[q]:plan.row_off[q + 1]]
                s, e, g = recall_precision(mine, exact[int(k)])
                shared, n_ex, n_g = shared + s, n_ex + e, n_g + g
                same_as_main &= bool(np.array_equal(mine, gpu_rows[int(k)]))
            pt = {"L": L, "K": K, "recall": round(shared / max(n_ex, 1), 4),
                  "precision": round(shared / max(n_g, 1), 4), "matches": n_g,
                  "evals": bucket_evaluations(index, wl, sub_pairs)}
            if (L, K) == (6, main_K):
                pt["equals_main_run"] = same_as_main
            out.append(pt)
            plan.close()
            index.close()
    return {"pairs": int(len(sel)), "points": out,
            "note": "fp32 rerank; evals = sum over pairs, tables, buckets of n_I * n_J"}


def run_reference(args, rank, world):
    """The FP64 CPU oracle on the host cores, on a bounded sample of pairs."""
    import oracle
    if rank != 0:
        return None
    wl = synth.workload(args.workload)
    rng = np.random.default_rng(0)
    sel = np.sort(rng.choice(len(wl.pairs), min(args.oracle_pairs, len(wl.pairs)), replace=False))
    desc = wl.generate()
    cores = os.cpu_count() or 1
    op = oracle.Params()
    t0 = time.perf_counter()
    oix = oracle.Index(desc, wl.n_desc, op, threads=cores)
    t_mu = time.perf_counter() - t0
    times = []
    for s in range(args.warmup + args.steps):
        oix._cache.clear()
        t0 = time.perf_counter()
        oix.match(wl.pairs[sel])
        if s >= args.warmup:
            times.append(time.perf_counter() - t0)
    per_pair = np.mean(times) / len(sel) + t_mu / len(wl.pairs)
    value = 1.0 / per_pair
    sample = "%d of %d pairs (hash both images + match), mean time pro-rated per pair" % (len(sel), len(wl.pairs))
    return {"metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": np.mean(times) * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (%s)" % args.workload,
            "config": {"workload": args.workload, "images": wl.n_images, "pairs": len(wl.pairs),
                       "descriptors": int(np.sum(wl.n_desc)), "L": op.L, "m": op.m, "K": op.K,
                       "ratio": "%d/%d" % (op.ratio_num, op.ratio_den), "sample_pairs": int(len(sel))},
            "impl": "reference",
            "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    if args.verify_workers < 0:
        args.verify_workers = os.cpu_count() or 1
    rank, world, local = dist_env()
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl" if args.impl == "ours" else "gloo")
    if args.impl == "reference":
        res = run_reference(args, rank, world)
    elif world > 1 and args.multi == "shard":
        import torch
        torch.cuda.set_device(local)
        dev = torch.device("cuda", local)
        res = run_sharded(args, rank, world, lambda a, wl, p, part: GpuShardEngine(a, wl, p, part, dev))
    else:
        res, _ = run_ours(args, rank, world, local)
    if rank == 0 and res is not None:
        print(json.dumps(res))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
