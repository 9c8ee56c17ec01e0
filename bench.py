#!/usr/bin/env python3
"""Throughput of cascade-hashing feature matching on one B300: pairs matched/s.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload grid5000]
                    [--rerank fp32|int|bf16|fp8] [--impl ours|reference]

A step is one pass of the whole hot path over the workload: centring
statistics, projection to bucket keys and codes, bucket construction, and the
persistent fused match launch of every block row (lookup, Hamming top-K,
rerank, ratio test).  `value` times steps whose descriptors are already
resident in HBM; `e2e` times the same work through the C ABI with the
descriptors in pinned host memory (H2D inside the step) and the per-query
results copied back (D2H inside the step).

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
POPC_PER_CLK_PER_SM = 16      # measured on B300 (integer population count pipe)
SM_COUNT = 148


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="grid5000", choices=sorted(synth.WORKLOADS))
    ap.add_argument("--rerank", default="fp32", choices=["fp32", "int", "bf16", "fp8"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--algo", default="auto", choices=["auto", "tile", "warp"], help="match kernel thread mapping")
    ap.add_argument("--projection", default="tc", choices=["tc", "ffma"], help="hash projection: tensor cores or FP32 FFMA")
    ap.add_argument("--block-images", type=int, default=400, help="Size_blk: images per schedule chunk")
    ap.add_argument("--budget-gb", type=float, default=150.0, help="HBM budget of the MBR schedule")
    ap.add_argument("--plain-pairs", type=int, default=200, help="pairs timed in the plain per-pair form")
    ap.add_argument("--oracle-pairs", type=int, default=12, help="pairs in the CPU-oracle sample")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--grid", default=None, help="GXxGY: a smaller grid of the same per-image shape (profiling)")
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
    if args.grid:
        gx, gy = (int(v) for v in args.grid.lower().split("x"))
        return synth.WORKLOADS[args.workload](gx=gx, gy=gy)
    return synth.workload(args.workload)


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
    wl.generate(desc=host.numpy())
    gen_s = time.time() - t0
    p = cm.Params.make(rerank=args.rerank, algo=args.algo, projection=args.projection)
    stream = torch.cuda.Stream(device=dev)

    # schedule blocks (MBR) under the HBM budget
    sched = cm.schedule_blocks(pairs, n_desc, p, int(args.budget_gb * 2 ** 30), args.block_images)
    rows = [np.asarray(r["pairs"], dtype=np.int64) for r in sched.rows if r["pairs"]]

    # ---- device-resident: descriptors in HBM before the timed region
    desc_dev = host.to(dev, non_blocking=False)
    with torch.cuda.stream(stream):
        index = cm.Index.build(p, n_desc, desc_dev, stream=stream)
        plans = [cm.MatchPlan(index, pairs[r], stream=stream) for r in rows]
        n_rows = sum(pl.rows for pl in plans)
        outs = [{"best_j": torch.empty(max(pl.rows, 1), dtype=torch.int32, device=dev)} for pl in plans]
    stream.synchronize()
    sums, _ = index.col_sums(stream)

    def step(ev=None):
        index.rehash(stream)
        for k, (pl, o) in enumerate(zip(plans, outs)):
            if ev is not None:
                ev[k][0].record(stream)
            pl.run(o, stream)
            if ev is not None:
                ev[k][1].record(stream)

    for _ in range(args.warmup):
        step()
    stream.synchronize()
    evs = [[[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in plans] for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        start.record(stream)
        for s in range(args.steps):
            step(evs[s])
        stop.record(stream)
        stop.synchronize()
    torch.cuda.synchronize()
    ms = start.elapsed_time(stop) / args.steps
    if world > 1:
        t = torch.tensor([ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    match_ms = [sum(e[k][0].elapsed_time(e[k][1]) for k in range(len(plans))) for e in evs]
    gpu_rows = {}
    for pl, o, r in zip(plans, outs, rows):
        bj = o["best_j"].cpu().numpy()
        for q, k in enumerate(r):
            gpu_rows[int(k)] = bj[pl.row_off[q]:pl.row_off[q + 1]]
    match_launch_ms = float(np.mean(match_ms)) / max(1, len(plans))
    n_pairs = len(pairs)
    value = n_pairs * world / (ms / 1e3)

    # algorithmic work of the match kernel: candidate evaluations (4 POPC each)
    evals = bucket_evaluations(index, wl, pairs)
    clocks = clk.summary()
    pk, pk_kind = peaks()
    sm_mhz = float(pk.get("sm_max_mhz", 2032.0))
    popc_peak = POPC_PER_CLK_PER_SM * SM_COUNT * sm_mhz * 1e6
    achieved = 4.0 * evals / len(plans) / (match_launch_ms / 1e3)
    roofline = {"bound": "alu", "achieved": achieved / 1e12, "peak": popc_peak / 1e12,
                "unit": "Tpopc/s", "frac": achieved / popc_peak, "traffic": None,
                "peak_kind": "derived: %d POPC/clk/SM (measured) x %d SMs x %.0f MHz (%s max clock)"
                             % (POPC_PER_CLK_PER_SM, SM_COUNT, sm_mhz, pk_kind),
                "kernel": "k_match", "evals_per_step": evals, "match_ms_per_step": float(np.mean(match_ms))}

    # ---- end to end through the C ABI: host descriptors in, host results out
    e2e_ms = [float("nan")]
    h2d = total * 128
    best_host = torch.empty(n_rows, dtype=torch.int32, pin_memory=True)
    del plans, outs, index
    torch.cuda.empty_cache()
    if args.e2e_steps > 0:
        e2e_ms = []
    for s in range(args.e2e_steps + 1 if args.e2e_steps > 0 else 0):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            ix = cm.Index.build(p, n_desc, host, mem=cm.MEM_HOST, stream=stream)
            off = 0
            for r in rows:
                pl = cm.MatchPlan(ix, pairs[r], stream=stream)
                o = {"best_j": torch.empty(max(pl.rows, 1), dtype=torch.int32, device=dev)}
                pl.run(o, stream)
                best_host[off:off + pl.rows].copy_(o["best_j"][:pl.rows], non_blocking=True)
                off += pl.rows
                pl.close()
        stream.synchronize()
        if s > 0:
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
        ix.close()
        del ix
    e2e_value = n_pairs * world / (np.mean(e2e_ms) / 1e3)

    # ---- plain per-pair form (no schedule): upload both images, hash, match, download, free
    plain = plain_per_pair(args, wl, host, sums, stream, dev) if args.plain_pairs > 0 else None

    # ---- CPU oracle on a bounded sample (rank 0 at N=1): baseline and match agreement
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.oracle_pairs > 0:
        cpu = cpu_baseline_and_agreement(args, wl, host.numpy(), sums, pairs, rows, gpu_rows)

    res = {
        "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8/fp32" if args.rerank == "fp32" else "u8/" + args.rerank,
        "data": "synthetic (seeded track model, %s)" % args.workload,
        "config": {"workload": args.workload, "images": wl.n_images, "pairs": n_pairs,
                   "descriptors": total, "rerank": args.rerank, "algo": args.algo, "projection": args.projection, "L": p.L, "m": p.m, "K": p.K,
                   "ratio": "%d/%d" % (p.ratio_num, p.ratio_den), "block_rows": len(rows),
                   "size_blk": args.block_images, "budget_gb": args.budget_gb,
                   "l2": "inputs (%.1f GB descriptors) larger than L2" % (total * 128 / 1e9),
                   "generate_s": round(gen_s, 1)},
        "e2e": {"value": e2e_value, "unit": "pairs/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": n_rows * 4, "ms_per_step": float(np.mean(e2e_ms))},
        "plain_fp32_per_pair": plain,
        # per step: colsum, mean, hash, bucket, then one match launch per block row
        "gpu_launches": args.steps * (4 + len(rows)),
        "roofline": roofline,
        "clocks": clocks,
    }
    if cpu is not None:
        res["cpu_baseline"] = cpu.pop("cpu_baseline")
        res["agreement"] = cpu
    return res, {"wl": wl, "host": host, "p": p, "stream": stream, "dev": dev}


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


def cpu_baseline_and_agreement(args, wl, desc, sums, pairs, rows, gpu_rows):
    """Times the FP64 oracle (as it stands) on a sample of pairs on all host
    cores and compares its match sets with the GPU's on the same pairs."""
    import oracle
    cores = os.cpu_count() or 1
    rng = np.random.default_rng(0)
    sel = np.sort(rng.choice(len(pairs), min(args.oracle_pairs, len(pairs)), replace=False))
    oix = oracle.Index(desc, wl.n_desc, oracle.Params(), threads=cores, sums=sums, n_total=wl.total_desc)
    t0 = time.perf_counter()
    res = oix.match(pairs[sel])
    dt = time.perf_counter() - t0
    inter = union = same = total = ng = no = 0
    for k, o in zip(sel, res):
        g = gpu_rows[int(k)]
        same += int((g == o["best_j"]).sum())
        total += len(g)
        gm = set(zip(np.nonzero(g >= 0)[0].tolist(), g[g >= 0].tolist()))
        om = set(zip(np.nonzero(o["best_j"] >= 0)[0].tolist(), o["best_j"][o["best_j"] >= 0].tolist()))
        inter += len(gm & om)
        union += len(gm | om)
        ng += len(gm)
        no += len(om)
    return {"cpu_baseline": {"value": len(sel) / dt, "unit": "pairs/s", "cores": cores, "kind": "oracle",
                             "sample": "%d of %d pairs, each: hash both images (FP64) + match; centring sums "
                                       "given" % (len(sel), len(pairs))},
            "pairs_checked": int(len(sel)), "match_set_jaccard": inter / union if union else 1.0,
            "per_query_agreement": same / total if total else 1.0, "gpu_matches": ng, "oracle_matches": no}


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
            "config": {"workload": args.workload}, "impl": "reference",
            "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    rank, world, local = dist_env()
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl" if args.impl == "ours" else "gloo")
    if args.impl == "reference":
        res = run_reference(args, rank, world)
    else:
        res, _ = run_ours(args, rank, world, local)
    if rank == 0 and res is not None:
        print(json.dumps(res))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
