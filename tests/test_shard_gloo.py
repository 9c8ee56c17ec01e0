"""Multi-rank sharding of one job, run as world-size-2 gloo process groups on CPU.

Each rank takes a contiguous range of MBR block rows, contributes the exact
column sums of the images it owns to the one all-reduce (the centring mean),
matches its rows' pairs and sends its results to rank 0.  The matcher here is
the FP64 oracle (CPU); the test checks the host logic: every pair is matched
exactly once, the reduced sums equal the single-process sums bit for bit, and
the gathered results equal the single-process run."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import paper_2505_22089_b300 as cm  # noqa: E402
import synth  # noqa: E402
from paper_2505_22089_b300 import shard  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _job():
    wl = synth.scaled("grid500", gx=4, gy=3, nmin=300, nmax=700)
    p = cm.Params.make()
    sched = cm.schedule_blocks(wl.pairs, wl.n_desc, p, budget=1 << 30, max_images_per_block=4)
    rows = [r["pairs"] for r in sched.rows]
    return wl, rows


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl, rows = _job()
    desc = wl.generate(threads=1)
    off = wl.row_off
    mine = shard.owned_images(wl.n_images, rank, world)
    local = np.zeros(128, np.uint64)
    n_local = 0
    for i in mine:
        local += desc[off[i]:off[i + 1]].astype(np.uint64).sum(0)
        n_local += int(wl.n_desc[i])
    sums, n_total = shard.global_col_sums(local, n_local)
    a, b = shard.row_ranges(shard.row_weights(rows, wl.pairs, wl.n_desc), world)[rank]
    ids = [k for r in rows[a:b] for k in r]
    oix = oracle.Index(desc, wl.n_desc, oracle.Params(), threads=1, sums=sums, n_total=n_total)
    res = oix.match(wl.pairs[np.asarray(ids, dtype=np.int64)]) if ids else []
    payload = {int(k): r["best_j"] for k, r in zip(ids, res)}
    gathered = [None] * world
    dist.all_gather_object(gathered, (rank, sums.tolist(), n_total, payload))
    if rank == 0:
        np.save(os.path.join(out_dir, "gathered.npy"), np.array(gathered, dtype=object), allow_pickle=True)
    dist.destroy_process_group()


def test_row_ranges_cover_contiguously():
    w = np.array([5, 0, 7, 3, 3, 9, 1, 0, 2])
    for world in (1, 2, 3, 4, 12):
        rg = shard.row_ranges(w, world)
        assert len(rg) == world and rg[0][0] == 0 and rg[-1][1] == len(w)
        assert all(rg[k][1] == rg[k + 1][0] for k in range(world - 1))
        loads = [int(w[a:b].sum()) for a, b in rg]
        assert sum(loads) == int(w.sum())
        if world == 2:
            assert max(loads) - min(loads) <= int(w.max())


def test_two_gloo_ranks_match_the_single_process_run(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    gathered = np.load(tmp_path / "gathered.npy", allow_pickle=True)
    wl, rows = _job()
    desc = wl.generate(threads=1)
    want_sums = desc.astype(np.uint64).sum(0)
    seen = {}
    for rank, sums, n_total, payload in gathered:
        assert np.array_equal(np.asarray(sums, np.uint64), want_sums)
        assert n_total == wl.total_desc
        for k, v in payload.items():
            assert k not in seen, "pair %d matched twice" % k
            seen[k] = v
    assert sorted(seen) == list(range(len(wl.pairs)))
    oix = oracle.Index(desc, wl.n_desc, oracle.Params(), threads=4)
    ref = oix.match(wl.pairs)
    for k, r in enumerate(ref):
        assert np.array_equal(seen[k], r["best_j"])


class _CpuEngine:
    """A stand-in for the bench's GPU engine with the same interface: exact
    column sums in numpy, the mean from the all-reduced sums, and the FP64
    oracle as the matcher of the rank's rows.  It lets the bench's sharded
    orchestration (schedule, partition, the one all-reduce, timing max over
    ranks, checksum and count combination) run on CPU ranks."""

    def __init__(self, args, wl, p, part):
        self.wl, self.part = wl, part
        self.desc = wl.generate(threads=1)
        off = wl.row_off
        self.local = np.zeros(128, np.uint64)
        for i in part["owned"]:
            self.local += self.desc[off[i]:off[i + 1]].astype(np.uint64).sum(0)
        self.rows = [r for r in part["rows"] if len(r)]
        self.res = None
        self.h2d_bytes = 0

    def local_sums(self):
        return torch.tensor(self.local.astype(np.int64))

    def apply_mean(self, sums, n_total):
        self.sums, self.n_total = sums.numpy().astype(np.uint64), n_total

    def match(self):
        oix = oracle.Index(self.desc, self.wl.n_desc, oracle.Params(), threads=1, sums=self.sums,
                           n_total=self.n_total)
        self.res = [oix.match(self.wl.pairs[r]) for r in self.rows]

    def timer(self):
        import time

        class T:
            def __enter__(s):
                s.t0 = time.perf_counter()
                return s

            def __exit__(s, *a):
                s.ms = (time.perf_counter() - s.t0) * 1e3
        return T()

    def sync(self):
        pass

    def upload(self):
        pass

    def download(self):
        return 0

    def launches(self, p):
        return 0

    def results(self):
        out, n = [], 0
        for r, rr in zip(self.rows, self.res):
            nd = self.wl.n_desc[self.wl.pairs[r][:, 0]].astype(np.int64)
            ro = np.concatenate([[0], np.cumsum(nd)])
            b = np.concatenate([x["best_j"] for x in rr]) if rr else np.zeros(0, np.int32)
            out.append((r, ro, b))
            n += int((b >= 0).sum())
        return out, n

    def scalar(self, v):
        return torch.tensor([float(v)], dtype=torch.float64)


def _bench_rank(rank, world, port, out_dir):
    import argparse
    import json
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    args = argparse.Namespace(workload="grid500", grid="4x3", rerank="fp32", algo="auto", projection="tc", K=8,
                              budget_gb=0.004, block_images=4, steps=1, warmup=1, e2e_steps=1,
                              workload_kw=dict(nmin=300, nmax=700))
    res = bench.run_sharded(args, rank, world, _CpuEngine)
    if rank == 0:
        with open(os.path.join(out_dir, "res%d.json" % world), "w") as f:
            json.dump(res, f)
    dist.destroy_process_group()


def test_bench_sharded_path_with_a_cpu_engine(tmp_path):
    """bench.run_sharded on 2 gloo ranks and on 1: every pair matched once,
    the same decision checksum and match count as the single run and as the
    oracle over the whole job, strong-scaling JSON keys."""
    import json
    import torch.multiprocessing as mp
    from paper_2505_22089_b300 import shard
    for world in (1, 2):
        mp.spawn(_bench_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    r1 = json.load(open(tmp_path / "res1.json"))
    r2 = json.load(open(tmp_path / "res2.json"))
    assert r2["n_gpus"] == 2 and r2["scaling"] == "strong" and r2["value"] > 0 and r2["ms_per_step"] > 0
    assert r2["decision_checksum"] == r1["decision_checksum"] and r2["matches"] == r1["matches"]
    assert sum(sh["pairs"] for sh in r2["shards"]) == r2["config"]["pairs"]
    assert all(sh["pairs"] > 0 for sh in r2["shards"])
    wl = synth.grid500(gx=4, gy=3, nmin=300, nmax=700)
    desc = wl.generate(threads=1)
    oix = oracle.Index(desc, wl.n_desc, oracle.Params(), threads=4)
    ref = oix.match(wl.pairs)
    ro = np.concatenate([[0], np.cumsum(wl.n_desc[wl.pairs[:, 0]].astype(np.int64))])
    b = np.concatenate([x["best_j"] for x in ref])
    assert shard.checksum(np.arange(len(wl.pairs)), ro, b) == r2["decision_checksum"]
    assert int((b >= 0).sum()) == r2["matches"]
