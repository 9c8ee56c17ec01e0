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
