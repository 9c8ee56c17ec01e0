"""Host-side partition of one matching job over several GPUs (one process per GPU).

Pairs are independent jobs, so a job shards with no device-to-device traffic:

* the pairs of the MBR schedule's block rows (Sec. 2.2, in GPS order) are cut
  into contiguous ranges, one per rank, balanced by their query rows; a rank
  makes resident only the images its pairs touch (an image needed by two
  ranks is uploaded from the host to both);
* the one exchange is the centring mean: every rank sums the descriptors of
  the images it owns as 128 exact integers, and an all-reduce (sum) of those
  1 KB gives every rank the same global sums, bit for bit, whatever the order
  of the reduction;
* results are combined on the host: each rank reduces its pairs' match lists
  to an order-independent checksum and a match count, and the ranks' values
  are summed, so a sharded run can be compared with a single-GPU run of the
  same job.

These helpers hold no matching arithmetic; they run with any torch.distributed
backend (gloo on CPU in the tests, NCCL between GPUs).
"""
from __future__ import annotations

import numpy as np


def row_weights(rows, pairs, n_desc) -> np.ndarray:
    """Work of each block row: the sum of N_i (query rows) over its pairs."""
    nd = np.asarray(n_desc, dtype=np.int64)
    pr = np.asarray(pairs).reshape(-1, 2)
    return np.array([int(nd[pr[np.asarray(r, dtype=np.int64), 0]].sum()) if len(r) else 0 for r in rows],
                    dtype=np.int64)


def row_ranges(weights, world: int) -> list:
    """Contiguous ranges [a, b) of rows, one per rank, cut where the running
    work crosses k / world of the total (every rank gets a range, maybe empty)."""
    w = np.asarray(weights, dtype=np.int64)
    total = int(w.sum())
    cum = np.concatenate([[0], np.cumsum(w)])
    cuts = [0]
    for k in range(1, world):
        target = total * k / world
        cuts.append(int(np.searchsorted(cum, target, side="left")))
    cuts.append(len(w))
    cuts = [min(max(c, cuts[i - 1] if i else 0), len(w)) for i, c in enumerate(cuts)]
    return [(cuts[k], cuts[k + 1]) for k in range(world)]


def images_of_rows(rows, pairs, a: int, b: int) -> list:
    """Images that rows [a, b) touch, ascending."""
    pr = np.asarray(pairs).reshape(-1, 2)
    ids = set()
    for r in rows[a:b]:
        if len(r):
            ids.update(pr[np.asarray(r, dtype=np.int64)].reshape(-1).tolist())
    return sorted(ids)


def owned_images(n_images: int, rank: int, world: int) -> np.ndarray:
    return np.arange(rank, n_images, world, dtype=np.int64)


def global_col_sums(local_sums, local_rows: int, group=None):
    """All-reduce (sum) of exact per-rank column sums and row counts."""
    import torch
    import torch.distributed as dist
    t = torch.tensor(np.concatenate([np.asarray(local_sums, dtype=np.int64), [int(local_rows)]]),
                     dtype=torch.int64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    v = t.numpy()
    return v[:128].astype(np.uint64), int(v[128])


def plan(rows, pairs, n_images: int, rank: int, world: int, n_desc) -> dict:
    """One rank's share of a job.  The block rows' pairs, in row order (the
    GPS band order), are cut into `world` contiguous ranges balanced by their
    query rows (a block row may be split between two ranks: 13 block rows do
    not divide evenly over 8 GPUs); a rank's pairs keep their row grouping,
    one plan per row.  It makes resident the images its pairs touch plus the
    images it owns, and contributes the column sums of the images it owns.
    Every image is owned by exactly one rank: the lowest rank whose pairs
    touch it, else rank i mod world (an image no pair names still counts in
    the mean)."""
    pr = np.asarray(pairs).reshape(-1, 2)
    nd = np.asarray(n_desc, dtype=np.int64)
    seq = [(r, int(k)) for r, row in enumerate(rows) for k in row]
    w = np.array([nd[pr[k, 0]] for _, k in seq], dtype=np.int64)
    ranges = row_ranges(w, world)
    touched = []
    for a, b in ranges:
        ids = set()
        for _, k in seq[a:b]:
            ids.update(pr[k].tolist())
        touched.append(ids)
    owner = np.full(n_images, -1, dtype=np.int64)
    for r in range(world):
        for i in sorted(touched[r]):
            if owner[i] < 0:
                owner[i] = r
    free = owner < 0
    owner[free] = np.arange(n_images, dtype=np.int64)[free] % world
    owned = np.nonzero(owner == rank)[0]
    a, b = ranges[rank]
    mine = {}
    for r, k in seq[a:b]:
        mine.setdefault(r, []).append(k)
    return {"range": (a, b), "rows": [np.asarray(mine[r], dtype=np.int64) for r in sorted(mine)],
            "owned": owned.astype(np.int64),
            "resident": np.array(sorted(touched[rank] | set(owned.tolist())), dtype=np.int64),
            "ranges": ranges}


_M61 = (1 << 61) - 1


def checksum(pair_ids, row_off, best_j) -> int:
    """Order-independent checksum of decisions: the sum, modulo 2^61 - 1, of a
    mixing hash of (pair, query, database index) over every match.  best_j is
    the concatenated per-query output of pairs pair_ids, pair k's queries at
    rows row_off[k] .. row_off[k + 1] - 1.  Sums of checksums of disjoint sets
    of pairs combine in any order, so ranks' values add up to the value a
    single run of the whole job gives."""
    b = np.asarray(best_j, dtype=np.int64)
    ro = np.asarray(row_off, dtype=np.int64)
    rows = np.nonzero(b >= 0)[0]
    if not len(rows):
        return 0
    k = np.searchsorted(ro, rows, side="right") - 1
    pid = np.asarray(pair_ids, dtype=np.uint64)[k]
    q = (rows - ro[k]).astype(np.uint64)
    with np.errstate(over="ignore"):
        x = pid * np.uint64(0x9E3779B97F4A7C15) ^ (q << np.uint64(20)) ^ b[rows].astype(np.uint64)
        x = (x ^ (x >> np.uint64(31))) * np.uint64(0xBF58476D1CE4E5B9)
        x = x ^ (x >> np.uint64(29))
    x = x % np.uint64(_M61)
    hi, lo = (x >> np.uint64(32)).astype(np.int64), (x & np.uint64(0xFFFFFFFF)).astype(np.int64)
    return (int(hi.sum()) * (1 << 32) + int(lo.sum())) % _M61
