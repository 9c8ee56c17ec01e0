"""Host-side partition of one matching job over several GPUs (one process per GPU).

Pairs are independent jobs, so a job shards with no device-to-device traffic:

* block rows of the MBR schedule (Sec. 2.2, in GPS order) are cut into
  contiguous ranges, one per rank, balanced by their pairs' query rows; a rank
  makes resident only the images its rows touch (an image needed by two ranks
  is uploaded from the host to both);
* the one exchange is the centring mean: every rank sums the descriptors of
  the images it owns (image i belongs to rank i mod world) as 128 exact
  integers, and an all-reduce (sum) of those 1 KB gives every rank the same
  global sums, bit for bit, whatever the order of the reduction;
* results are gathered on the host.

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
