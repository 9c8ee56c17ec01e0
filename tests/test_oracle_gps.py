"""Pins of the scheduler oracle: GPS ordering (Algorithm 2) and the MBR
schedule-block reading of Sec. 2.2 / Sec. 2.3.2."""
import os
import random

import numpy as np
import pytest

from oracle import gps

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.startswith("#") or ":" not in line:
                continue
            k, v = line.split(":", 1)
            out[k.strip()] = v.split()
    return out


def test_hand_worked_path_example():
    g = _golden("gps_path4.txt")
    edges = [tuple(int(x) for x in e.split("-")) for e in g["edges"]]
    order = gps.gps_order(4, edges)
    assert order == [int(x) for x in g["order"]]
    assert gps.bandwidth(order, edges) == int(g["bandwidth"][0])


@pytest.mark.parametrize("n", [2, 5, 40, 300])
def test_shuffled_path_has_bandwidth_one(n):
    ids = list(range(n))
    random.Random(n).shuffle(ids)
    edges = [(ids[k], ids[k + 1]) for k in range(n - 1)]
    order = gps.gps_order(n, edges)
    assert sorted(order) == list(range(n))
    assert gps.bandwidth(order, edges) == 1


@pytest.mark.parametrize("r,c", [(3, 7), (5, 5), (6, 20), (12, 9)])
def test_grid_bandwidth_close_to_short_side(r, c):
    # A 4-connected r x c grid has bandwidth exactly min(r, c); level-structure
    # orderings reach min(r,c) or min(r,c)+1 (diagonal fronts).
    ids = list(range(r * c))
    random.Random(r * 100 + c).shuffle(ids)
    node = lambda x, y: ids[y * c + x]
    edges = []
    for y in range(r):
        for x in range(c):
            if x + 1 < c:
                edges.append((node(x, y), node(x + 1, y)))
            if y + 1 < r:
                edges.append((node(x, y), node(x, y + 1)))
    order = gps.gps_order(r * c, edges)
    bw = gps.bandwidth(order, edges)
    assert min(r, c) <= bw <= min(r, c) + 1
    assert bw <= gps.bandwidth(list(range(r * c)), edges)


def test_disconnected_and_isolated_nodes():
    edges = [(5, 6), (6, 7), (1, 2)]
    order = gps.gps_order(10, edges)
    assert sorted(order) == [1, 2, 5, 6, 7]        # isolated nodes dropped (step (4))
    assert order[:2] in ([1, 2], [2, 1])           # components in order of smallest id


def _check_schedule(pairs, nbytes, budget, rows):
    seen = np.zeros(len(pairs), dtype=int)
    resident = set()
    for row in rows:
        for w in row["load"]:
            assert w not in resident
            resident.add(w)
        assert sum(nbytes[w] for w in resident) <= budget
        for k in row["pairs"]:
            a, b = pairs[k]
            assert a in resident and b in resident
            seen[k] += 1
        for w in row["free"]:
            assert w in resident
            resident.discard(w)
    assert not resident
    assert np.all(seen == 1)


@pytest.mark.parametrize("budget_imgs,blk", [(1000, 400), (40, 10), (12, 4), (6, 3), (2, 1)])
def test_schedule_covers_every_pair_once_within_budget(budget_imgs, blk):
    # 12 x 10 grid, 12-neighbourhood, ordered pairs both ways; images of uneven size
    gx, gy = 12, 10
    rng = np.random.default_rng(budget_imgs)
    nbytes = [int(b) for b in rng.integers(50, 100, size=gx * gy)]
    pairs = []
    for k in range(gx * gy):
        x, y = k % gx, k // gx
        for dx in range(-2, 3):
            for dy in range(-2, 3):
                if 0 < dx * dx + dy * dy <= 4 and 0 <= x + dx < gx and 0 <= y + dy < gy:
                    pairs.append((k, (y + dy) * gx + x + dx))
    budget = budget_imgs * 100
    rows = gps.schedule(pairs, nbytes, budget, blk)
    _check_schedule(pairs, nbytes, budget, rows)
    # MBR iterations shrink the matrix to empty (Sec. 3.3.2, fig. 10)
    its = [r["iteration"] for r in rows]
    assert its == sorted(its)


def test_schedule_rejects_pair_over_budget():
    with pytest.raises(ValueError):
        gps.schedule([(0, 1)], [60, 60], 100, 4)
    with pytest.raises(ValueError):
        gps.schedule([(0, 0)], [10], 100, 4)


def test_single_window_when_budget_holds_everything():
    pairs = [(0, 1), (1, 2), (2, 0), (3, 4)]
    rows = gps.schedule(pairs, [1] * 5, 10 ** 6, 400)
    assert len(rows) == 1 and rows[0]["pairs"] == [0, 1, 2, 3]
    assert sorted(rows[0]["load"]) == [0, 1, 2, 3, 4] and sorted(rows[0]["free"]) == [0, 1, 2, 3, 4]
