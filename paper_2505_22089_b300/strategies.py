"""Data-schedule strategies other than the MBR blocks, as schedule rows for
cm_schedule_from_rows, so that every strategy runs through the same pipeline
call (cm_run_schedule) and is measured the same way (Sec. 2.2 and the
strategies the paper compares in Sec. 4: one pair at a time, blocks of pairs
fed without regard to image connections, images fed in connection order with
a load/free list, and graph partitions with a pre-defined vertex count).

Each function returns rows [{"load": [...], "free": [...], "pairs": [...]}]
over the pair indices of `pairs`; a row loads only images that are not
resident and frees only resident ones, and the resident set never exceeds
`budget` bytes (image_bytes[i] per image).  Host logic only.
"""
from __future__ import annotations

from collections import OrderedDict, defaultdict

import numpy as np


def _pairs(pairs) -> np.ndarray:
    return np.asarray(pairs, dtype=np.int64).reshape(-1, 2)


def per_pair(pairs) -> list:
    """No schedule: each pair loads its two images, is matched alone, frees them."""
    P = _pairs(pairs)
    return [{"load": [int(i), int(j)], "free": [int(i), int(j)], "pairs": [k]} for k, (i, j) in enumerate(P)]


def pair_blocks(pairs, image_bytes, budget: int) -> list:
    """Blocks of consecutive input pairs whose images fit the budget together,
    each fed at once (load the block's images, match, free them all), with no
    regard to which images the next block shares."""
    P = _pairs(pairs)
    ib = np.asarray(image_bytes, dtype=np.int64)
    rows, cur, imgs, used = [], [], [], 0
    for k, (i, j) in enumerate(P):
        need = [x for x in dict.fromkeys((int(i), int(j))) if x not in imgs]
        add = int(sum(ib[x] for x in need))
        if cur and used + add > budget:
            rows.append({"load": imgs, "free": list(imgs), "pairs": cur})
            cur, imgs, used = [], [], 0
            need = list(dict.fromkeys((int(i), int(j))))
            add = int(sum(ib[x] for x in need))
        imgs = imgs + need
        used += add
        cur.append(k)
    if cur:
        rows.append({"load": imgs, "free": list(imgs), "pairs": cur})
    return rows


def connection_order(pairs, n_images: int, order_fn) -> list:
    """Images in the order of their connections (order_fn: GPS ordering of the
    symmetrised pair graph), images without pairs appended."""
    P = _pairs(pairs)
    e = sorted({(min(int(i), int(j)), max(int(i), int(j))) for i, j in P})
    order = list(order_fn(n_images, e)) if e else []
    rest = sorted(set(range(n_images)) - set(order))
    return order + rest


def load_free_list(pairs, image_bytes, budget: int, order) -> list:
    """Images fed in connection order, one pair matched at a time: pairs sorted
    by the positions of their images in `order` (lower, then upper); a missing
    image is loaded, and while the budget is exceeded the least recently used
    resident image not needed by the pair is freed."""
    P = _pairs(pairs)
    ib = np.asarray(image_bytes, dtype=np.int64)
    pos = {int(im): n for n, im in enumerate(order)}
    ks = sorted(range(len(P)), key=lambda k: (min(pos[int(P[k, 0])], pos[int(P[k, 1])]),
                                              max(pos[int(P[k, 0])], pos[int(P[k, 1])]), k))
    res = OrderedDict()   # image -> None, least recently used first
    used = 0
    rows = []
    for k in ks:
        i, j = int(P[k, 0]), int(P[k, 1])
        need = [x for x in dict.fromkeys((i, j)) if x not in res]
        free = []
        while res and used + sum(int(ib[x]) for x in need) > budget:
            victim = next((x for x in res if x not in (i, j)), None)
            if victim is None:
                break
            del res[victim]
            used -= int(ib[victim])
            free.append(victim)
        if free:   # frees are issued after the previous row, before this row's loads
            if rows:
                rows[-1]["free"] += free
            else:
                raise AssertionError("nothing resident to free before the first row")
        for x in need:
            res[x] = None
            used += int(ib[x])
        res.move_to_end(i)
        res.move_to_end(j)
        rows.append({"load": need, "free": [], "pairs": [k]})
    if rows:
        rows[-1]["free"] += list(res)
    return rows


def graph_partition(pairs, image_bytes, budget: int, order, part_images: int) -> list:
    """The view graph split into sub-graphs of `part_images` consecutive images
    of `order`; part a is loaded and its internal pairs matched; then, for each
    later part b sharing pairs with a, b is loaded, the pairs between a and b
    are matched and b is freed; then a is freed.  Two parts must fit the budget."""
    P = _pairs(pairs)
    ib = np.asarray(image_bytes, dtype=np.int64)
    part = {}
    parts = [list(order[s:s + part_images]) for s in range(0, len(order), part_images)]
    for a, members in enumerate(parts):
        for im in members:
            part[int(im)] = a
    by = defaultdict(list)
    for k, (i, j) in enumerate(P):
        a, b = part[int(i)], part[int(j)]
        by[(min(a, b), max(a, b))].append(k)
    largest = max((int(sum(ib[x] for x in m)) for m in parts), default=0)
    if 2 * largest > budget and len(parts) > 1:
        raise ValueError("two partitions of %d images exceed the budget" % part_images)
    rows = []
    for a, members in enumerate(parts):
        later = sorted(b for (x, b) in by if x == a and b != a)
        if not by.get((a, a)) and not later:
            continue
        rows.append({"load": [int(x) for x in members], "free": [], "pairs": list(by.get((a, a), []))})
        for b in later:
            rows.append({"load": [int(x) for x in parts[b]], "free": [int(x) for x in parts[b]],
                         "pairs": list(by[(a, b)])})
        rows[-1]["free"] += [int(x) for x in members]
    return rows


def residency(rows, image_bytes) -> dict:
    """Replays a row list: rows, image loads, rows with pairs (launches) and the
    peak resident bytes."""
    ib = np.asarray(image_bytes, dtype=np.int64)
    res, used, peak, loads = set(), 0, 0, 0
    for r in rows:
        for x in r["load"]:
            res.add(x)
            used += int(ib[x])
            loads += 1
        peak = max(peak, used)
        for x in r["free"]:
            res.discard(x)
            used -= int(ib[x])
    return {"rows": len(rows), "loads": loads, "peak_resident_bytes": int(peak),
            "launches": sum(1 for r in rows if r["pairs"])}
