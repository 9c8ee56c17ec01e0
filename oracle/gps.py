"""Scheduler oracle: GPS ordering (Algorithm 2) and MBR schedule blocks (Sec. 2.2).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Plain Python, written
for reading, not speed.

Readings where the paper is silent (each is one line of the design notes):

* G1  the graph may be disconnected: each connected component is ordered on
      its own, components in order of their smallest node id, numberings
      concatenated.  Nodes of degree 0 are not part of M_mbr (step (4)).
* G2  "minimum degree" ties are broken by the smallest node id.
* G3  a level structure rooted at r is the BFS layering from r; its depth is
      the index of its last level.
* G4  combined level structure: with k the common depth, node w has the two
      candidate levels i = lev_u(w) and k - lev_v(w); if they agree that is its
      level, otherwise it goes to whichever candidate level holds fewer nodes
      at that moment (ties to i); nodes are placed in ascending id order.
* G5  numbering is level by level; inside level 0 nodes are sorted by
      (degree, id); inside level l > 0 by (smallest number already given to a
      neighbour in level l-1, or +inf; degree; id).
* S1  Size_blk = maximum images per chunk; chunks are consecutive runs of the
      permuted order, closed early if adding an image would exceed half the
      budget, so that any two chunks fit together.
* S2  block row r = the window of consecutive chunks r .. r+l-1 whose bytes fit
      the budget; it takes every unprocessed edge whose lower chunk is r and
      whose upper chunk lies in the window.  Edges farther apart wait for the
      next MBR iteration (step (5)).
* S3  loads of row r = images of the window not yet resident; after row r the
      first chunk is freed (Sec. 2.3.2 step (3)); at the end of an iteration
      every resident image is freed.
* S4  if an iteration places no edge, its remaining edges are scheduled one
      per row (both images loaded, then freed), which always terminates.
* S5  an edge {a, b} carries every input pair (a, b) or (b, a); each input
      pair index appears in exactly one row.
"""
from __future__ import annotations

from collections import defaultdict


def level_structure(adj, root, nodes):
    """BFS levels from `root` restricted to `nodes` (G3)."""
    lev = {root: 0}
    levels = [[root]]
    while True:
        nxt = []
        for x in levels[-1]:
            for y in sorted(adj[x]):
                if y in nodes and y not in lev:
                    lev[y] = len(levels)
                    nxt.append(y)
        if not nxt:
            break
        levels.append(nxt)
    return lev, levels


def pseudo_peripheral_pair(adj, nodes):
    """Algorithm 2, procedure PseudoPeripheralNodeSelection (G2)."""
    deg = {x: len(adj[x]) for x in nodes}
    u = min(nodes, key=lambda x: (deg[x], x))
    lev_u, levels_u = level_structure(adj, u, nodes)
    while True:
        v = min(levels_u[-1], key=lambda x: (deg[x], x))
        lev_v, levels_v = level_structure(adj, v, nodes)
        if len(levels_v) > len(levels_u):
            u, lev_u, levels_u = v, lev_v, levels_v
        else:
            return u, v, lev_u, lev_v, len(levels_u) - 1


def gps_component(adj, nodes):
    """Algorithm 2, procedure GpsOrdering, for one connected component (G4, G5)."""
    if len(nodes) == 1:
        return list(nodes)
    u, v, lev_u, lev_v, k = pseudo_peripheral_pair(adj, nodes)
    size = [0] * (k + 1)
    level = {}
    undecided = []
    for w in sorted(nodes):
        i, j = lev_u[w], k - lev_v[w]
        if i == j:
            level[w] = i
            size[i] += 1
        else:
            undecided.append((w, i, j))
    for w, i, j in undecided:
        c = i if size[i] <= size[j] else j
        level[w] = c
        size[c] += 1
    by_level = defaultdict(list)
    for w in nodes:
        by_level[level[w]].append(w)
    number = {}
    order = []
    for lvl in range(k + 1):
        members = by_level.get(lvl, [])
        if lvl == 0:
            members.sort(key=lambda w: (len(adj[w]), w))
        else:
            def key(w):
                prev = [number[y] for y in adj[w] if y in number and level[y] == lvl - 1]
                return (min(prev) if prev else float("inf"), len(adj[w]), w)
            members.sort(key=key)
        for w in members:
            number[w] = len(order)
            order.append(w)
    return order


def gps_order(n, edges):
    """Permutation (list of node ids, new position -> node) of the non-isolated
    nodes of the undirected graph with `n` nodes and `edges` (G1)."""
    adj = defaultdict(set)
    for a, b in edges:
        if a != b:
            adj[a].add(b)
            adj[b].add(a)
    seen = set()
    order = []
    for s in range(n):
        if s in seen or not adj[s]:
            continue
        comp = set()
        stack = [s]
        while stack:
            x = stack.pop()
            if x in comp:
                continue
            comp.add(x)
            stack.extend(adj[x] - comp)
        seen |= comp
        order += gps_component(adj, comp)
    return order


def bandwidth(order, edges):
    pos = {w: k for k, w in enumerate(order)}
    return max((abs(pos[a] - pos[b]) for a, b in edges), default=0)


def schedule(pairs, image_bytes, budget, max_images_per_block):
    """MBR schedule blocks (Sec. 2.2 steps (1)-(5); Sec. 2.3.2; Algorithm 1).

    Returns a list of rows: dict(iteration, load, free, pairs) where `pairs`
    are indices into the input pair list.  Raises ValueError when one pair
    cannot fit the budget."""
    n = len(image_bytes)
    edge_pairs = defaultdict(list)            # S5
    for k, (a, b) in enumerate(pairs):
        if a == b:
            raise ValueError("pair with i == j")
        e = (min(a, b), max(a, b))
        edge_pairs[e].append(k)
        if image_bytes[a] + image_bytes[b] > budget:
            raise ValueError("pair does not fit the budget")
    remaining = set(edge_pairs)
    rows = []
    it = 0
    while remaining:
        order = gps_order(n, remaining)
        # S1: chunks
        chunks, cur, cur_bytes = [], [], 0
        for w in order:
            b = image_bytes[w]
            if cur and (len(cur) >= max_images_per_block or cur_bytes + b > budget // 2):
                chunks.append(cur)
                cur, cur_bytes = [], 0
            cur.append(w)
            cur_bytes += b
        if cur:
            chunks.append(cur)
        chunk_of = {w: c for c, ch in enumerate(chunks) for w in ch}
        chunk_bytes = [sum(image_bytes[w] for w in ch) for ch in chunks]
        by_lower = defaultdict(list)
        for e in sorted(remaining):
            ca, cb = chunk_of[e[0]], chunk_of[e[1]]
            by_lower[min(ca, cb)].append((max(ca, cb), e))
        resident = []
        placed = 0
        for r in range(len(chunks)):
            hi, tot = r, chunk_bytes[r]                 # S2: window
            while hi + 1 < len(chunks) and tot + chunk_bytes[hi + 1] <= budget:
                hi += 1
                tot += chunk_bytes[hi]
            take = [e for (cu, e) in by_lower.get(r, []) if cu <= hi]
            want = [w for c in range(r, hi + 1) for w in chunks[c]]
            load = [w for w in want if w not in set(resident)]   # S3
            resident += load
            is_last = r == len(chunks) - 1
            free = list(chunks[r]) if not is_last else list(resident)
            resident = [w for w in resident if w not in set(free)]
            pidx = sorted(k for e in take for k in edge_pairs[e])
            rows.append({"iteration": it, "load": load, "free": free, "pairs": pidx})
            for e in take:
                remaining.discard(e)
            placed += len(take)
        if placed == 0:                                  # S4
            for e in sorted(remaining):
                rows.append({"iteration": it, "load": [e[0], e[1]], "free": [e[0], e[1]],
                             "pairs": sorted(edge_pairs[e])})
            remaining.clear()
        it += 1
    return rows
