"""Pins of the SAO oracle (Sec. 2.3.3, Fig. 4) against definitions that do not
share its code: edit distances as shortest paths of single edits (breadth-first
search over strings and over cyclic strings), nearest neighbours from a k-d
tree and from best-first search over the Delaunay graph, and geometric facts
of the score (similarity maps keep every angular order, a mirror reverses it,
one misplaced neighbour costs at most two edits)."""
import heapq
from collections import deque

import numpy as np
import pytest

from oracle import sao

scipy_spatial = pytest.importorskip("scipy.spatial")


# ---------------------------------------------------------------- edit distances
def _bfs_edit(a, b, alphabet, cyclic=False):
    """Fewest single insertions / deletions / substitutions turning a into b;
    for cyclic strings the states are necklaces (a string equals all its
    rotations) and an edit may act at any position of the cycle."""
    def canon(s):
        if not cyclic or not s:
            return tuple(s)
        return min(tuple(s[i:] + s[:i]) for i in range(len(s)))
    limit = max(len(a), len(b)) + 1
    start, goal = canon(list(a)), canon(list(b))
    seen, frontier = {start: 0}, deque([start])
    while frontier:
        s = frontier.popleft()
        if s == goal:
            return seen[s]
        s_l = list(s)
        nxt = []
        for i in range(len(s_l)):
            nxt.append(s_l[:i] + s_l[i + 1:])
            for c in alphabet:
                if c != s_l[i]:
                    nxt.append(s_l[:i] + [c] + s_l[i + 1:])
        if len(s_l) < limit:
            for i in range(len(s_l) + 1):
                for c in alphabet:
                    nxt.append(s_l[:i] + [c] + s_l[i:])
        for t in nxt:
            t = canon(t)
            if t not in seen:
                seen[t] = seen[s] + 1
                frontier.append(t)
    raise AssertionError("unreachable")


def test_levenshtein_textbook_values():
    assert sao.levenshtein("kitten", "sitting") == 3
    assert sao.levenshtein("flaw", "lawn") == 2
    assert sao.levenshtein("", "abc") == 3
    assert sao.levenshtein("abc", "") == 3
    assert sao.levenshtein("abc", "abc") == 0


def test_levenshtein_equals_shortest_edit_path():
    rng = np.random.default_rng(7)
    for _ in range(150):
        a = rng.integers(0, 3, rng.integers(0, 5)).tolist()
        b = rng.integers(0, 3, rng.integers(0, 5)).tolist()
        assert sao.levenshtein(a, b) == _bfs_edit(a, b, (0, 1, 2)), (a, b)


def test_cyclic_edit_distance_equals_shortest_necklace_edit_path():
    rng = np.random.default_rng(8)
    for _ in range(150):
        a = rng.integers(0, 3, rng.integers(0, 5)).tolist()
        b = rng.integers(0, 3, rng.integers(0, 5)).tolist()
        assert sao.cyclic_edit_distance(a, b) == _bfs_edit(a, b, (0, 1, 2), cyclic=True), (a, b)


def test_cyclic_edit_distance_properties():
    rng = np.random.default_rng(9)
    for _ in range(50):
        a = rng.permutation(8).tolist()
        b = rng.permutation(8).tolist()
        r = int(rng.integers(0, 8))
        d = sao.cyclic_edit_distance(a, b)
        assert sao.cyclic_edit_distance(a[r:] + a[:r], b) == d
        assert sao.cyclic_edit_distance(b, a) == d
        assert sao.cyclic_edit_distance(a, a[r:] + a[:r]) == 0
        assert d <= sao.levenshtein(a, b)
    # three distinct labels in the opposite cyclic order: no single edit keeps the multiset
    assert sao.cyclic_edit_distance([0, 1, 2], [2, 1, 0]) == 2
    # disjoint label sets: one substitution per position
    assert sao.cyclic_edit_distance([0, 1, 2, 3], [4, 5, 6, 7]) == 4


# ---------------------------------------------------------------- neighbours
def test_knn_equals_kd_tree():
    rng = np.random.default_rng(10)
    P = rng.uniform(0, 4000, (600, 2)).astype(np.float32).astype(np.float64)
    k = 8
    nb = sao.knn(P, k)
    _, idx = scipy_spatial.cKDTree(P).query(P, k + 1)
    for m in range(len(P)):
        want = [int(x) for x in idx[m] if x != m][:k]
        assert list(nb[m]) == want, m


def test_knn_set_is_found_on_the_delaunay_graph():
    """Best-first search from p over the Delaunay graph, taking the closest
    frontier vertex each time, meets the k nearest neighbours first: the
    neighbour set of Fig. 4 is the Euclidean k-NN set."""
    rng = np.random.default_rng(11)
    P = rng.uniform(0, 1000, (400, 2))
    tri = scipy_spatial.Delaunay(P)
    indptr, adj = tri.vertex_neighbor_vertices
    k = 8
    nb = sao.knn(P, k)
    for m in range(len(P)):
        d2 = lambda v: float(((P[v] - P[m]) ** 2).sum())   # noqa: E731
        heap = [(d2(int(v)), int(v)) for v in adj[indptr[m]:indptr[m + 1]]]
        heapq.heapify(heap)
        seen, got = {m} | {v for _, v in heap}, []
        while heap and len(got) < k:
            _, v = heapq.heappop(heap)
            got.append(v)
            for w in adj[indptr[v]:indptr[v + 1]]:
                if int(w) not in seen:
                    seen.add(int(w))
                    heapq.heappush(heap, (d2(int(w)), int(w)))
        assert got == list(nb[m]), m


def test_knn_ties_by_index_and_small_sets():
    P = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1], [5, 5]], dtype=np.float64)
    nb = sao.knn(P, 3)
    assert list(nb[0]) == [1, 2, 3]           # four at distance 1: lowest indices
    assert [len(x) for x in sao.knn(P[:2], 8)] == [1, 1]
    assert sao.knn(P[:0], 4) == []


def test_angular_order():
    c = (10.0, 20.0)
    pts = np.array([[11, 20], [10, 21], [9, 20], [10, 19], [11, 21], [12, 20], [10, 20]], dtype=np.float64)
    # angles from the +x axis: 0, 90, 180, 270, 45, 0 (same ray as label 0), zero vector = 0
    assert sao.angular_order(c, pts, [0, 1, 2, 3, 4, 5, 6]) == [0, 5, 6, 4, 1, 2, 3]
    assert sao.angular_order(c, pts, [3, 2]) == [2, 3]
    assert sao.angular_order(c, pts, []) == []
    # a ray just below the +x axis comes last, not first
    pts2 = np.array([[11, 20 - 1e-9], [10, 21]], dtype=np.float64)
    assert sao.angular_order(c, pts2, [0, 1]) == [1, 0]


# ---------------------------------------------------------------- scores
def _ids(n):
    return (np.arange(n, dtype=np.uint32) << 16) | np.arange(n, dtype=np.uint32)


def _quantised(rng, n, lo=0, hi=4096):
    # sixteenth-pixel keypoints: integer translations and power-of-two scales stay exact in float32
    return (rng.integers(lo * 16, hi * 16, (n, 2)) / 16.0).astype(np.float32)


def test_similarity_maps_keep_every_order():
    rng = np.random.default_rng(12)
    P = _quantised(rng, 700)
    for Q in (np.stack([-2 * P[:, 1] + 16384, 2 * P[:, 0] - 300], 1),     # rotation 90, scale 2, shift
              np.stack([0.5 * P[:, 0] + 7, 0.5 * P[:, 1] - 9], 1),        # scale 1/2, shift
              -P + 5000):                                                  # rotation 180
        s = sao.sao_scores(P, Q.astype(np.float32), _ids(700), 8)
        assert (s == 0).all()
    # a rotation by an arbitrary angle (rounded keypoints): no near-tie flips on this draw
    th = 0.7
    R = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
    Pf = rng.uniform(0, 4000, (700, 2)).astype(np.float32)
    Q = (Pf.astype(np.float64) @ R.T * 1.3 + [200, -50]).astype(np.float32)
    assert (sao.sao_scores(Pf, Q, _ids(700), 8) == 0).all()


def test_mirror_reverses_the_orders():
    rng = np.random.default_rng(13)
    P = _quantised(rng, 300)
    Q = np.stack([4096 - P[:, 0], P[:, 1]], 1).astype(np.float32)   # reflection: same neighbours, reversed order
    s = sao.sao_scores(P, Q, _ids(300), 8)
    want = np.float32(sao.cyclic_edit_distance(list(range(8)), list(range(7, -1, -1)))) / np.float32(8)
    assert want == np.float32(0.75)     # 8 distinct labels against their reversal: 6 edits
    assert (s == want).all()


def test_one_misplaced_match():
    """Under an exact similarity, one match whose database keypoint is moved
    far away has no neighbour in common (score 1); every other match loses or
    gains at most that one neighbour, which costs at most two edits."""
    rng = np.random.default_rng(14)
    n, k = 500, 8
    P = _quantised(rng, n, 0, 2048)
    Q = (2 * P + 100).astype(np.float32)
    m = int(np.argmin(((P - [200, 200]) ** 2).sum(1)))   # a match near one corner
    Q[m] = [2 * 1900 + 100, 2 * 1900 + 100]              # moved to the opposite corner
    s = sao.sao_scores(P, Q, _ids(n), k)
    assert s[m] == 1.0
    others = np.delete(s, m)
    assert (others <= np.float32(2) / np.float32(k)).all()
    assert (others > 0).sum() >= k                       # its old neighbours noticed


def test_degenerate_sizes():
    rng = np.random.default_rng(15)
    for n in (0, 1, 2, 3):
        P = rng.uniform(0, 100, (n, 2)).astype(np.float32)
        Q = rng.uniform(0, 100, (n, 2)).astype(np.float32)
        s = sao.sao_scores(P, Q, _ids(n), 8)
        assert s.shape == (n,)
        if n <= 3:   # every other match is a neighbour on both sides; two labels have one cyclic order
            assert (s == 0).all()
    s, keep = sao.sao_filter(np.zeros((0, 2), np.float32), np.zeros((0, 2), np.float32), _ids(0))
    assert s.size == 0 and keep.size == 0


def test_many_to_one_matches_share_a_database_keypoint():
    P = np.array([[0, 0], [10, 0], [0, 10], [10, 10], [5, 5]], dtype=np.float32)
    Q = np.array([[0, 0], [10, 0], [0, 10], [10, 10]], dtype=np.float32)
    mt = np.array([(0 << 16) | 0, (1 << 16) | 1, (2 << 16) | 2, (3 << 16) | 3, (4 << 16) | 3], dtype=np.uint32)
    s = sao.sao_scores(P, Q, mt, 3)
    assert s.shape == (5,) and np.isfinite(s).all()
    # matches 3 and 4 sit on the same database keypoint: each is the other's nearest there
    assert (s >= 0).all() and (s <= 1).all()
