"""Oracle of the spatial-angular-order (SAO) local geometric constraint
(Sec. 2.3.3, Fig. 4): a dissimilarity score per initial match from the cyclic
edit distance between the angular orders of its neighbours in the two images.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Plain numpy and Python
loops, written for reading, not speed; every step is the plain definition.

Readings where the paper is silent (each is one line of the design notes):

* O1  neighbours of match m: in the query image, the k nearest neighbours of
      its keypoint p_m among the query keypoints of the pair's other initial
      matches; in the database image, independently, the k nearest neighbours
      of q_m among their database keypoints (squared Euclidean distance in
      FP64, ties by match index).  Both are labelled by match index, so a
      neighbour that is near p_m but whose partner is not near q_m (or the
      reverse) costs edits.  The paper derives the neighbours from the
      Delaunay triangulation; the Delaunay graph is the structure in which the
      k nearest neighbours are found (each one is adjacent to p_m or to a
      closer neighbour), so the set is the Euclidean k-NN set.
* O2  angular order: the neighbours sorted by the angle of p_n - p_m (of
      q_n - q_m for O_q) from the horizontal axis, in [0, 2*pi), ties by match
      index; a zero vector has angle 0.  Where the sequence starts does not
      matter: the distance is cyclic.
* O3  d_ced: the cyclic edit distance, the smallest unit-cost Levenshtein
      distance over all rotations of both sequences.
* O4  N = the number of neighbours found, min(k, n - 1); Score = d_ced / N
      (float32); N = 0 gives Score 0.
* O5  a match is kept when Score <= tau; one pass over the initial matches
      (neighbours are taken among all initial matches, not the survivors).
      Defaults: k = 8, tau = 0.875 (a match is dropped only when at most one
      of its 8 neighbours keeps its place in the angular order): on planted
      affine pairs with 1 px noise this drops about 94 % of random outliers
      and keeps about 99 % of inliers at a 50 % outlier share.
"""
from __future__ import annotations

import numpy as np


def levenshtein(a, b) -> int:
    """Unit-cost edit distance (insert, delete, substitute) by the textbook
    dynamic programme over prefixes."""
    n, m = len(a), len(b)
    prev = list(range(m + 1))
    for i in range(1, n + 1):
        cur = [i] + [0] * m
        for j in range(1, m + 1):
            cur[j] = min(prev[j] + 1, cur[j - 1] + 1, prev[j - 1] + (0 if a[i - 1] == b[j - 1] else 1))
        prev = cur
    return prev[m]


def cyclic_edit_distance(a, b) -> int:
    """O3: min over every rotation of a and every rotation of b."""
    a, b = list(a), list(b)
    if not a or not b:
        return levenshtein(a, b)
    return min(levenshtein(a[i:] + a[:i], b[j:] + b[:j]) for i in range(len(a)) for j in range(len(b)))


def knn(pts: np.ndarray, k: int):
    """O1: for each point, the indices of its k nearest other points, nearest
    first, by (squared distance, index)."""
    n = len(pts)
    P = np.asarray(pts, dtype=np.float64)
    out = []
    for m in range(n):
        dx = P[:, 0] - P[m, 0]
        dy = P[:, 1] - P[m, 1]
        d2 = dx * dx + dy * dy
        idx = np.arange(n)
        keep = idx != m
        order = np.lexsort((idx[keep], d2[keep]))
        out.append(idx[keep][order][:k])
    return out


def angular_order(center, pts: np.ndarray, labels) -> list:
    """O2: the labels sorted by the angle of pts[label] - center in [0, 2*pi),
    ties by label."""
    P = np.asarray(pts, dtype=np.float64)
    c = np.asarray(center, dtype=np.float64)
    lab = np.asarray(labels, dtype=np.int64)
    if len(lab) == 0:
        return []
    ang = np.arctan2(P[lab, 1] - c[1], P[lab, 0] - c[0])
    ang = np.where(ang < 0, ang + 2 * np.pi, ang)
    return lab[np.lexsort((lab, ang))].tolist()


def sao_scores(kp_i: np.ndarray, kp_j: np.ndarray, matches: np.ndarray, k: int = 8) -> np.ndarray:
    """Score of every initial match (O4).  matches[m] = query << 16 | database
    index; kp_i / kp_j: float32 [n][2] keypoints of the two images."""
    mt = np.asarray(matches, dtype=np.uint32)
    q = (mt >> 16).astype(np.int64)
    j = (mt & 0xFFFF).astype(np.int64)
    P = np.asarray(kp_i, dtype=np.float32)[q].astype(np.float64)
    Q = np.asarray(kp_j, dtype=np.float32)[j].astype(np.float64)
    nb_p, nb_q = knn(P, k), knn(Q, k)
    score = np.zeros(len(mt), dtype=np.float32)
    for m in range(len(mt)):
        N = len(nb_p[m])
        if N == 0:
            continue
        d = cyclic_edit_distance(angular_order(P[m], P, nb_p[m]), angular_order(Q[m], Q, nb_q[m]))
        score[m] = np.float32(d) / np.float32(N)
    return score


def sao_filter(kp_i, kp_j, matches, k: int = 8, tau: float = 0.875):
    """O5: (scores, keep mask)."""
    s = sao_scores(kp_i, kp_j, matches, k)
    return s, s <= np.float32(tau)
