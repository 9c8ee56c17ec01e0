"""Oracle of VLAD image encoding, the retrieval front end that builds the view
graph (Sec. 2.1, Fig. 2a; Algorithm 1's codebook and retrieval steps).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  numpy, integers and
FP64, every step the plain definition.

Readings where the paper is silent (each is one line of the design notes):

* VL1  the codebook is an input: C codewords on the descriptors' integer grid
       (uint8 [C][128], e.g. k-means centroids rounded to integers).  Training
       the codebook is outside the encoding path.
* VL2  each descriptor is assigned to its nearest codeword by exact squared
       Euclidean distance on the integers; ties go to the smaller codeword index.
* VL3  the raw VLAD of an image is, per codeword c, the sum over the image's
       descriptors assigned to c of (x - c), concatenated codeword-major
       (C x 128 integers).
* VL4  normalisation: signed square root of every component, then L2
       normalisation of the whole vector; an all-zero vector stays zero.
"""
from __future__ import annotations

import numpy as np


def assign(desc: np.ndarray, codebook: np.ndarray) -> np.ndarray:
    """VL2: index of the nearest codeword of every descriptor (int64)."""
    X = np.asarray(desc, dtype=np.int64)
    Cb = np.asarray(codebook, dtype=np.int64)
    out = np.empty(len(X), dtype=np.int64)
    step = max(1, (1 << 23) // max(1, Cb.size))   # rows per block: ~8 M differences at a time
    for r0 in range(0, len(X), step):
        Xr = X[r0:r0 + step]
        d2 = ((Xr[:, None, :] - Cb[None, :, :]) ** 2).sum(-1)   # exact integers
        out[r0:r0 + len(Xr)] = np.argmin(d2, axis=1)            # first minimum: the smaller index
    return out


def raw_vlad(desc: np.ndarray, codebook: np.ndarray, a: np.ndarray | None = None) -> np.ndarray:
    """VL3: int64 [C][128] residual sums of one image."""
    X = np.asarray(desc, dtype=np.int64)
    Cb = np.asarray(codebook, dtype=np.int64)
    if a is None:
        a = assign(X, Cb)
    v = np.zeros(Cb.shape, dtype=np.int64)
    for c in range(len(Cb)):
        mine = X[a == c]
        if len(mine):
            v[c] = (mine - Cb[c]).sum(0)
    return v


def normalise(v: np.ndarray) -> np.ndarray:
    """VL4: signed square root, then L2 normalisation (FP64)."""
    s = np.sign(v) * np.sqrt(np.abs(np.asarray(v, dtype=np.float64)))
    n = np.sqrt((s * s).sum())
    return s / n if n > 0 else s


def encode(desc: np.ndarray, n_desc, codebook: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """VLAD of every image of a concatenated descriptor array: (vlad FP64
    [n_images][C * 128], assignment per row)."""
    nd = np.asarray(n_desc, dtype=np.int64)
    off = np.concatenate([[0], np.cumsum(nd)])
    a = assign(desc, codebook)
    out = np.zeros((len(nd), codebook.shape[0] * codebook.shape[1]), dtype=np.float64)
    for i in range(len(nd)):
        v = raw_vlad(desc[off[i]:off[i + 1]], codebook, a[off[i]:off[i + 1]])
        out[i] = normalise(v).reshape(-1)
    return out, a
