"""FP64 CPU oracle for cascade-hashing feature matching.

TEST INFRASTRUCTURE ONLY: the product path never imports this package.  Only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference legs
of ``bench.py`` use it.  It shares no code with the CUDA library.

The arithmetic lives in ``oracle.c`` (plain C, FP64); this module compiles it,
marshals numpy arrays and runs independent images / pairs on host threads
(ctypes releases the GIL during each call).  ``gps.py`` holds the scheduler
oracle (Algorithm 2 and the schedule-block reading of Sec. 2.2).

Parity status: every function is pinned by tests under ``tests/`` against
properties fixed by the paper and by mathematics (see the test files).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
D = 128


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/liboracle.so (no fast-math: FP64 as written)."""
    src = os.path.join(_HERE, "oracle.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class _Image(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("desc", ctypes.c_void_p), ("keys", ctypes.c_void_p),
                ("code", ctypes.c_void_p), ("off", ctypes.c_void_p), ("idx", ctypes.c_void_p)]


class _Params(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("m", ctypes.c_int32), ("nbits", ctypes.c_int32), ("K", ctypes.c_int32),
                ("ratio_num", ctypes.c_int32), ("ratio_den", ctypes.c_int32)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        vp, i32, i64, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
        lib.orc_splitmix64_first.restype = u64
        lib.orc_splitmix64_first.argtypes = [u64]
        lib.orc_weights.argtypes = [u64, i32, vp]
        lib.orc_col_sums.argtypes = [vp, i64, vp]
        lib.orc_hash_centred.argtypes = [vp, i64, vp, i32, i32, i32, vp, vp, vp]
        lib.orc_hash.argtypes = [vp, i64, vp, vp, i32, i32, i32, vp, vp, vp]
        lib.orc_buckets.argtypes = [vp, i32, i32, i32, vp, vp]
        lib.orc_match_pair.restype = i64
        lib.orc_match_pair.argtypes = [ctypes.POINTER(_Image), ctypes.POINTER(_Image), ctypes.POINTER(_Params),
                                       i32, i32, vp, vp, vp, vp, vp]
        lib.orc_brute_nn.argtypes = [vp, i32, vp, i32, i32, i32, vp, vp, vp]
        _lib = lib
    return _lib


@dataclass(frozen=True)
class Params:
    """Cascade-hashing parameters (paper defaults, Sec. 2.3.1: L=6, m=8, n=128, K=8)."""
    L: int = 6
    m: int = 8
    nbits: int = 128
    K: int = 8
    ratio_num: int = 4     # t_r = 4/5 = 0.8
    ratio_den: int = 5
    seed: int = 0x5EED

    @property
    def P(self) -> int:
        return self.L * self.m + self.nbits


def _p(a):
    return a.ctypes.data if a is not None else None


def splitmix64_first(seed: int) -> int:
    return int(_load().orc_splitmix64_first(seed))


def weights(p: Params) -> np.ndarray:
    """W[128][P] float32 (readings R1, R2 of oracle.c)."""
    W = np.empty((D, p.P), dtype=np.float32)
    _load().orc_weights(p.seed, p.P, _p(W))
    return W


def col_sums(desc: np.ndarray) -> np.ndarray:
    desc = np.ascontiguousarray(desc, dtype=np.uint8).reshape(-1, D)
    s = np.zeros(D, dtype=np.uint64)
    _load().orc_col_sums(_p(desc), desc.shape[0], _p(s))
    return s


def mean_from_sums(sums: np.ndarray, n_total: int) -> np.ndarray:
    """mu = sums / N_total in FP64 (reading R3)."""
    return sums.astype(np.float64) / float(n_total)


def hash_centred(xc: np.ndarray, W: np.ndarray, p: Params, marginal: bool = True):
    xc = np.ascontiguousarray(xc, dtype=np.float64).reshape(-1, D)
    n = xc.shape[0]
    keys = np.empty((n, p.L), dtype=np.uint8)
    code = np.empty((n, p.nbits // 32), dtype=np.uint32)
    marg = np.empty((n, p.P), dtype=np.uint8) if marginal else None
    _load().orc_hash_centred(_p(xc), n, _p(np.ascontiguousarray(W, dtype=np.float32)), p.L, p.m, p.nbits,
                             _p(keys), _p(code), _p(marg))
    return keys, code, marg


def hash_desc(desc: np.ndarray, mu: np.ndarray, W: np.ndarray, p: Params, marginal: bool = True):
    desc = np.ascontiguousarray(desc, dtype=np.uint8).reshape(-1, D)
    n = desc.shape[0]
    keys = np.empty((n, p.L), dtype=np.uint8)
    code = np.empty((n, p.nbits // 32), dtype=np.uint32)
    marg = np.empty((n, p.P), dtype=np.uint8) if marginal else None
    _load().orc_hash(_p(desc), n, _p(np.ascontiguousarray(mu, dtype=np.float64)),
                     _p(np.ascontiguousarray(W, dtype=np.float32)), p.L, p.m, p.nbits, _p(keys), _p(code),
                     _p(marg))
    return keys, code, marg


def buckets(keys: np.ndarray, p: Params):
    keys = np.ascontiguousarray(keys, dtype=np.uint8)
    n = keys.shape[0]
    off = np.empty((p.L, (1 << p.m) + 1), dtype=np.int32)
    idx = np.empty((p.L, n), dtype=np.int32)
    _load().orc_buckets(_p(keys), n, p.L, p.m, _p(off), _p(idx))
    return off, idx


@dataclass
class HashedImage:
    desc: np.ndarray
    keys: np.ndarray
    code: np.ndarray
    off: np.ndarray
    idx: np.ndarray
    marginal: np.ndarray | None = None

    @property
    def n(self) -> int:
        return int(self.desc.shape[0])

    def _c(self) -> _Image:
        return _Image(self.n, _p(self.desc), _p(self.keys), _p(self.code), _p(self.off), _p(self.idx))


def hash_image(desc, mu, W, p: Params, marginal: bool = False) -> HashedImage:
    desc = np.ascontiguousarray(desc, dtype=np.uint8).reshape(-1, D)
    keys, code, marg = hash_desc(desc, mu, W, p, marginal)
    off, idx = buckets(keys, p)
    return HashedImage(desc, keys, code, off, idx, marg)


def match_pair(I: HashedImage, J: HashedImage, p: Params, topk: bool = False, q0: int = 0, q1: int | None = None):
    """Per-query outputs of Sec. 2.3.1 steps (1)-(4) for queries [q0, q1) of I against J."""
    q1 = I.n if q1 is None else q1
    nq = q1 - q0
    best = np.empty(nq, dtype=np.int32)
    d1 = np.empty(nq, dtype=np.uint32)
    d2 = np.empty(nq, dtype=np.uint32)
    nc = np.empty(nq, dtype=np.int32)
    tk = np.empty((nq, p.K), dtype=np.int32) if topk else None
    ci, cj = I._c(), J._c()
    cp = _Params(p.L, p.m, p.nbits, p.K, p.ratio_num, p.ratio_den)
    _load().orc_match_pair(ctypes.byref(ci), ctypes.byref(cj), ctypes.byref(cp), q0, q1, _p(best), _p(d1),
                           _p(d2), _p(nc), _p(tk))
    out = {"best_j": best, "d1sq": d1, "d2sq": d2, "ncand": nc}
    if topk:
        out["topk"] = tk
    return out


def brute_nn(descI, descJ, ratio_num: int = 4, ratio_den: int = 5):
    descI = np.ascontiguousarray(descI, dtype=np.uint8).reshape(-1, D)
    descJ = np.ascontiguousarray(descJ, dtype=np.uint8).reshape(-1, D)
    nI = descI.shape[0]
    best = np.empty(nI, dtype=np.int32)
    d1 = np.empty(nI, dtype=np.uint32)
    d2 = np.empty(nI, dtype=np.uint32)
    _load().orc_brute_nn(_p(descI), nI, _p(descJ), descJ.shape[0], ratio_num, ratio_den, _p(best), _p(d1), _p(d2))
    return {"best_j": best, "d1sq": d1, "d2sq": d2}


class Index:
    """Oracle over a whole dataset: global centring mean (R3), weights, and
    per-image hashing on demand (cached), with pairs matched on host threads."""

    def __init__(self, desc: np.ndarray, n_desc, p: Params, threads: int | None = None,
                 sums: np.ndarray | None = None, n_total: int | None = None):
        self.p = p
        self.desc = desc.reshape(-1, D)
        self.n_desc = np.asarray(n_desc, dtype=np.int64)
        self.off = np.zeros(len(self.n_desc) + 1, dtype=np.int64)
        np.cumsum(self.n_desc, out=self.off[1:])
        self.threads = threads or (os.cpu_count() or 1)
        self.W = weights(p)
        if sums is None:
            sums = self._sums()
            n_total = int(self.off[-1])
        self.sums = sums
        self.mu = mean_from_sums(sums, n_total)
        self._cache: dict[int, HashedImage] = {}

    def _sums(self) -> np.ndarray:
        n = self.desc.shape[0]
        chunks = np.linspace(0, n, self.threads + 1).astype(np.int64)
        with ThreadPoolExecutor(self.threads) as ex:
            parts = list(ex.map(lambda k: col_sums(self.desc[chunks[k]:chunks[k + 1]]), range(self.threads)))
        return np.sum(parts, axis=0, dtype=np.uint64)

    def image_desc(self, i: int) -> np.ndarray:
        return self.desc[self.off[i]:self.off[i + 1]]

    def image(self, i: int, marginal: bool = False) -> HashedImage:
        h = self._cache.get(i)
        if h is None or (marginal and h.marginal is None):
            h = hash_image(self.image_desc(i), self.mu, self.W, self.p, marginal)
            self._cache[i] = h
        return h

    def hash_images(self, ids, marginal: bool = False):
        ids = [int(i) for i in ids if int(i) not in self._cache or (marginal and self._cache[int(i)].marginal is None)]
        with ThreadPoolExecutor(self.threads) as ex:
            for i, h in zip(ids, ex.map(lambda i: hash_image(self.image_desc(i), self.mu, self.W, self.p,
                                                             marginal), ids)):
                self._cache[i] = h

    def match(self, pairs, topk: bool = False):
        pairs = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
        self.hash_images(np.unique(pairs))
        with ThreadPoolExecutor(self.threads) as ex:
            return list(ex.map(lambda ij: match_pair(self._cache[int(ij[0])], self._cache[int(ij[1])], self.p,
                                                     topk), pairs))
