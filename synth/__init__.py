"""Seeded synthetic workloads shaped like the paper's UAV matching jobs.

Test and benchmark fixture: it builds image layouts, pair lists and uint8
descriptors, and holds none of the matching method's arithmetic.  The paper's
own datasets (three UAV photo sets, Table 1) are not available, so these
workloads stand in for them:

* ``pair2k``      one pair, 2,000 descriptors per image, 40 % of B are noisy
                  (sigma 8) copies of A's descriptors.
* ``strip30``     30 images x 8,000 on a flight strip, each image paired with
                  its 4 nearest along the strip (120 ordered pairs).
* ``grid500``     500 images on a 25 x 20 grid, N_i ~ U{2,000..20,000}, one
                  pair per undirected 12-neighbourhood edge (2,777 pairs).
* ``oblique200``  40 stations x 5 views (nadir + 4 oblique), 16,000 each,
                  each image paired with its 16 nearest footprints (3,200 pairs).
* ``grid5000``    5,000 images x 20,000 on a 100 x 50 grid, every image paired
                  with each 12-neighbourhood neighbour (58,504 ordered pairs).

``scaled(name, ...)`` gives smaller versions with the same structure for tests.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libsynth.so")


class _World(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("cells_x", ctypes.c_int32), ("cells_y", ctypes.c_int32),
                ("tracks_per_cell", ctypes.c_int32), ("img_w", ctypes.c_float), ("img_h", ctypes.c_float),
                ("kp_noise", ctypes.c_float)]


_IMAGE_DTYPE = np.dtype([("n", "<i4"), ("cx0", "<i4"), ("cy0", "<i4"), ("cx1", "<i4"), ("cy1", "<i4"),
                         ("quota", "<i4"), ("sigma", "<f4"), ("A", "<f4", (6,))])


def build(force: bool = False) -> str:
    """Compile the generator into synth/libsynth.so (plain C, pthreads)."""
    src = os.path.join(_HERE, "gen.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-o", tmp, src, "-lm", "-lpthread"])
        os.replace(tmp, _SO)
    return _SO


_lib = None


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        lib.syn_generate.restype = ctypes.c_int
        lib.syn_generate.argtypes = [ctypes.POINTER(_World), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                     ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_int]
        lib.syn_half_normal.restype = ctypes.c_float
        lib.syn_half_normal.argtypes = [ctypes.c_uint32]
        _lib = lib
    return _lib


@dataclass
class Workload:
    """Image layout + pair list; descriptors are generated on demand."""
    name: str
    seed: int
    images: np.ndarray               # structured array, _IMAGE_DTYPE
    pairs: np.ndarray                # int32 [P, 2] (query image, database image)
    cells_x: int
    cells_y: int
    tracks_per_cell: int
    img_w: float = 6000.0
    img_h: float = 4000.0
    kp_noise: float = 0.5
    notes: dict = field(default_factory=dict)

    @property
    def n_images(self) -> int:
        return int(self.images.shape[0])

    @property
    def n_desc(self) -> np.ndarray:
        return self.images["n"].astype(np.int32)

    @property
    def row_off(self) -> np.ndarray:
        off = np.zeros(self.n_images + 1, dtype=np.int64)
        np.cumsum(self.n_desc, out=off[1:])
        return off

    @property
    def total_desc(self) -> int:
        return int(self.n_desc.astype(np.int64).sum())

    def _world(self) -> _World:
        return _World(self.seed, self.cells_x, self.cells_y, self.tracks_per_cell, self.img_w, self.img_h,
                      self.kp_noise)

    def generate(self, i0: int = 0, i1: int | None = None, desc: np.ndarray | None = None,
                 kp: np.ndarray | None = None, track: np.ndarray | None = None, want_kp: bool = False,
                 want_track: bool = False, threads: int | None = None):
        """Generate images [i0, i1) as one concatenated uint8 [rows, 128] array.

        ``desc`` may be any writable C-contiguous uint8 buffer (e.g. a pinned
        host tensor viewed through numpy) of the right size."""
        lib = _load()
        i1 = self.n_images if i1 is None else i1
        off = self.row_off
        rows = int(off[i1] - off[i0])
        if desc is None:
            desc = np.empty((rows, 128), dtype=np.uint8)
        assert desc.dtype == np.uint8 and desc.flags.c_contiguous and desc.size >= rows * 128
        if want_kp and kp is None:
            kp = np.empty((rows, 2), dtype=np.float32)
        if want_track and track is None:
            track = np.empty(rows, dtype=np.int64)
        imgs = np.ascontiguousarray(self.images)
        w = self._world()
        threads = threads or max(1, os.cpu_count() or 1)
        lib.syn_generate(ctypes.byref(w), imgs.ctypes.data, off.ctypes.data, i0, i1, desc.ctypes.data,
                         kp.ctypes.data if kp is not None else None,
                         track.ctypes.data if track is not None else None, int(threads))
        out = [desc]
        if want_kp:
            out.append(kp)
        if want_track:
            out.append(track)
        return out[0] if len(out) == 1 else tuple(out)

    def shared_fraction(self) -> np.ndarray:
        """Expected fraction of the query image's descriptors that are observations
        of a track the database image also observes, per pair (from the layout)."""
        im = self.images
        fr = np.zeros(len(self.pairs))
        for k, (i, j) in enumerate(self.pairs):
            a, b = im[i], im[j]
            ox = max(0, min(a["cx1"], b["cx1"]) - max(a["cx0"], b["cx0"]))
            oy = max(0, min(a["cy1"], b["cy1"]) - max(a["cy0"], b["cy0"]))
            fr[k] = ox * oy * min(a["quota"], b["quota"]) / max(1, a["n"])
        return fr


def _affine(cx: float, cy: float, scale: float, theta: float, w: float, h: float) -> list:
    c, s = math.cos(theta), math.sin(theta)
    # pixel = R(theta) * scale * (world - centre) + (w/2, h/2)
    return [scale * c, -scale * s, w / 2 - scale * (c * cx - s * cy),
            scale * s, scale * c, h / 2 - scale * (s * cx + c * cy)]


def _images(recs) -> np.ndarray:
    arr = np.zeros(len(recs), dtype=_IMAGE_DTYPE)
    for k, r in enumerate(recs):
        arr[k] = (r["n"], r["cx0"], r["cy0"], r["cx1"], r["cy1"], r["quota"], r["sigma"], r["A"])
    return arr


def pair2k(seed: int = 1, n: int = 2000, shared: int = 800) -> Workload:
    """One pair: A holds n base descriptors, B holds `shared` sigma-8 copies of A's."""
    recs = []
    for k, sigma in enumerate((0.0, 8.0)):
        recs.append(dict(n=n, cx0=0, cy0=0, cx1=1, cy1=1, quota=shared, sigma=sigma,
                         A=_affine(0.5, 0.5, 4000.0, 0.1 * k, 6000.0, 4000.0)))
    return Workload("pair2k", seed, _images(recs), np.array([[0, 1]], dtype=np.int32), 1, 1, shared)


def strip30(seed: int = 2, n_images: int = 30, n: int = 8000, nbrs: int = 4, phi: float = 0.6) -> Workload:
    """Flight strip: image k covers cells [2k, 2k+6); pairs = 4 nearest along the strip."""
    span, step = 6, 2
    quota = int(phi * n / span)
    sigma = 8.0 / math.sqrt(2.0)
    recs = [dict(n=n, cx0=step * k, cy0=0, cx1=step * k + span, cy1=1, quota=quota, sigma=sigma,
                 A=_affine(step * k + span / 2, 0.5, 1000.0, 0.0, 6000.0, 4000.0)) for k in range(n_images)]
    pairs = []
    for i in range(n_images):
        order = sorted((j for j in range(n_images) if j != i), key=lambda j: (abs(i - j), j))
        pairs += [(i, j) for j in order[:nbrs]]
    return Workload("strip30", seed, _images(recs), np.array(pairs, dtype=np.int32),
                    step * (n_images - 1) + span, 1, quota)


def _grid(name, seed, gx, gy, n_of, phi, directed, span=5, step=2, nb_r2=4):
    sigma = 8.0 / math.sqrt(2.0)
    recs = []
    ns = [n_of(k) for k in range(gx * gy)]
    qmax = 0
    for k in range(gx * gy):
        x, y = k % gx, k // gx
        q = int(phi * ns[k] / (span * span))
        qmax = max(qmax, q)
        recs.append(dict(n=ns[k], cx0=step * x, cy0=step * y, cx1=step * x + span, cy1=step * y + span,
                         quota=q, sigma=sigma,
                         A=_affine(step * x + span / 2, step * y + span / 2, 1200.0, 0.3 * ((k * 7) % 11),
                                   6000.0, 4000.0)))
    offs = [(dx, dy) for dx in range(-2, 3) for dy in range(-2, 3) if 0 < dx * dx + dy * dy <= nb_r2]
    pairs = []
    for k in range(gx * gy):
        x, y = k % gx, k // gx
        for dx, dy in offs:
            u, v = x + dx, y + dy
            if 0 <= u < gx and 0 <= v < gy:
                j = v * gx + u
                if directed or k < j:
                    pairs.append((k, j))
    return Workload(name, seed, _images(recs), np.array(pairs, dtype=np.int32),
                    step * (gx - 1) + span, step * (gy - 1) + span, qmax)


def grid500(seed: int = 3, gx: int = 25, gy: int = 20, nmin: int = 2000, nmax: int = 20000,
            phi: float = 0.85) -> Workload:
    """Uneven grid flight: N_i ~ U{nmin..nmax}; one pair per undirected 12-neighbourhood edge."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ns = rng.integers(nmin, nmax + 1, size=gx * gy)
    return _grid("grid500", seed, gx, gy, lambda k: int(ns[k]), phi, directed=False)


def grid5000(seed: int = 5, gx: int = 100, gy: int = 50, n: int = 20000, phi: float = 0.75) -> Workload:
    """Large grid flight: every image paired with each 12-neighbourhood neighbour (ordered jobs)."""
    return _grid("grid5000", seed, gx, gy, lambda k: n, phi, directed=True)


def oblique200(seed: int = 4, sx: int = 8, sy: int = 5, n: int = 16000, nbrs: int = 16,
               phi: float = 0.45) -> Workload:
    """40 stations x (nadir + 4 oblique views); each image paired with its 16 nearest footprints."""
    span, step, off = 6, 3, 3
    quota = int(phi * n / (span * span))
    sigma = 8.0 / math.sqrt(2.0)
    views = [(0, 0), (off, 0), (-off, 0), (0, off), (0, -off)]
    recs, centres = [], []
    for st in range(sx * sy):
        x, y = st % sx, st // sx
        for vi, (ox, oy) in enumerate(views):
            cx0 = step * x + ox + off
            cy0 = step * y + oy + off
            centres.append((cx0 + span / 2, cy0 + span / 2))
            recs.append(dict(n=n, cx0=cx0, cy0=cy0, cx1=cx0 + span, cy1=cy0 + span, quota=quota, sigma=sigma,
                             A=_affine(cx0 + span / 2, cy0 + span / 2, 1000.0, 1.3 * vi, 6000.0, 4000.0)))
    c = np.array(centres)
    pairs = []
    for i in range(len(recs)):
        d2 = ((c - c[i]) ** 2).sum(1)
        order = sorted((j for j in range(len(recs)) if j != i), key=lambda j: (d2[j], j))
        pairs += [(i, j) for j in order[:nbrs]]
    return Workload("oblique200", seed, _images(recs), np.array(pairs, dtype=np.int32),
                    step * (sx - 1) + span + 2 * off, step * (sy - 1) + span + 2 * off, quota)


def scaled(name: str, **kw) -> Workload:
    """Same structure, smaller sizes (for parity tests)."""
    return {"pair2k": pair2k, "strip30": strip30, "grid500": grid500, "grid5000": grid5000,
            "oblique200": oblique200}[name](**kw)


WORKLOADS = {
    "pair2k": pair2k,
    "strip30": strip30,
    "grid500": grid500,
    "oblique200": oblique200,
    "grid5000": grid5000,
}


def workload(name: str) -> Workload:
    return WORKLOADS[name]()
