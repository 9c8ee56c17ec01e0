"""Python binding of the cashmatch C ABI (include/cashmatch.h).

Argument marshalling only: every step of the matching path runs in the CUDA
library ``libcashmatch.so`` built from ``csrc/`` for sm_103a.  PyTorch provides
device memory (the index arena, outputs) and streams.  There is no fallback:
if the library is missing or no GPU is present the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import weakref
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcashmatch.so")

CM_OK, CM_ERR_INVALID, CM_ERR_BUDGET, CM_ERR_CUDA, CM_ERR_TIMEOUT, CM_ERR_NOMEM, CM_ERR_STATE = range(7)
RERANK = {"fp32": 0, "bf16": 1, "fp8": 2, "int": 3}
ALGO = {"auto": 0, "tile": 1, "warp": 2, "tc": 3, "bucket": 4}
PROJ = {"tc": 0, "ffma": 1}
MEM_HOST, MEM_DEVICE, MEM_DEVICE_INPLACE = 0, 1, 2
# Arena headroom the binding adds to cm_index_bytes for match-plan tables
# (24 bytes per planned pair): room for about 600,000 pairs of plans.
PLAN_HEADROOM = 16 << 20
# A plan also holds its per-query lists (4 K bytes per query row with the
# bucket-major scan; 6 K, 10 K with FP8, for the hand-over of the tile and
# tensor-core scans to the tensor-core rerank); the default arena has room for
# plans totalling this many times the index's descriptors as query rows.
TC_PLAN_ROWS_FACTOR = 16


def default_headroom(p, n_desc) -> int:
    """Arena bytes the binding adds to cm_index_bytes by default."""
    nd = np.asarray(n_desc, dtype=np.int64)
    bucket = p.algo in (ALGO["auto"], ALGO["bucket"])
    per_row = 0
    if p.rerank in (RERANK["bf16"], RERANK["fp8"]) or p.algo == ALGO["tc"]:
        per_row += p.K * (10 if p.rerank == RERANK["fp8"] else 6)   # the scan -> rerank hand-over
    if bucket:
        per_row += 4 * p.K                                           # the bucket-major scan's key lists
    extra = TC_PLAN_ROWS_FACTOR * int(nd.sum()) * per_row
    if p.algo == ALGO["tc"]:   # per-table lists of the tensor-core scan, for a few plans
        extra += 4 * 160 * int(nd.max() if len(nd) else 0) * p.L * p.K * 4
    return PLAN_HEADROOM + extra

# Every symbol include/cashmatch.h declares (checked by the CPU tests).
EXPORTS = [
    "cm_version", "cm_last_error", "cm_params_default", "cm_params_check", "cm_make_weights", "cm_image_bytes",
    "cm_index_bytes", "cm_plan_bytes", "cm_schedule_blocks", "cm_schedule_num_rows", "cm_schedule_num_iterations",
    "cm_schedule_get_row", "cm_free_schedule", "cm_gps_order", "cm_index_create", "cm_index_set_mean",
    "cm_index_mean_device", "cm_index_col_sums", "cm_index_check", "cm_index_load", "cm_index_rehash", "cm_index_evict", "cm_build_index",
    "cm_index_image_view", "cm_index_destroy", "cm_match_plan_create", "cm_match_plan_rows", "cm_match_plan_run",
    "cm_match_plan_run_marked",
    "cm_match_plan_compact", "cm_match_plan_mutual", "cm_match_plan_destroy", "cm_match_pairs", "cm_sequence_create", "cm_sequence_launch",
    "cm_sequence_kernels", "cm_sequence_destroy", "cm_schedule_arena_bytes", "cm_pipeline_workspace_bytes", "cm_run_schedule",
    "cm_verify_affine", "cm_affine_verify_cb", "cm_sao_filter", "cm_schedule_from_rows", "cm_vlad_workspace_bytes", "cm_vlad_encode",
    "cm_workspace_status", "cm_nn_workspace_bytes", "cm_nn_pairs", "cm_selftest_wait", "cm_match_plan_sao_bytes",
    "cm_match_plan_sao", "cm_pipeline_workspace_bytes_ex", "cm_run_schedule_ex", "cm_autotune", "cm_match_pair_noalloc",
    "cm_match_pairs_workspace_bytes", "cm_index_workspace_bytes", "cm_free_index", "cm_index_mean_host",
    "cm_probe_int", "cm_index_col_sums_of", "cm_index_set_mean_device", "cm_index_hash",
]


class CMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("cashmatch error %d: %s" % (status, msg))
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("m", ctypes.c_int32), ("n_bits", ctypes.c_int32), ("K", ctypes.c_int32),
                ("ratio_num", ctypes.c_int32), ("ratio_den", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("rerank", ctypes.c_int32), ("query_tile", ctypes.c_int32), ("algo", ctypes.c_int32),
                ("projection", ctypes.c_int32)]

    @classmethod
    def make(cls, L=6, m=8, K=8, ratio=(4, 5), seed=0x5EED, rerank="fp32", query_tile=0, n_bits=128, algo="auto",
             projection="tc"):
        return cls(L, m, n_bits, K, ratio[0], ratio[1], seed, RERANK[rerank] if isinstance(rerank, str) else rerank,
                   query_tile, ALGO[algo] if isinstance(algo, str) else algo,
                   PROJ[projection] if isinstance(projection, str) else projection)

    @property
    def P(self):
        return self.L * self.m + self.n_bits


class MatchOut(ctypes.Structure):
    _fields_ = [("best_j", ctypes.c_void_p), ("d1sq", ctypes.c_void_p), ("d2sq", ctypes.c_void_p),
                ("topk", ctypes.c_void_p), ("stats", ctypes.c_void_p)]


class CompactOut(ctypes.Structure):
    _fields_ = [("counts", ctypes.c_void_p), ("offsets", ctypes.c_void_p), ("total", ctypes.c_void_p),
                ("matches", ctypes.c_void_p), ("capacity", ctypes.c_uint64)]


class PipelineStats(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int32), ("workers", ctypes.c_int32), ("pairs", ctypes.c_int64),
                ("queries", ctypes.c_int64), ("matches", ctypes.c_int64), ("kernels", ctypes.c_int64),
                ("h2d_bytes", ctypes.c_uint64), ("d2h_bytes", ctypes.c_uint64), ("wall_ms", ctypes.c_double),
                ("gpu_ms", ctypes.c_double), ("verify_ms", ctypes.c_double), ("stall_ms", ctypes.c_double),
                ("tail_ms", ctypes.c_double), ("prefetched_rows", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class AffineVerifier(ctypes.Structure):
    _fields_ = [("keypoints", ctypes.c_void_p), ("thresh_px", ctypes.c_float), ("max_iters", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("inliers", ctypes.c_void_p), ("sao_k", ctypes.c_int32),
                ("sao_max_score", ctypes.c_float), ("sao_kept", ctypes.c_void_p)]


VERIFY_FN = ctypes.CFUNCTYPE(ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p,
                             ctypes.c_int64, ctypes.POINTER(ctypes.c_uint32))


class PipelineOpts(ctypes.Structure):
    _fields_ = [("sao_k", ctypes.c_int32), ("sao_max_score", ctypes.c_float), ("d_kp", ctypes.c_void_p),
                ("d_kp_off", ctypes.c_void_p), ("centre", ctypes.c_int32)]


class TuneResult(ctypes.Structure):
    _fields_ = [("query_tile", ctypes.c_int32), ("algo", ctypes.c_int32), ("K", ctypes.c_int32),
                ("trials", ctypes.c_int32), ("ms", ctypes.c_float), ("agreement", ctypes.c_float)]


class ScheduleRow(ctypes.Structure):
    _fields_ = [("iteration", ctypes.c_int32), ("n_load", ctypes.c_int32), ("load", ctypes.POINTER(ctypes.c_int32)),
                ("n_free", ctypes.c_int32), ("free_ids", ctypes.POINTER(ctypes.c_int32)),
                ("n_pairs", ctypes.c_int64), ("pairs", ctypes.POINTER(ctypes.c_int64))]


_lib = None


def lib():
    """Load libcashmatch.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libcashmatch.so is not built: run python -m paper_2505_22089_b300.build")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
        P = ctypes.POINTER(Params)
        sig = {
            "cm_version": (ctypes.c_char_p, []),
            "cm_last_error": (ctypes.c_char_p, []),
            "cm_params_default": (i32, [P]),
            "cm_params_check": (i32, [P]),
            "cm_make_weights": (i32, [P, vp]),
            "cm_image_bytes": (i32, [P, i32, ctypes.POINTER(u64)]),
            "cm_index_bytes": (i32, [P, i32, vp, i32, ctypes.POINTER(u64)]),
            "cm_schedule_blocks": (i32, [vp, i64, i32, vp, P, u64, i32, ctypes.POINTER(vp)]),
            "cm_schedule_num_rows": (i32, [vp]),
            "cm_schedule_from_rows": (i32, [i32, vp, vp, i64, i32, ctypes.POINTER(vp)]),
            "cm_schedule_num_iterations": (i32, [vp]),
            "cm_schedule_get_row": (i32, [vp, i32, ctypes.POINTER(ScheduleRow)]),
            "cm_free_schedule": (None, [vp]),
            "cm_gps_order": (i32, [i32, i64, vp, vp, ctypes.POINTER(i32)]),
            "cm_index_create": (i32, [P, i32, vp, vp, u64, ctypes.POINTER(vp)]),
            "cm_index_set_mean": (i32, [vp, vp, u64, vp]),
            "cm_index_mean_device": (i32, [vp, vp, u64, vp]),
            "cm_index_col_sums": (i32, [vp, vp, ctypes.POINTER(u64), vp]),
            "cm_index_check": (i32, [vp, vp]),
            "cm_index_load": (i32, [vp, i32, vp, vp, i32, vp]),
            "cm_index_rehash": (i32, [vp, vp]),
            "cm_index_evict": (i32, [vp, i32, vp, vp]),
            "cm_build_index": (i32, [P, i32, vp, vp, i32, vp, u64, vp, ctypes.POINTER(vp)]),
            "cm_index_image_view": (i32, [vp, i32] + [ctypes.POINTER(vp)] * 5),
            "cm_index_destroy": (None, [vp]),
            "cm_match_plan_create": (i32, [vp, vp, i64, vp, ctypes.POINTER(vp)]),
            "cm_match_plan_rows": (i64, [vp]),
            "cm_match_plan_run": (i32, [vp, ctypes.POINTER(MatchOut), vp]),
            "cm_match_plan_run_marked": (i32, [vp, ctypes.POINTER(MatchOut), vp, vp]),
            "cm_match_plan_destroy": (None, [vp]),
            "cm_match_plan_compact": (i32, [vp, vp, vp, vp, vp, vp, u64, vp]),
            "cm_match_plan_mutual": (i32, [vp, vp, vp, vp]),
            "cm_match_pairs": (i32, [vp, vp, i64, vp, u64, vp, vp, vp, vp]),
            "cm_match_pairs_workspace_bytes": (i32, [vp, vp, i64, ctypes.POINTER(u64)]),
            "cm_index_workspace_bytes": (i32, [vp, vp, i32, ctypes.POINTER(u64)]),
            "cm_free_index": (None, [vp]),
            "cm_index_mean_host": (i32, [vp, vp, vp]),
            "cm_probe_int": (i32, [i32, i32, vp, u64, vp, ctypes.POINTER(ctypes.c_double)]),
            "cm_index_col_sums_of": (i32, [vp, i32, vp, vp, vp]),
            "cm_index_set_mean_device": (i32, [vp, vp, u64, vp]),
            "cm_index_hash": (i32, [vp, vp]),
            "cm_match_pair_noalloc": (i32, [P, vp, i32, vp, i32, vp, u64, vp, vp, vp, vp]),
            "cm_sequence_create": (i32, [vp, i32, i32, vp, vp, vp, vp, ctypes.POINTER(vp)]),
            "cm_sequence_launch": (i32, [vp, vp]),
            "cm_sequence_kernels": (i32, [vp]),
            "cm_sequence_destroy": (None, [vp]),
            "cm_schedule_arena_bytes": (i32, [vp, P, i32, vp, vp, i64, ctypes.POINTER(u64)]),
            "cm_plan_bytes": (i32, [P, i64, i64, i32, ctypes.POINTER(u64)]),
            "cm_pipeline_workspace_bytes": (i32, [vp, vp, vp, i64, ctypes.POINTER(u64)]),
            "cm_run_schedule": (i32, [vp, vp, vp, i64, vp, vp, u64, vp, vp, i32, vp,
                                      ctypes.POINTER(PipelineStats)]),
            "cm_verify_affine": (i32, [vp, vp, i64, vp, ctypes.c_float, i32, u64, vp, vp, ctypes.POINTER(i64)]),
            "cm_affine_verify_cb": (i32, [vp, i32, i64, vp, i64, vp]),
            "cm_sao_filter": (i32, [vp, vp, i64, vp, i32, ctypes.c_float, vp, vp, ctypes.POINTER(i64)]),
            "cm_vlad_workspace_bytes": (i32, [i32, i64, ctypes.POINTER(u64)]),
            "cm_vlad_encode": (i32, [vp, vp, i32, vp, i32, vp, u64, vp, vp, vp]),
            "cm_workspace_status": (i32, [vp, vp]),
            "cm_selftest_wait": (i32, [i32, vp]),
            "cm_match_plan_sao_bytes": (i32, [vp, ctypes.POINTER(u64)]),
            "cm_match_plan_sao": (i32, [vp, vp, vp, vp, vp, i32, ctypes.c_float, vp, vp, u64, vp]),
            "cm_pipeline_workspace_bytes_ex": (i32, [vp, vp, vp, i64, vp, ctypes.POINTER(u64)]),
            "cm_run_schedule_ex": (i32, [vp, vp, vp, i64, vp, vp, u64, vp, vp, i32, vp, vp, vp]),
            "cm_nn_workspace_bytes": (i32, [vp, i32, vp, i64, ctypes.POINTER(u64)]),
            "cm_nn_pairs": (i32, [vp, vp, i32, vp, i64, i32, i32, vp, u64, vp, vp, vp, vp]),
            "cm_autotune": (i32, [vp, vp, i64, vp, i32, ctypes.c_float, vp, ctypes.POINTER(TuneResult)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(status):
    if status != CM_OK:
        raise CMError(status, lib().cm_last_error().decode())


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def version() -> str:
    return lib().cm_version().decode()


def make_weights(p: Params) -> np.ndarray:
    W = np.empty((128, p.P), dtype=np.float32)
    check(lib().cm_make_weights(ctypes.byref(p), W.ctypes.data))
    return W


def image_bytes(p: Params, n: int) -> int:
    b = ctypes.c_uint64()
    check(lib().cm_image_bytes(ctypes.byref(p), int(n), ctypes.byref(b)))
    return b.value


def index_bytes(p: Params, n_desc, inplace: bool = False) -> int:
    nd = np.ascontiguousarray(n_desc, dtype=np.int32)
    b = ctypes.c_uint64()
    check(lib().cm_index_bytes(ctypes.byref(p), len(nd), nd.ctypes.data, int(inplace), ctypes.byref(b)))
    return b.value


def gps_order(n: int, edges) -> list:
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 2))
    order = np.empty(max(n, 1), dtype=np.int32)
    cnt = ctypes.c_int32()
    check(lib().cm_gps_order(n, e.shape[0], e.ctypes.data, order.ctypes.data, ctypes.byref(cnt)))
    return [int(x) for x in order[:cnt.value]]


class Schedule:
    """A cm_schedule: rows (load / free / pair ids per block row) read into
    Python, and the handle, kept for cm_run_schedule."""

    def __init__(self, h: ctypes.c_void_p, pairs: np.ndarray):
        self.h = h
        self.pairs = pairs
        self.rows = []
        r = ScheduleRow()

        def ids(ptr, n):
            return np.ctypeslib.as_array(ptr, shape=(n,)).tolist() if n > 0 else []

        for k in range(lib().cm_schedule_num_rows(h)):
            check(lib().cm_schedule_get_row(h, k, ctypes.byref(r)))
            self.rows.append({"iteration": r.iteration, "load": ids(r.load, r.n_load),
                              "free": ids(r.free_ids, r.n_free), "pairs": ids(r.pairs, r.n_pairs)})
        self.iterations = lib().cm_schedule_num_iterations(h)

    def close(self):
        if getattr(self, "h", None):
            lib().cm_free_schedule(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def schedule_blocks(pairs, n_desc, p: Params, budget: int, max_images_per_block: int) -> Schedule:
    pr = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
    nd = np.ascontiguousarray(n_desc, dtype=np.int32)
    h = ctypes.c_void_p()
    check(lib().cm_schedule_blocks(pr.ctypes.data, pr.shape[0], len(nd), nd.ctypes.data, ctypes.byref(p),
                                   int(budget), int(max_images_per_block), ctypes.byref(h)))
    return Schedule(h, pr)


def schedule_from_rows(rows, pairs, n_images: int) -> Schedule:
    """cm_schedule_from_rows: rows = [{"load": [...], "free": [...], "pairs": [...],
    "iteration": int (optional)}], pair ids into `pairs`."""
    pr = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
    keep = []
    crows = (ScheduleRow * max(len(rows), 1))()
    for k, r in enumerate(rows):
        ld = np.ascontiguousarray(r.get("load", []), dtype=np.int32)
        fr = np.ascontiguousarray(r.get("free", []), dtype=np.int32)
        ps = np.ascontiguousarray(r.get("pairs", []), dtype=np.int64)
        keep += [ld, fr, ps]
        crows[k] = ScheduleRow(int(r.get("iteration", 0)), len(ld), ld.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                               len(fr), fr.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), len(ps),
                               ps.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    h = ctypes.c_void_p()
    check(lib().cm_schedule_from_rows(len(rows), ctypes.cast(crows, ctypes.c_void_p), pr.ctypes.data if len(pr) else None,
                                      len(pr), int(n_images), ctypes.byref(h)))
    del keep
    return Schedule(h, pr)


def schedule_arena_bytes(sched: Schedule, p: Params, n_desc) -> int:
    """cm_schedule_arena_bytes: arena an index needs to run `sched` with run_schedule."""
    nd = np.ascontiguousarray(n_desc, dtype=np.int32)
    b = ctypes.c_uint64()
    check(lib().cm_schedule_arena_bytes(sched.h, ctypes.byref(p), len(nd), nd.ctypes.data, sched.pairs.ctypes.data,
                                        len(sched.pairs), ctypes.byref(b)))
    return b.value


def plan_bytes(p: Params, n_pairs: int, rows: int, max_query_rows: int) -> int:
    """cm_plan_bytes: arena bytes a plan takes from its index."""
    b = ctypes.c_uint64()
    check(lib().cm_plan_bytes(ctypes.byref(p), int(n_pairs), int(rows), int(max_query_rows), ctypes.byref(b)))
    return b.value


def pairs_plan_bytes(p: Params, n_desc, pairs) -> int:
    """Arena bytes of one plan over `pairs` (query rows = sum of N_i)."""
    pr = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
    nd = np.asarray(n_desc, dtype=np.int64)
    rows = int(nd[pr[:, 0]].sum()) if len(pr) else 0
    max_ni = int(nd[pr[:, 0]].max()) if len(pr) else 0
    return plan_bytes(p, len(pr), rows, max_ni)


def verify_affine(kp_i, kp_j, matches, thresh_px: float = 3.0, max_iters: int = 1000, seed: int = 1):
    """cm_verify_affine on host arrays: returns (A 2x3, inlier mask, inlier count)."""
    ki = np.ascontiguousarray(kp_i, dtype=np.float32)
    kj = np.ascontiguousarray(kp_j, dtype=np.float32)
    mt = np.ascontiguousarray(matches, dtype=np.uint32)
    A = np.zeros(6, dtype=np.float32)
    mask = np.zeros(max(len(mt), 1), dtype=np.uint8)
    n = ctypes.c_int64()
    check(lib().cm_verify_affine(ki.ctypes.data, kj.ctypes.data, len(mt), mt.ctypes.data if len(mt) else None,
                                 float(thresh_px), int(max_iters), int(seed), A.ctypes.data, mask.ctypes.data,
                                 ctypes.byref(n)))
    return A.reshape(2, 3), mask[: len(mt)].astype(bool), n.value


def sao_filter(kp_i, kp_j, matches, k: int = 8, max_score: float = 0.875):
    """cm_sao_filter on host arrays: returns (scores float32, keep mask, kept count)."""
    ki = np.ascontiguousarray(kp_i, dtype=np.float32)
    kj = np.ascontiguousarray(kp_j, dtype=np.float32)
    mt = np.ascontiguousarray(matches, dtype=np.uint32)
    score = np.zeros(max(len(mt), 1), dtype=np.float32)
    keep = np.zeros(max(len(mt), 1), dtype=np.uint8)
    n = ctypes.c_int64()
    check(lib().cm_sao_filter(ki.ctypes.data, kj.ctypes.data, len(mt), mt.ctypes.data if len(mt) else None, int(k),
                              float(max_score), score.ctypes.data, keep.ctypes.data, ctypes.byref(n)))
    return score[: len(mt)], keep[: len(mt)].astype(bool), n.value


def vlad_encode(desc, n_desc, codebook, stream=None, want_assign: bool = False, check_status: bool = True):
    """cm_vlad_encode.  desc: CUDA uint8 [n][128] (all images' rows), n_desc:
    rows per image, codebook: CUDA uint8 [C][128].  Returns (vlad float32
    [n_images][C * 128], assignments uint16 as int32 tensor or None)."""
    import torch
    nd = np.ascontiguousarray(n_desc, dtype=np.int64)
    off = np.concatenate([[0], np.cumsum(nd)]).astype(np.int64)
    C = int(codebook.shape[0])
    ws = ctypes.c_uint64()
    check(lib().cm_vlad_workspace_bytes(len(nd), int(off[-1]), ctypes.byref(ws)))
    work = torch.empty(int(ws.value) + 256, dtype=torch.uint8, device=desc.device)
    wbase = (work.data_ptr() + 255) // 256 * 256
    out = torch.empty((len(nd), C * 128), dtype=torch.float32, device=desc.device)
    asg = torch.empty(int(off[-1]), dtype=torch.int16, device=desc.device) if want_assign else None
    check(lib().cm_vlad_encode(_ptr(desc), off.ctypes.data, len(nd), _ptr(codebook), C, ctypes.c_void_p(wbase),
                               int(ws.value), _ptr(asg), _ptr(out), _stream(stream)))
    if check_status:
        check(lib().cm_workspace_status(ctypes.c_void_p(wbase), _stream(stream)))
    a = asg.to(torch.int32) & 0xFFFF if asg is not None else None
    return out, a


PROBE = {"popc": 0, "lop3": 1, "ham4": 2, "ham3": 3}


def probe_int(kind: str, iters: int = 4096, stream=None) -> float:
    """cm_probe_int: measured operations (or 128-bit distances) per clock per SM."""
    import torch
    work = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    r = ctypes.c_double()
    check(lib().cm_probe_int(PROBE[kind], int(iters), _ptr(work), work.numel(), _stream(stream), ctypes.byref(r)))
    return float(r.value)


def nn_pairs(desc, n_desc, pairs, ratio=(4, 5), stream=None, check_status: bool = True):
    """cm_nn_pairs: exhaustive nearest neighbours with the exact ratio test.
    desc: CUDA uint8 [n][128] (all images), n_desc: rows per image, pairs:
    [n_pairs][2].  Returns (best_j, d1sq, d2sq) CUDA tensors (int32; the
    squared distances as int64 with 0xFFFFFFFF for a missing q1 / q2) and the
    per-pair row offsets."""
    import torch
    nd = np.ascontiguousarray(n_desc, dtype=np.int64)
    off = np.concatenate([[0], np.cumsum(nd)]).astype(np.int64)
    pr = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
    rows = np.concatenate([[0], np.cumsum(nd[pr[:, 0]])]).astype(np.int64) if len(pr) else np.zeros(1, np.int64)
    ws = ctypes.c_uint64()
    check(lib().cm_nn_workspace_bytes(off.ctypes.data, len(nd), pr.ctypes.data if len(pr) else None, len(pr),
                                      ctypes.byref(ws)))
    work = torch.empty(int(ws.value) + 256, dtype=torch.uint8, device=desc.device)
    wbase = (work.data_ptr() + 255) // 256 * 256
    n = int(rows[-1])
    best = torch.empty(max(n, 1), dtype=torch.int32, device=desc.device)
    d1 = torch.empty(max(n, 1), dtype=torch.int32, device=desc.device)
    d2 = torch.empty(max(n, 1), dtype=torch.int32, device=desc.device)
    check(lib().cm_nn_pairs(_ptr(desc), off.ctypes.data, len(nd), pr.ctypes.data if len(pr) else None, len(pr),
                            int(ratio[0]), int(ratio[1]), ctypes.c_void_p(wbase), int(ws.value), _ptr(best), _ptr(d1),
                            _ptr(d2), _stream(stream)))
    if check_status:
        check(lib().cm_workspace_status(ctypes.c_void_p(wbase), _stream(stream)))
    return best[:n], d1[:n].to(torch.int64) & 0xFFFFFFFF, d2[:n].to(torch.int64) & 0xFFFFFFFF, rows


def _cudart():
    import torch  # noqa: F401  (loads the CUDA runtime)
    for name in ("libcudart.so.13", "libcudart.so"):
        try:
            rt = ctypes.CDLL(name)
            rt.cudaMemcpy.restype = ctypes.c_int
            rt.cudaMemcpy.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int]
            return rt
        except OSError:
            continue
    raise RuntimeError("CUDA runtime library not found")


def device_to_numpy(ptr: int, shape, dtype) -> np.ndarray:
    """Copy `shape` elements of `dtype` from a device address into a new numpy array."""
    import torch
    torch.cuda.synchronize()
    out = np.empty(shape, dtype=dtype)
    if out.nbytes:
        rc = _cudart().cudaMemcpy(out.ctypes.data, ctypes.c_void_p(ptr), out.nbytes, 2)  # DeviceToHost
        if rc != 0:
            raise RuntimeError("cudaMemcpy failed: %d" % rc)
    return out


class Index:
    """An arena-backed index (cm_index).  The arena is a torch uint8 CUDA tensor."""

    def __init__(self, p: Params, n_desc, arena_bytes: int | None = None, inplace: bool = False, device="cuda",
                 arena=None):
        """Empty index.  `arena` (optional) is a CUDA uint8 tensor to use as the
        device arena; otherwise one of `arena_bytes` (default: room for every
        image) is allocated."""
        import torch
        self.p = Params.from_buffer_copy(p)   # the index's own copy (cm_autotune may change it)
        self.n_desc = np.ascontiguousarray(n_desc, dtype=np.int32)
        if arena is None:
            if arena_bytes is None:
                arena_bytes = index_bytes(p, self.n_desc, inplace) + default_headroom(p, self.n_desc)
            arena = torch.empty(int(arena_bytes) + 256, dtype=torch.uint8, device=device)
        self.arena = arena
        base = (self.arena.data_ptr() + 255) // 256 * 256
        arena_bytes = self.arena.numel() - (base - self.arena.data_ptr())
        self.h = ctypes.c_void_p()
        check(lib().cm_index_create(ctypes.byref(p), len(self.n_desc), self.n_desc.ctypes.data,
                                    ctypes.c_void_p(base), int(arena_bytes), ctypes.byref(self.h)))
        self._keep = []
        self._plans = []

    @classmethod
    def build(cls, p: Params, n_desc, desc, mem: int | None = None, stream=None, arena_bytes: int | None = None):
        """Index with every image resident.  `desc` = all rows concatenated: a CUDA
        uint8 tensor (used in place unless mem says otherwise) or a host array/tensor."""
        import torch
        self = cls.__new__(cls)
        self.p = Params.from_buffer_copy(p)
        self.n_desc = np.ascontiguousarray(n_desc, dtype=np.int32)
        on_dev = isinstance(desc, torch.Tensor) and desc.is_cuda
        if mem is None:
            mem = MEM_DEVICE_INPLACE if on_dev else MEM_HOST
        if arena_bytes is None:
            arena_bytes = index_bytes(p, self.n_desc, mem == MEM_DEVICE_INPLACE) + default_headroom(p, self.n_desc)
        self.arena = torch.empty(int(arena_bytes) + 256, dtype=torch.uint8, device="cuda")
        base = (self.arena.data_ptr() + 255) // 256 * 256
        ptr = desc.data_ptr() if isinstance(desc, torch.Tensor) else np.ascontiguousarray(desc).ctypes.data
        self._keep = [desc]
        self._plans = []
        self.h = ctypes.c_void_p()
        check(lib().cm_build_index(ctypes.byref(p), len(self.n_desc), self.n_desc.ctypes.data, ctypes.c_void_p(ptr),
                                   mem, ctypes.c_void_p(base), int(arena_bytes), _stream(stream),
                                   ctypes.byref(self.h)))
        return self

    def set_mean(self, sums, n_total: int, stream=None):
        s = np.ascontiguousarray(sums, dtype=np.uint64)
        check(lib().cm_index_set_mean(self.h, s.ctypes.data, int(n_total), _stream(stream)))

    def mean_host(self, descs, stream=None):
        """cm_index_mean_host: the centring mean from every image's host rows
        (descs[i]: uint8 [n_i][128] array or pinned CPU tensor), summed on the GPU."""
        ptrs = (ctypes.c_void_p * len(descs))(*[d.data_ptr() if hasattr(d, "data_ptr") else
                                                np.ascontiguousarray(d).ctypes.data for d in descs])
        self._keep.append(descs)
        check(lib().cm_index_mean_host(self.h, ptrs, _stream(stream)))

    def workspace_bytes(self, sched, block: int = -1) -> int:
        """cm_index_workspace_bytes: device bytes match_pairs needs for row `block` of sched (-1: any row)."""
        b = ctypes.c_uint64()
        check(lib().cm_index_workspace_bytes(self.h, sched.h, int(block), ctypes.byref(b)))
        return int(b.value)

    def match_pairs(self, pairs, workspace, best_j, d1sq=None, d2sq=None, stream=None):
        """cm_match_pairs: one fused match launch over `pairs` (all resident),
        asynchronous on the stream; `workspace` is a CUDA uint8 tensor of at
        least match_pairs_bytes(pairs) + 256 bytes (aligned here)."""
        pr = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
        base = (workspace.data_ptr() + 255) // 256 * 256
        ws = workspace.numel() - (base - workspace.data_ptr())
        check(lib().cm_match_pairs(self.h, pr.ctypes.data, len(pr), ctypes.c_void_p(base), int(ws), _ptr(best_j),
                                   _ptr(d1sq), _ptr(d2sq), _stream(stream)))

    def match_pairs_bytes(self, pairs) -> int:
        pr = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
        b = ctypes.c_uint64()
        check(lib().cm_match_pairs_workspace_bytes(self.h, pr.ctypes.data, len(pr), ctypes.byref(b)))
        return int(b.value)

    def col_sums_of(self, ids, d_sums, stream=None):
        """cm_index_col_sums_of: exact column sums of resident images `ids` into
        d_sums (CUDA int64/uint64 tensor of 128 entries), asynchronous."""
        ids = np.ascontiguousarray(ids, dtype=np.int32)
        check(lib().cm_index_col_sums_of(self.h, len(ids), ids.ctypes.data if len(ids) else None, _ptr(d_sums),
                                         _stream(stream)))

    def set_mean_device(self, d_sums, n_total: int, stream=None):
        check(lib().cm_index_set_mean_device(self.h, _ptr(d_sums), int(n_total), _stream(stream)))

    def hash(self, stream=None):
        check(lib().cm_index_hash(self.h, _stream(stream)))

    def mean_device(self, desc, stream=None):
        check(lib().cm_index_mean_device(self.h, _ptr(desc), desc.shape[0], _stream(stream)))

    def col_sums(self, stream=None):
        """(exact uint64 column sums, row count) behind the current centring mean."""
        s = np.zeros(128, dtype=np.uint64)
        n = ctypes.c_uint64()
        check(lib().cm_index_col_sums(self.h, s.ctypes.data, ctypes.byref(n), _stream(stream)))
        return s, n.value

    def load(self, ids, descs, mem: int, stream=None):
        ids = np.ascontiguousarray(ids, dtype=np.int32)
        ptrs = (ctypes.c_void_p * len(ids))(*[d.data_ptr() if hasattr(d, "data_ptr") else
                                               np.ascontiguousarray(d).ctypes.data for d in descs])
        self._keep += list(descs)
        check(lib().cm_index_load(self.h, len(ids), ids.ctypes.data, ptrs, mem, _stream(stream)))

    def evict(self, ids, stream=None):
        ids = np.ascontiguousarray(ids, dtype=np.int32)
        check(lib().cm_index_evict(self.h, len(ids), ids.ctypes.data, _stream(stream)))

    def rehash(self, stream=None):
        check(lib().cm_index_rehash(self.h, _stream(stream)))

    def check(self, stream=None):
        """Raises CMError(CM_ERR_TIMEOUT) if a bounded device wait gave up."""
        check(lib().cm_index_check(self.h, _stream(stream)))

    def autotune(self, pairs, Ks=None, min_agreement: float = 0.999, stream=None) -> dict:
        """cm_autotune on a sample of resident pairs; the choice applies to plans made afterwards."""
        pr = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
        ks = np.ascontiguousarray(Ks if Ks is not None else [], dtype=np.int32)
        r = TuneResult()
        check(lib().cm_autotune(self.h, pr.ctypes.data, len(pr), ks.ctypes.data if len(ks) else None, len(ks),
                                float(min_agreement), _stream(stream), ctypes.byref(r)))
        self.p.query_tile, self.p.algo, self.p.K = r.query_tile, r.algo, r.K
        return {"query_tile": r.query_tile, "algo": {v: k for k, v in ALGO.items()}[r.algo], "K": r.K,
                "trials": r.trials, "ms": r.ms, "agreement": r.agreement}

    def image_view(self, image: int) -> dict:
        """Copies of a resident image's keys, codes and bucket tables (host numpy)."""
        ptrs = [ctypes.c_void_p() for _ in range(5)]
        check(lib().cm_index_image_view(self.h, image, *[ctypes.byref(x) for x in ptrs]))
        n, L, B = int(self.n_desc[image]), self.p.L, 1 << self.p.m
        keyw = device_to_numpy(ptrs[0].value, (n,), np.uint64)
        keys = np.stack([(keyw >> np.uint64(8 * t)) & np.uint64(0xFF) for t in range(L)], 1).astype(np.uint8) \
            if n else np.zeros((0, L), np.uint8)
        return {"keys": keys,
                "code": device_to_numpy(ptrs[1].value, (n, 4), np.uint32),
                "scode": device_to_numpy(ptrs[2].value, (L, n, 4), np.uint32),
                "sidx": device_to_numpy(ptrs[3].value, (L, n), np.uint16),
                "off": device_to_numpy(ptrs[4].value, (L, B + 1), np.uint32)}

    def image_bits(self, image: int):
        """Copies of a resident image's keys (uint8 [n][L]) and codes (uint32 [n][4]) only."""
        ptrs = [ctypes.c_void_p() for _ in range(2)]
        check(lib().cm_index_image_view(self.h, image, ctypes.byref(ptrs[0]), ctypes.byref(ptrs[1]), None, None,
                                        None))
        n, L = int(self.n_desc[image]), self.p.L
        if not n:
            return np.zeros((0, L), np.uint8), np.zeros((0, 4), np.uint32)
        keyw = device_to_numpy(ptrs[0].value, (n,), np.uint64)
        keys = np.ascontiguousarray(keyw.view(np.uint8).reshape(n, 8)[:, :L])
        return keys, device_to_numpy(ptrs[1].value, (n, 4), np.uint32)

    def close(self):
        for ref in getattr(self, "_plans", []):
            pl = ref()
            if pl is not None:
                pl.close()
        if getattr(self, "h", None):
            lib().cm_index_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def match_pair_noalloc(p: Params, desc_i, desc_j, col_sums, n_total: int, best_j, d1sq=None, d2sq=None,
                       stream=None):
    """cm_match_pair_noalloc: one pair matched with the library's static device
    scratch only.  desc_i / desc_j: contiguous CUDA uint8 [n][128]; best_j
    (int32), d1sq, d2sq (4-byte, optional): CUDA tensors of at least n_i entries."""
    import torch

    def _rows(name, t):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.uint8 and t.dim() == 2
                and t.shape[1] == 128 and t.is_contiguous()):
            raise ValueError("%s must be a contiguous CUDA uint8 tensor of shape [n, 128]" % name)
        return int(t.shape[0])

    n_i, n_j = _rows("desc_i", desc_i), _rows("desc_j", desc_j)
    for name, t, need in (("best_j", best_j, True), ("d1sq", d1sq, False), ("d2sq", d2sq, False)):
        if t is None and not need:
            continue
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.element_size() == 4 and t.is_contiguous()
                and t.numel() >= n_i and (name != "best_j" or t.dtype == torch.int32)):
            raise ValueError("%s must be a contiguous CUDA tensor of 4-byte entries (int32 for best_j) with at "
                             "least %d entries" % (name, n_i))
    sums = np.ascontiguousarray(col_sums, dtype=np.uint64)
    if sums.shape != (128,):
        raise ValueError("col_sums must hold 128 column sums")
    check(lib().cm_match_pair_noalloc(ctypes.byref(p), _ptr(desc_i), n_i, _ptr(desc_j), n_j, sums.ctypes.data,
                                      int(n_total), _ptr(best_j), _ptr(d1sq), _ptr(d2sq), _stream(stream)))


class MatchPlan:
    """cm_match_plan over a list of pairs of resident images."""

    def __init__(self, index: Index, pairs, stream=None):
        self.index = index
        self.pairs = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
        self.h = ctypes.c_void_p()
        check(lib().cm_match_plan_create(index.h, self.pairs.ctypes.data, self.pairs.shape[0], _stream(stream),
                                         ctypes.byref(self.h)))
        self.rows = int(lib().cm_match_plan_rows(self.h))
        self.K = int(index.p.K)   # the plan keeps the index's parameters of this moment
        index._plans.append(weakref.ref(self))
        nd = index.n_desc[self.pairs[:, 0]].astype(np.int64) if len(self.pairs) else np.zeros(0, np.int64)
        self.row_off = np.concatenate([[0], np.cumsum(nd)]).astype(np.int64)

    def alloc_out(self, d12: bool = True, topk: bool = False, stats: bool = True):
        import torch
        n = max(self.rows, 1)
        out = {"best_j": torch.empty(n, dtype=torch.int32, device="cuda")}
        if d12:
            out["d1sq"] = torch.empty(n, dtype=torch.int32, device="cuda")
            out["d2sq"] = torch.empty(n, dtype=torch.int32, device="cuda")
        if topk:
            out["topk"] = torch.empty(n * self.K, dtype=torch.int32, device="cuda")
        if stats:
            out["stats"] = torch.zeros(4, dtype=torch.int32, device="cuda")
        return out

    def run(self, out: dict, stream=None, scan_done=None):
        """scan_done: an optional torch.cuda.Event, recorded on the stream after
        the lookup launch (before the rerank launch of the tensor-core forms)."""
        mo = MatchOut(*[ctypes.c_void_p(out[k].data_ptr()) if out.get(k) is not None else None
                        for k in ("best_j", "d1sq", "d2sq", "topk", "stats")])
        if scan_done is None:
            check(lib().cm_match_plan_run(self.h, ctypes.byref(mo), _stream(stream)))
            return
        if not scan_done.cuda_event:   # torch creates the event at its first record
            scan_done.record(stream)
        check(lib().cm_match_plan_run_marked(self.h, ctypes.byref(mo), ctypes.c_void_p(scan_done.cuda_event),
                                             _stream(stream)))

    def compact(self, best_j, capacity: int | None = None, stream=None):
        """Per-pair match lists from a run's best_j: returns CUDA tensors
        (counts int32 [P], offsets int64 [P], total int64 [1], matches int32 [capacity]);
        a match is query << 16 | database index."""
        import torch
        n = max(len(self.pairs), 1)
        cap = self.rows if capacity is None else int(capacity)
        counts = torch.empty(n, dtype=torch.int32, device=best_j.device)
        offsets = torch.empty(n, dtype=torch.int64, device=best_j.device)
        total = torch.zeros(1, dtype=torch.int64, device=best_j.device)
        matches = torch.empty(max(cap, 1), dtype=torch.int32, device=best_j.device)
        check(lib().cm_match_plan_compact(self.h, _ptr(best_j), _ptr(counts), _ptr(offsets), _ptr(total),
                                          _ptr(matches), cap, _stream(stream)))
        return counts, offsets, total, matches

    def mutual(self, best_j, stream=None):
        """cm_match_plan_mutual: decisions kept only where the reverse pair agrees (new CUDA tensor)."""
        import torch
        out = torch.empty_like(best_j)
        check(lib().cm_match_plan_mutual(self.h, _ptr(best_j), _ptr(out), _stream(stream)))
        return out

    def sao(self, best_j, kp, kp_off, k: int = 8, max_score: float = 0.875, stream=None, want_score: bool = False):
        """cm_match_plan_sao: decisions with the SAO local constraint applied
        (new CUDA tensor) and, optionally, the per-row scores.  kp: CUDA float
        [rows][2] of all images, kp_off: CUDA int64 [n_images + 1]."""
        import torch
        out = torch.empty_like(best_j)
        b = ctypes.c_uint64()
        check(lib().cm_match_plan_sao_bytes(self.h, ctypes.byref(b)))
        work = torch.empty(int(b.value) + 256, dtype=torch.uint8, device=best_j.device)
        wbase = (work.data_ptr() + 255) // 256 * 256
        score = torch.empty(best_j.numel(), dtype=torch.float32, device=best_j.device) if want_score else None
        check(lib().cm_match_plan_sao(self.h, _ptr(best_j), _ptr(out), _ptr(kp), _ptr(kp_off), int(k),
                                      float(max_score), _ptr(score), ctypes.c_void_p(wbase), int(b.value),
                                      _stream(stream)))
        self._sao_work = work   # kept until the next call: the launch may still read it
        return (out, score) if want_score else out

    def close(self):
        if getattr(self, "h", None):
            lib().cm_match_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Sequence:
    """cm_sequence: the device work of a resident block sequence (optional
    rehash, then each plan's match launch and compaction) captured once as a
    CUDA graph and replayed with one launch."""

    def __init__(self, index: Index, plans, outs, compacts=None, rehash: bool = True, stream=None):
        import torch
        self.index = index
        self._keep = (list(plans), list(outs), list(compacts or []))
        n = len(plans)
        ph = (ctypes.c_void_p * max(n, 1))(*[pl.h for pl in plans])
        mo = (MatchOut * max(n, 1))(*[MatchOut(*[ctypes.c_void_p(o[k].data_ptr()) if o.get(k) is not None else None
                                                 for k in ("best_j", "d1sq", "d2sq", "topk", "stats")])
                                      for o in outs])
        co = None
        if compacts is not None:
            co = (CompactOut * max(n, 1))(*[CompactOut(_ptr(c["counts"]), _ptr(c["offsets"]), _ptr(c.get("total")),
                                                       _ptr(c.get("matches")), int(c.get("capacity", 0)))
                                            if c is not None else CompactOut() for c in compacts])
        cap = torch.cuda.Stream() if stream is None else stream
        if stream is None:
            cap.wait_stream(torch.cuda.current_stream())
        self.h = ctypes.c_void_p()
        check(lib().cm_sequence_create(index.h, int(rehash), n, ph, mo, co, _stream(cap), ctypes.byref(self.h)))
        self.kernels = int(lib().cm_sequence_kernels(self.h))

    def launch(self, stream=None):
        check(lib().cm_sequence_launch(self.h, _stream(stream)))

    def close(self):
        if getattr(self, "h", None):
            lib().cm_sequence_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def compact_out(plan: "MatchPlan", capacity: int | None = None) -> dict:
    """Device buffers for one plan's compaction inside a Sequence."""
    import torch
    n = max(len(plan.pairs), 1)
    cap = plan.rows if capacity is None else int(capacity)
    return {"counts": torch.empty(n, dtype=torch.int32, device="cuda"),
            "offsets": torch.empty(n, dtype=torch.int64, device="cuda"),
            "total": torch.zeros(1, dtype=torch.int64, device="cuda"),
            "matches": torch.empty(max(cap, 1), dtype=torch.int32, device="cuda"), "capacity": cap}


def run_schedule(index: Index, sched: Schedule, desc_host, verify=None, keypoints=None, thresh_px: float = 3.0,
                 max_iters: int = 500, seed: int = 7, workers: int = 4, stream=None, sao_k: int = 0,
                 sao_max_score: float = 0.875, sao_kept=None, gpu_sao_k: int = 0, kp_dev=None, kp_off_dev=None,
                 centre: bool = False):
    """cm_run_schedule.  desc_host: per image a host uint8 [n][128] array or
    pinned CPU tensor.  verify: None (count matches only), "affine" (the
    library's RANSAC callback over `keypoints`, per image float [n][2], after
    the SAO local constraint when sao_k > 0; sao_kept: optional int64 array,
    one entry per pair, receiving the matches SAO kept), or a Python callable
    f(row, pair_id, (i, j), matches: np.ndarray uint32) -> int.  gpu_sao_k > 0
    runs the SAO constraint on the GPU for every row before the matches reach
    the host (kp_dev: CUDA float [rows][2] of all images, kp_off_dev: CUDA
    int64 [n_images + 1]); verification then sees only the kept matches.
    centre=True: the run computes the centring mean itself from desc_host (the
    index needs none beforehand and must have nothing resident).
    Returns (stats dict, inliers per pair or None)."""
    import torch
    pairs = sched.pairs
    opts = None
    if gpu_sao_k or centre:
        opts = PipelineOpts(int(gpu_sao_k), float(sao_max_score), kp_dev.data_ptr() if gpu_sao_k else None,
                            kp_off_dev.data_ptr() if gpu_sao_k else None, int(bool(centre)))
    ws = ctypes.c_uint64()
    check(lib().cm_pipeline_workspace_bytes_ex(index.h, sched.h, pairs.ctypes.data, len(pairs),
                                               ctypes.byref(opts) if opts is not None else None, ctypes.byref(ws)))
    work = torch.empty(int(ws.value) + 256, dtype=torch.uint8, device="cuda")
    wbase = (work.data_ptr() + 255) // 256 * 256
    ptrs = (ctypes.c_void_p * len(desc_host))(*[d.data_ptr() if hasattr(d, "data_ptr") else
                                                np.ascontiguousarray(d).ctypes.data for d in desc_host])
    keep = [desc_host, work]
    inliers = None
    fn, user = None, None
    if verify == "affine":
        kps = [np.ascontiguousarray(k, dtype=np.float32) for k in keypoints]
        kp_ptrs = (ctypes.c_void_p * len(kps))(*[k.ctypes.data for k in kps])
        inliers = np.full(len(pairs), -1, dtype=np.int64)
        if sao_kept is not None:
            assert sao_kept.dtype == np.int64 and sao_kept.shape == (len(pairs),) and sao_kept.flags.c_contiguous
        v = AffineVerifier(ctypes.cast(kp_ptrs, ctypes.c_void_p), float(thresh_px), int(max_iters), int(seed),
                           inliers.ctypes.data, int(sao_k), float(sao_max_score),
                           sao_kept.ctypes.data if sao_kept is not None else None)
        keep += [kps, kp_ptrs, v]
        fn = ctypes.cast(lib().cm_affine_verify_cb, ctypes.c_void_p)
        user = ctypes.cast(ctypes.pointer(v), ctypes.c_void_p)
    elif callable(verify):
        def _cb(_user, row, pair_id, pair_p, n, matches):
            ij = ctypes.cast(pair_p, ctypes.POINTER(ctypes.c_int32))
            arr = np.ctypeslib.as_array(matches, shape=(n,)).copy() if n else np.zeros(0, np.uint32)
            return int(verify(row, pair_id, (ij[0], ij[1]), arr))
        cb = VERIFY_FN(_cb)
        keep.append(cb)
        fn = ctypes.cast(cb, ctypes.c_void_p)
    st = PipelineStats()
    check(lib().cm_run_schedule_ex(index.h, sched.h, pairs.ctypes.data, len(pairs), ptrs, ctypes.c_void_p(wbase),
                                   int(ws.value), fn, user, int(workers),
                                   ctypes.byref(opts) if opts is not None else None, _stream(stream),
                                   ctypes.byref(st)))
    del keep
    return st.as_dict(), inliers
