"""Python binding of libabx.so (argument marshalling only).

Every function here calls the C ABI declared in ``include/abx.h`` with the
same name; all computation runs in the library's CUDA kernels.  There is no
CPU fallback: if the library cannot be loaded, or no sm_103 GPU is present,
the calls raise.

Feature matrices may be numpy arrays (host) or CUDA torch tensors (device);
torch is only used for device memory and the current CUDA stream.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libabx.so")

FP32_SIMT, FP32, BF16, FP8 = 0, 1, 2, 3
PRECISIONS = {"fp32_simt": FP32_SIMT, "fp32": FP32, "bf16": BF16, "fp8": FP8}
DTW, MEAN = 0, 1
ANGULAR, COSINE, EUCLIDEAN, KL = 0, 1, 2, 3
MEM_HOST, MEM_DEVICE_COPY, MEM_DEVICE_BORROW = 0, 1, 2

_ERRORS = {
    -1: "invalid argument", -2: "zero-norm frame", -3: "out of memory", -4: "CUDA error",
    -5: "unsupported", -6: "state",
}


class AbxError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_ERRORS.get(code, code)}: {msg}")
        self.code = code


class CellsInfo(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in
                ("n_items", "n_groups", "n_blocks", "n_cells", "n_triplets", "max_group")]


class DistInfo(ctypes.Structure):
    _fields_ = [("n_pairs", ctypes.c_int64), ("n_frame_pairs", ctypes.c_int64),
                ("n_tiles", ctypes.c_int64), ("n_frames", ctypes.c_int64),
                ("mode", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("distance", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class ScoreStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in
                ("n_cells", "n_triplets", "n_undecided", "n_recheck_pairs", "n_flips",
                 "num2_total", "count2_total", "n_exact_pairs")]


class TaskInput(ctypes.Structure):
    _fields_ = [("feats", ctypes.c_void_p), ("n_frames", ctypes.c_int64),
                ("dim", ctypes.c_int32), ("mem", ctypes.c_int32),
                ("item_offsets", ctypes.c_void_p), ("n_items", ctypes.c_int64),
                ("labels", ctypes.c_void_p)]


class TaskSpec(ctypes.Structure):
    _fields_ = [("on_attr", ctypes.c_int32), ("n_by", ctypes.c_int32),
                ("by", ctypes.c_int32 * 8), ("across_attr", ctypes.c_int32),
                ("n_level_tokens", ctypes.c_int32), ("levels", ctypes.c_int32 * 16)]


def task_spec(on: int, by: Sequence[int] = (), across: Optional[int] = None,
              levels: Sequence[Sequence[int]] = ()) -> "TaskSpec":
    sp = TaskSpec()
    sp.on_attr = on
    sp.n_by = len(by)
    for i, v in enumerate(by):
        sp.by[i] = v
    sp.across_attr = -1 if across is None else across
    tok, n = _level_tokens(levels)
    sp.n_level_tokens = n
    for i in range(n):
        sp.levels[i] = int(tok[i])
    return sp


SERVER_MAX_SPECS = 4


class ServerConfig(ctypes.Structure):
    _fields_ = [("n_attr", ctypes.c_int32), ("n_specs", ctypes.c_int32),
                ("specs", TaskSpec * SERVER_MAX_SPECS),
                ("mode", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("recheck", ctypes.c_int32), ("weighted", ctypes.c_int32),
                ("margin", ctypes.c_float), ("max_inflight", ctypes.c_int32),
                ("max_batch_jobs", ctypes.c_int32), ("hbm_budget", ctypes.c_int64),
                ("tune", ctypes.c_int32), ("fail_inject", ctypes.c_int32),
                ("n_planners", ctypes.c_int32)]


class JobResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("n_specs", ctypes.c_int32),
                ("errors", ctypes.c_double * SERVER_MAX_SPECS),
                ("triplets", ctypes.c_int64 * SERVER_MAX_SPECS),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_launch", ctypes.c_double), ("t_done", ctypes.c_double),
                ("batch_id", ctypes.c_int64), ("batch_jobs", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("failed", ctypes.c_int64), ("batches", ctypes.c_int64),
                ("max_inflight_seen", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("peak_bytes", ctypes.c_int64), ("cancelled", ctypes.c_int64),
                ("retried", ctypes.c_int64)]


class BatchInfo(ctypes.Structure):
    _fields_ = [("n_tasks", ctypes.c_int32), ("n_classes", ctypes.c_int32),
                ("graph_kernels", ctypes.c_int64), ("n_triplets", ctypes.c_int64),
                ("n_pairs_cap", ctypes.c_int64), ("n_pairs", ctypes.c_int64),
                ("n_frame_pairs", ctypes.c_int64), ("flops", ctypes.c_double),
                ("device_bytes", ctypes.c_int64),
                ("use_graph", ctypes.c_int32), ("tile_variant", ctypes.c_int32 * 8),
                ("dtw_variant", ctypes.c_int32 * 8), ("class_dim", ctypes.c_int32 * 8)]


_lib = None
_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_P = ctypes.POINTER


def lib() -> ctypes.CDLL:
    """Load libabx.so from the package directory (raises if it is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run __graft_entry__.build() or "
                              "python -m paper_2505_02692_b300.build")
        L = ctypes.CDLL(LIB_PATH)
        sig = {
            "abx_last_error": (ctypes.c_char_p, []),
            "abx_version": (ctypes.c_char_p, []),
            "abx_ctx_create": (_i32, [ctypes.c_int, _P(_vp)]),
            "abx_ctx_destroy": (_i32, [_vp]),
            "abx_load_items": (_i32, [_vp, _vp, _i64, _i32, _P(_i64), _i64, _P(_i32), _i32, _i32,
                                      _vp, _P(_vp)]),
            "abx_items_free": (_i32, [_vp]),
            "abx_build_cells": (_i32, [_vp, _vp, _i32, _P(_i32), _i32, _i32, _P(_vp)]),
            "abx_cells_get_info": (_i32, [_vp, _P(CellsInfo)]),
            "abx_cells_free": (_i32, [_vp]),
            "abx_cells_set_subsampler": (_i32, [_vp, _i32, _i32, ctypes.c_uint64]),
            "abx_distances": (_i32, [_vp, _vp, _vp, _i32, _i32, _vp, _P(_vp)]),
            "abx_distances_ex": (_i32, [_vp, _vp, _vp, _i32, _i32, _i32, _vp, _P(_vp)]),
            "abx_dist_get_info": (_i32, [_vp, _P(DistInfo)]),
            "abx_dist_sync": (_i32, [_vp]),
            "abx_dist_lookup": (_i32, [_vp, _i64, _P(_i64), _P(_i64), _P(ctypes.c_float),
                                       _P(ctypes.c_float), _P(ctypes.c_float), _P(_i32)]),
            "abx_dist_free": (_i32, [_vp]),
            "abx_refine_pairs": (_i32, [_vp, _vp, _i64, _P(_i64), _P(_i64), _P(ctypes.c_float),
                                        _P(ctypes.c_float), _vp]),
            "abx_score": (_i32, [_vp, _vp, _vp, _P(_i32), _i32, _i32, _i32, _vp,
                                 _P(ctypes.c_double), _P(ScoreStats)]),
            "abx_score_cells": (_i32, [_vp, _vp, _vp, _i32, _vp, _i64, _P(_i32), _P(_i64),
                                       _P(_i64), _P(_i64)]),
            "abx_score_ex": (_i32, [_vp, _vp, _vp, _P(_i32), _i32, _i32, _i32, ctypes.c_float,
                                    _vp, _P(ctypes.c_double), _P(ScoreStats)]),
            "abx_score_submit": (_i32, [_vp, _vp, _vp, _P(_i32), _i32, _i32, _i32,
                                        ctypes.c_float, _vp, _P(_vp)]),
            "abx_score_wait": (_i32, [_vp, _P(ctypes.c_double), _P(ScoreStats)]),
            "abx_dtw_pairs_noalloc": (_i32, [_vp, _i64, _i32, _P(_i64), _i64, _P(_i64), _i64,
                                             _vp, _vp, _vp]),
            "abx_dtw_pairs_noalloc_check": (_i32, [_vp]),
            "abx_slice_frames": (_i32, [_i64, _i64, _i64, _i32, _P(_i64), _P(_i64)]),
            "abx_slice_items": (_i32, [_i64, _P(_i64), _P(_i64), _i64, _i32, _P(_i64),
                                       _P(_i64)]),
            "abx_batch_create": (_i32, [_vp, _i32, _P(TaskInput), _i32, _i32, _P(_i32), _i32,
                                        _i32, _i32, _i32, _P(_i32), _i32, _i32, _i32,
                                        ctypes.c_float, _i32, _vp, _P(_vp)]),
            "abx_batch_create_multi": (_i32, [_vp, _i32, _P(TaskInput), _i32, _i32, _P(TaskSpec),
                                              _i32, _i32, _i32, _i32, ctypes.c_float, _i32, _vp,
                                              _P(_vp)]),
            "abx_batch_run": (_i32, [_vp, _vp]),
            "abx_batch_ready": (_i32, [_vp]),
            "abx_batch_wait": (_i32, [_vp, _P(ctypes.c_double), _P(_i64), _P(ScoreStats)]),
            "abx_batch_get_info": (_i32, [_vp, _P(BatchInfo)]),
            "abx_batch_set_graph": (_i32, [_vp, _i32]),
            "abx_batch_free": (_i32, [_vp]),
            "abx_server_create": (_i32, [_vp, _P(ServerConfig), _P(_vp)]),
            "abx_server_submit": (_i32, [_vp, _P(TaskInput), _P(_i64)]),
            "abx_server_poll": (_i32, [_vp, _i64, _P(JobResult)]),
            "abx_server_cancel": (_i32, [_vp, _i64]),
            "abx_server_wait": (_i32, [_vp, _i64, _P(JobResult)]),
            "abx_server_get_stats": (_i32, [_vp, _P(ServerStats)]),
            "abx_server_now": (ctypes.c_double, [_vp]),
            "abx_server_destroy": (_i32, [_vp]),
            "abx_kernel_launches": (_i64, []),
            "abx_cosine_error_bound": (ctypes.c_double, [_i32, _i32]),
            "abx_prof_enable": (_i32, [_i32]),
            "abx_prof_reset": (_i32, []),
            "abx_prof_read": (_i32, [_i32, ctypes.c_char_p, _i32, _P(ctypes.c_double),
                                     _P(_i64)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(rc: int):
    if rc != 0:
        raise AbxError(rc, lib().abx_last_error().decode())


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(_P(ct))


def _stream(stream) -> int:
    if stream is not None:
        return int(stream)
    try:
        import torch
        if torch.cuda.is_available() and torch.cuda.is_initialized():
            return int(torch.cuda.current_stream().cuda_stream)
    except Exception:  # noqa: BLE001 -- torch is optional plumbing
        pass
    return 0


def version() -> str:
    return lib().abx_version().decode()


def kernel_launches() -> int:
    """Kernels this library has launched in the process."""
    return int(lib().abx_kernel_launches())


def cosine_error_bound(precision: int, dim: int) -> float:
    """Bound on the cosine error of two stored frames at `precision` (host only)."""
    v = float(lib().abx_cosine_error_bound(int(precision), int(dim)))
    if v < 0:
        raise AbxError(-1, "invalid precision or dimension")
    return v


def prof_enable(on: bool = True):
    _check(lib().abx_prof_enable(int(on)))


def prof_reset():
    _check(lib().abx_prof_reset())


def prof_read():
    """{kernel name: (milliseconds, launches)} accumulated since the reset."""
    out = {}
    i = 0
    buf = ctypes.create_string_buffer(128)
    while True:
        ms = ctypes.c_double()
        n = _i64()
        if lib().abx_prof_read(i, buf, 128, ctypes.byref(ms), ctypes.byref(n)) != 0:
            break
        out[buf.value.decode()] = (ms.value, n.value)
        i += 1
    return out


# ----------------------------------------------------------------- objects

class Context:
    """abx_ctx on one CUDA device."""

    def __init__(self, device: int = 0):
        h = _vp()
        _check(lib().abx_ctx_create(device, ctypes.byref(h)))
        self.h = h
        self.device = device

    def close(self):
        if self.h:
            lib().abx_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass


class Items:
    def __init__(self, ctx: Context, h, n_items: int, keep=None):
        self.ctx, self.h, self.n_items, self._keep = ctx, h, n_items, keep

    def free(self):
        if self.h:
            lib().abx_items_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:  # noqa: BLE001
            pass


class Cells:
    def __init__(self, ctx: Context, items: Items, h, by, across):
        self.ctx, self.items, self.h, self.by, self.across = ctx, items, h, list(by), across

    @property
    def info(self) -> CellsInfo:
        i = CellsInfo()
        _check(lib().abx_cells_get_info(self.h, ctypes.byref(i)))
        return i

    def set_subsampler(self, max_size_group: int = 0, max_x_across: int = 0, seed: int = 0):
        """Subsampler (Sec. 3.1): caps on |A|, |B|, |X| per cell and on the
        across_x values; a seeded SplitMix64 draw (see include/abx.h)."""
        _check(lib().abx_cells_set_subsampler(self.h, int(max_size_group), int(max_x_across),
                                              int(seed) & ((1 << 64) - 1)))

    def free(self):
        if self.h:
            _check(lib().abx_cells_free(self.h))  # fails while a score job is outstanding
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:  # noqa: BLE001
            pass


class Dist:
    def __init__(self, ctx: Context, cells: Cells, h):
        self.ctx, self.cells, self.h = ctx, cells, h

    @property
    def info(self) -> DistInfo:
        i = DistInfo()
        _check(lib().abx_dist_get_info(self.h, ctypes.byref(i)))
        return i

    def sync(self):
        _check(lib().abx_dist_sync(self.h))

    def lookup(self, x, y):
        """(distance, lo, hi, path length) for item pairs (x[k], y[k])."""
        x = np.ascontiguousarray(x, dtype=np.int64)
        y = np.ascontiguousarray(y, dtype=np.int64)
        n = x.size
        d = np.empty(n, np.float32)
        lo = np.empty(n, np.float32)
        hi = np.empty(n, np.float32)
        ln = np.empty(n, np.int32)
        _check(lib().abx_dist_lookup(self.h, n, _ptr(x, _i64), _ptr(y, _i64),
                                     _ptr(d, ctypes.c_float), _ptr(lo, ctypes.c_float),
                                     _ptr(hi, ctypes.c_float), _ptr(ln, _i32)))
        return d, lo, hi, ln

    def free(self):
        if self.h:
            _check(lib().abx_dist_free(self.h))  # fails while a score job is outstanding
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:  # noqa: BLE001
            pass


# ------------------------------------------------------- C-ABI functions

def abx_load_items(ctx: Context, feats, item_offsets, labels, mem: Optional[int] = None,
                   stream=None) -> Items:
    """Register features (numpy host array or CUDA torch tensor) and labels."""
    offs = np.ascontiguousarray(item_offsets, dtype=np.int64)
    lab = np.ascontiguousarray(labels, dtype=np.int32)
    if lab.ndim == 1:
        lab = lab[:, None]
    n_items = offs.size - 1
    keep = None
    if isinstance(feats, np.ndarray):
        f = np.ascontiguousarray(feats, dtype=np.float32)
        ptr, n_frames, dim = f.ctypes.data, f.shape[0], f.shape[1]
        if mem is None:
            mem = MEM_HOST
        keep = f
    else:  # torch tensor
        f = feats
        if not f.is_contiguous() or str(f.dtype) != "torch.float32":
            raise ValueError("feats must be a contiguous float32 tensor")
        ptr, n_frames, dim = f.data_ptr(), f.shape[0], f.shape[1]
        if mem is None:
            mem = MEM_DEVICE_COPY if f.is_cuda else MEM_HOST
        keep = f if mem == MEM_DEVICE_BORROW else None
    h = _vp()
    _check(lib().abx_load_items(ctx.h, ctypes.c_void_p(ptr), n_frames, dim, _ptr(offs, _i64),
                                n_items, _ptr(lab, _i32), lab.shape[1], mem,
                                ctypes.c_void_p(_stream(stream)), ctypes.byref(h)))
    return Items(ctx, h, n_items, keep)


def abx_build_cells(ctx: Context, items: Items, on: int, by: Sequence[int] = (),
                    across: Optional[int] = None) -> Cells:
    b = np.ascontiguousarray(list(by) or [0], dtype=np.int32)
    h = _vp()
    _check(lib().abx_build_cells(ctx.h, items.h, on, _ptr(b, _i32), len(by),
                                 -1 if across is None else across, ctypes.byref(h)))
    return Cells(ctx, items, h, by, across)


def abx_distances(ctx: Context, items: Items, cells: Cells, mode: int = DTW,
                  precision: int = FP32_SIMT, stream=None, distance: int = ANGULAR) -> Dist:
    h = _vp()
    _check(lib().abx_distances_ex(ctx.h, items.h, cells.h, mode, distance, precision,
                                  ctypes.c_void_p(_stream(stream)), ctypes.byref(h)))
    return Dist(ctx, cells, h)


def abx_refine_pairs(ctx: Context, items: Items, x, y, stream=None):
    """Refined recheck stage for item pairs (x[k], y[k]): (lo, hi), an
    interval from TF32 tensor-core products of the FP32 features that holds
    the exact DTW distance."""
    x = np.ascontiguousarray(x, dtype=np.int64)
    y = np.ascontiguousarray(y, dtype=np.int64)
    n = x.size
    if y.size != n:
        raise ValueError("x and y differ in length")
    lo = np.empty(n, np.float32)
    hi = np.empty(n, np.float32)
    _check(lib().abx_refine_pairs(ctx.h, items.h, n, _ptr(x, _i64), _ptr(y, _i64),
                                  _ptr(lo, ctypes.c_float), _ptr(hi, ctypes.c_float),
                                  _stream(stream)))
    return lo, hi


def _level_tokens(levels: Sequence[Sequence[int]]):
    tok = []
    for i, lv in enumerate(levels):
        if isinstance(lv, int):
            lv = (lv,)
        if i:
            tok.append(-1)
        tok.extend(int(a) for a in lv)
    return np.ascontiguousarray(tok or [0], dtype=np.int32), len(tok)


RECHECK_OFF, RECHECK_INTERVAL, RECHECK_MARGIN = 0, 1, 2


def abx_score(ctx: Context, dist: Dist, cells: Cells, levels: Sequence[Sequence[int]] = (),
              weighted: bool = False, recheck=True, stream=None, margin: float = 0.0):
    """(ABX error 1 - D, ScoreStats).  ``recheck``: False/True (intervals) or
    one of RECHECK_OFF / RECHECK_INTERVAL / RECHECK_MARGIN (with ``margin``)."""
    tok, n = _level_tokens(levels)
    err = ctypes.c_double()
    st = ScoreStats()
    mode = int(recheck) if not isinstance(recheck, bool) else (1 if recheck else 0)
    _check(lib().abx_score_ex(ctx.h, dist.h, cells.h, _ptr(tok, _i32), n, int(weighted),
                              mode, float(margin), ctypes.c_void_p(_stream(stream)),
                              ctypes.byref(err), ctypes.byref(st)))
    return err.value, st


class ScoreJob:
    """An enqueued score (abx_score_submit); ``wait()`` gives what abx_score
    returns.  Keeps its distances and cells referenced until waited for."""

    def __init__(self, h, dist: Dist, cells: Cells):
        self.h = h
        self._keep = (dist, cells)

    def wait(self):
        if self.h is None:
            raise AbxError(-6, "score job already waited for")
        err = ctypes.c_double()
        st = ScoreStats()
        h, self.h = self.h, None
        self._keep = None
        _check(lib().abx_score_wait(h, ctypes.byref(err), ctypes.byref(st)))
        return err.value, st

    def __del__(self):
        # a job dropped without a wait still has to release its distances
        # and cells (the library refuses to free them while it is pending)
        if getattr(self, "h", None) is not None:
            try:
                self.wait()
            except Exception:  # noqa: BLE001
                pass


def abx_score_submit(ctx: Context, dist: Dist, cells: Cells,
                     levels: Sequence[Sequence[int]] = (), weighted: bool = False,
                     recheck=True, stream=None, margin: float = 0.0) -> ScoreJob:
    """Enqueue abx_score without waiting; ``.wait()`` on the result returns
    (ABX error, ScoreStats)."""
    tok, n = _level_tokens(levels)
    mode = int(recheck) if not isinstance(recheck, bool) else (1 if recheck else 0)
    h = _vp()
    _check(lib().abx_score_submit(ctx.h, dist.h, cells.h, _ptr(tok, _i32), n, int(weighted),
                                  mode, float(margin), ctypes.c_void_p(_stream(stream)),
                                  ctypes.byref(h)))
    return ScoreJob(h, dist, cells)


def abx_score_cells(ctx: Context, dist: Dist, cells: Cells, recheck: bool = True, stream=None):
    """Per-cell keys (on_ax, on_b, across_ab, across_x, by...), N and |C|."""
    n = _i64()
    z = np.zeros(1, np.int32)
    z64 = np.zeros(1, np.int64)
    s = ctypes.c_void_p(_stream(stream))
    _check(lib().abx_score_cells(ctx.h, dist.h, cells.h, int(recheck), s, 0, _ptr(z, _i32),
                                 _ptr(z64, _i64), _ptr(z64, _i64), ctypes.byref(n)))
    total = n.value
    kw = 4 + len(cells.by)
    keys = np.zeros((max(total, 1), kw), np.int32)
    num2 = np.zeros(max(total, 1), np.int64)
    cnt = np.zeros(max(total, 1), np.int64)
    if total:
        _check(lib().abx_score_cells(ctx.h, dist.h, cells.h, int(recheck), s, total,
                                     _ptr(keys, _i32), _ptr(num2, _i64), _ptr(cnt, _i64),
                                     ctypes.byref(n)))
    return keys[:total], num2[:total], cnt[:total]


def _check_noalloc_buffers(feats, dist, length, n_pairs: int):
    """Reject buffers the C side cannot check (it gets raw device pointers):
    feats a contiguous 2-D float32 CUDA tensor, dist a contiguous float32 CUDA
    tensor of at least n_pairs elements, length (optional) int32 likewise, all
    on one device.  Raises ValueError before anything reaches the library."""
    import torch

    def cuda(t, dtype):
        return (getattr(t, "is_cuda", False) and getattr(t, "dtype", None) == dtype
                and t.is_contiguous())

    if not (cuda(feats, torch.float32) and feats.dim() == 2):
        raise ValueError("feats must be a contiguous 2-D float32 CUDA tensor")
    if not (cuda(dist, torch.float32) and dist.numel() >= n_pairs):
        raise ValueError(f"dist must be a contiguous float32 CUDA tensor of >= {n_pairs} "
                         "elements")
    if length is not None and not (cuda(length, torch.int32) and length.numel() >= n_pairs):
        raise ValueError(f"length must be a contiguous int32 CUDA tensor of >= {n_pairs} "
                         "elements")
    if dist.device != feats.device or (length is not None and length.device != feats.device):
        raise ValueError("feats, dist and length must be on one device")


def abx_dtw_pairs_noalloc(feats, item_offsets, pairs, dist, length=None, stream=None):
    """DTW distances of explicit item pairs without any library allocation.

    ``feats`` (contiguous float32, n_frames x dim), ``dist`` (float32, at
    least n_pairs) and ``length`` (int32, optional) are CUDA torch tensors
    owned by the caller; ``item_offsets`` and ``pairs`` (n_pairs x 2) are host
    arrays.  Pairs with a zero-norm frame get NaN; abx_dtw_pairs_noalloc_check
    reports them."""
    offs = np.ascontiguousarray(item_offsets, dtype=np.int64)
    pr = np.ascontiguousarray(pairs, dtype=np.int64).reshape(-1, 2)
    _check_noalloc_buffers(feats, dist, length, pr.shape[0])
    _check(lib().abx_dtw_pairs_noalloc(
        ctypes.c_void_p(feats.data_ptr()), feats.shape[0], feats.shape[1], _ptr(offs, _i64),
        offs.size - 1, _ptr(pr, _i64), pr.shape[0], ctypes.c_void_p(dist.data_ptr()),
        ctypes.c_void_p(length.data_ptr() if length is not None else 0),
        ctypes.c_void_p(_stream(stream))))


def abx_dtw_pairs_noalloc_check(stream=None):
    """Raise AbxError (ABX_E_ZERO_NORM) if the last abx_dtw_pairs_noalloc call
    met a zero-norm frame; synchronises the stream."""
    _check(lib().abx_dtw_pairs_noalloc_check(ctypes.c_void_p(_stream(stream))))


def abx_slice_items(t_on, t_off, dt: int, libri_light: bool = False):
    """First and last frame (inclusive) kept for each unit (App. A); integer
    times in one unit.  Empty slices have last < first."""
    on = np.ascontiguousarray(t_on, dtype=np.int64)
    off = np.ascontiguousarray(t_off, dtype=np.int64)
    first = np.empty_like(on)
    last = np.empty_like(on)
    _check(lib().abx_slice_items(on.size, _ptr(on, _i64), _ptr(off, _i64), int(dt),
                                 int(libri_light), _ptr(first, _i64), _ptr(last, _i64)))
    return first, last


# ------------------------------------------------------- paper-style API

@dataclass
class Score:
    """Score(task, "angular") of Sec. 3.1, computed by the CUDA path."""
    cells: Cells
    dist: Dist
    recheck: bool = True

    def collapse(self, levels: Sequence[Sequence[int]] = (), weighted: bool = False) -> float:
        err, self.stats = abx_score(self.cells.ctx, self.dist, self.cells, levels, weighted,
                                    self.recheck)
        return err


def score(ctx: Context, items: Items, on: int, by: Sequence[int] = (),
          across: Optional[int] = None, mode: int = DTW, precision: int = FP32_SIMT,
          recheck: bool = True) -> Score:
    cells = abx_build_cells(ctx, items, on, by, across)
    dist = abx_distances(ctx, items, cells, mode, precision)
    return Score(cells, dist, recheck)


# ----------------------------------------------------------------- batches

class Batch:
    """abx_batch: many tasks in shared launches (one CUDA graph per run)."""

    def __init__(self, ctx: Context, h, n_tasks: int, keep, n_specs: int = 1):
        self.ctx, self.h, self.n_tasks, self._keep = ctx, h, n_tasks, keep
        self.n_specs = n_specs

    @property
    def info(self) -> BatchInfo:
        i = BatchInfo()
        _check(lib().abx_batch_get_info(self.h, ctypes.byref(i)))
        return i

    def run(self, stream=None):
        _check(lib().abx_batch_run(self.h, ctypes.c_void_p(_stream(stream))))

    def set_graph(self, on: bool):
        _check(lib().abx_batch_set_graph(self.h, int(on)))

    def ready(self) -> bool:
        rc = lib().abx_batch_ready(self.h)
        if rc < 0:
            _check(rc)
        return rc == 1

    def wait(self):
        """(errors per task, triples per task, ScoreStats totals) of the last run;
        with several specs the arrays are (n_tasks, n_specs)."""
        shape = (self.n_tasks,) if self.n_specs == 1 else (self.n_tasks, self.n_specs)
        err = np.empty(shape, np.float64)
        trip = np.empty(shape, np.int64)
        st = ScoreStats()
        _check(lib().abx_batch_wait(self.h, _ptr(err, ctypes.c_double), _ptr(trip, _i64),
                                    ctypes.byref(st)))
        return err, trip, st

    def free(self):
        if self.h:
            lib().abx_batch_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:  # noqa: BLE001
            pass


def _task_inputs(tasks):
    arr = (TaskInput * len(tasks))()
    keep = []
    n_attr = None
    for k, (feats, offs, labels) in enumerate(tasks):
        o = np.ascontiguousarray(offs, dtype=np.int64)
        lab = np.ascontiguousarray(labels, dtype=np.int32)
        if lab.ndim == 1:
            lab = lab[:, None]
        if n_attr is None:
            n_attr = lab.shape[1]
        if isinstance(feats, np.ndarray):
            f = np.ascontiguousarray(feats, dtype=np.float32)
            ptr, mem = f.ctypes.data, MEM_HOST
        else:
            f = feats
            if not f.is_contiguous() or str(f.dtype) != "torch.float32":
                raise ValueError("feats must be a contiguous float32 tensor")
            ptr, mem = f.data_ptr(), (MEM_DEVICE_COPY if f.is_cuda else MEM_HOST)
        keep.extend([f, o, lab])
        arr[k].feats = ptr
        arr[k].n_frames = f.shape[0]
        arr[k].dim = f.shape[1]
        arr[k].mem = mem
        arr[k].item_offsets = o.ctypes.data
        arr[k].n_items = o.size - 1
        arr[k].labels = lab.ctypes.data
    return arr, keep, n_attr


def abx_batch_create_multi(ctx: Context, tasks, specs, mode: int = DTW, precision: int = FP32,
                           weighted: bool = False, recheck=True, margin: float = 0.0,
                           tune: bool = False, stream=None) -> Batch:
    """Several task specs (see task_spec) over the same tasks, one feature copy."""
    arr, keep, n_attr = _task_inputs(tasks)
    sp = (TaskSpec * len(specs))(*specs)
    rmode = int(recheck) if not isinstance(recheck, bool) else (1 if recheck else 0)
    h = _vp()
    _check(lib().abx_batch_create_multi(ctx.h, len(tasks), arr, n_attr or 1, len(specs), sp,
                                        mode, precision, int(weighted), rmode, float(margin),
                                        int(tune), ctypes.c_void_p(_stream(stream)),
                                        ctypes.byref(h)))
    return Batch(ctx, h, len(tasks), None, len(specs))


def abx_batch_create(ctx: Context, tasks, on: int, by: Sequence[int] = (),
                     across: Optional[int] = None, mode: int = DTW, precision: int = FP32,
                     levels: Sequence[Sequence[int]] = (), weighted: bool = False,
                     recheck=True, margin: float = 0.0, tune: bool = False,
                     stream=None) -> Batch:
    """tasks: sequence of (feats, item_offsets, labels); feats a numpy array or
    a CUDA float32 torch tensor (copied into the batch)."""
    arr, keep, n_attr = _task_inputs(tasks)
    b = np.ascontiguousarray(list(by) or [0], dtype=np.int32)
    tok, n = _level_tokens(levels)
    rmode = int(recheck) if not isinstance(recheck, bool) else (1 if recheck else 0)
    h = _vp()
    _check(lib().abx_batch_create(ctx.h, len(tasks), arr, n_attr or 1, on, _ptr(b, _i32), len(by),
                                  -1 if across is None else across, mode, precision,
                                  _ptr(tok, _i32), n, int(weighted), rmode, float(margin),
                                  int(tune), ctypes.c_void_p(_stream(stream)),
                                  ctypes.byref(h)))
    return Batch(ctx, h, len(tasks), None)


# ----------------------------------------------------------------- serving

class Server:
    """abx_server: continuous batching of ABX jobs on one GPU."""

    def __init__(self, ctx: Context, n_attr: int, specs, mode: int = DTW,
                 precision: int = BF16, recheck=True, margin: float = 0.0,
                 weighted: bool = False, max_inflight: int = 1, max_batch_jobs: int = 32,
                 hbm_budget: int = 0, tune: bool = False, fail_inject: int = 0,
                 n_planners: int = 0):
        cfg = ServerConfig()
        cfg.n_attr = n_attr
        cfg.n_specs = len(specs)
        for i, sp in enumerate(specs):
            cfg.specs[i] = sp
        cfg.mode, cfg.precision, cfg.weighted = mode, precision, int(weighted)
        cfg.recheck = int(recheck) if not isinstance(recheck, bool) else (1 if recheck else 0)
        cfg.margin = float(margin)
        cfg.max_inflight, cfg.max_batch_jobs = max_inflight, max_batch_jobs
        cfg.hbm_budget, cfg.tune = int(hbm_budget), int(tune)
        cfg.fail_inject, cfg.n_planners = int(fail_inject), int(n_planners)
        h = _vp()
        _check(lib().abx_server_create(ctx.h, ctypes.byref(cfg), ctypes.byref(h)))
        self.ctx, self.h, self._keep = ctx, h, {}

    def submit(self, feats, item_offsets, labels) -> int:
        """Queue one job; its buffers are kept alive here until its result is taken.
        The server reads device features on its own streams, so a CUDA tensor's
        pending work on the current stream is waited for first."""
        if not isinstance(feats, np.ndarray) and getattr(feats, "is_cuda", False):
            import torch
            torch.cuda.current_stream(feats.device).synchronize()
        arr, keep, _ = _task_inputs([(feats, item_offsets, labels)])
        t = _i64()
        _check(lib().abx_server_submit(self.h, arr, ctypes.byref(t)))
        self._keep[t.value] = (arr, keep)
        return t.value

    def cancel(self, ticket: int):
        """Remove a job that is still queued (its result: ABX_E_CANCELLED)."""
        _check(lib().abx_server_cancel(self.h, ticket))

    def poll(self, ticket: int):
        r = JobResult()
        rc = lib().abx_server_poll(self.h, ticket, ctypes.byref(r))
        if rc < 0:
            _check(rc)
        if rc == 0:
            return None
        self._keep.pop(ticket, None)
        return r

    def wait(self, ticket: int) -> JobResult:
        r = JobResult()
        _check(lib().abx_server_wait(self.h, ticket, ctypes.byref(r)))
        self._keep.pop(ticket, None)
        return r

    def now(self) -> float:
        return float(lib().abx_server_now(self.h))

    @property
    def stats(self) -> ServerStats:
        st = ServerStats()
        _check(lib().abx_server_get_stats(self.h, ctypes.byref(st)))
        return st

    def close(self):
        if self.h:
            lib().abx_server_destroy(self.h)
            self.h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass
