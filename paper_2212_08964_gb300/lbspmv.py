"""Python binding of liblbspmv (include/lbspmv.h): argument marshalling only.

Every computation runs in the library's CUDA kernels.  PyTorch supplies device memory and
the current stream.  There is no CPU fallback: if the library cannot be built or loaded,
every call raises.

Names follow the C ABI: ``spmv`` (one call, Listing lst:spmv's signature), ``partition``
(the merge-path split, Alg. alg:work-oriented), ``Plan`` (a sparsity structure with its
partition and optional CSC view), ``BatchedPlan`` (many matrices as one block-diagonal
tile set) and ``SpMV`` (a ``torch.autograd.Function`` whose backward runs A^T g over the CSC
view and g[row] * x[col] per nonzero).
"""
from __future__ import annotations

import ctypes
import threading

import numpy as np
import torch

from . import _build

__all__ = [
    "LbError",
    "ensure_loaded",
    "library_path",
    "spmv",
    "spmv_static",
    "partition",
    "num_tiles",
    "Plan",
    "BatchedPlan",
    "CscPlan",
    "SpMV",
    "spmv_autograd",
    "validate_csr",
    "coo_row_offsets",
    "calibrate",
    "sssp",
    "device_error",
    "set_profile_events",
    "SCHEDULES",
    "MERGE_SHAPES",
]

LB_OK = 0
LB_ERR_INVALID_ARG = -1
LB_ERR_UNSUPPORTED = -3
LB_ERR_TIMEOUT = -6
LB_ERR_TOO_LARGE = -7
# Fixed workspace of lb_spmv_static: tiles of STATIC_TILE_ITEMS work items, at most
# STATIC_MAX_TILES of them (m + nnz <= STATIC_MAX_TILES * STATIC_TILE_ITEMS).
STATIC_MAX_TILES = 1 << 19
STATIC_TILE_ITEMS = 248

SCHEDULES = {
    "auto": 0,
    "thread_mapped": 1,
    "warp_mapped": 2,
    "block_mapped": 3,
    "group_mapped": 4,
    "merge_path": 5,
    "nonzero_split": 6,
}
_SCHED_NAMES = {v: k for k, v in SCHEDULES.items()}
# (threads, items per thread) shapes of the merge-path kernel compiled into the library.
MERGE_SHAPES = [(128, 16), (256, 8), (256, 16), (384, 8), (512, 8)]

_DTYPES = {torch.float32: 0, torch.bfloat16: 1, torch.float16: 2}
# A plan's tile sets (lb_plan_tiles): block tiles of the passes over the forward partition,
# warp tiles of the transposed product, warp tiles of the merge-path forward.
TILE_SETS = {"rows": 0, "transposed": 1, "merge": 2}


class LbError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        msg = _lib.lb_status_string(status).decode() if _lib is not None else str(status)
        super().__init__(f"{what}: {msg}")


class _Tuning(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int), ("items_per_thread", ctypes.c_int), ("group_size", ctypes.c_int)]


class Calibration(ctypes.Structure):
    """lb_calibration: measured gather rate and streaming bandwidths of the current GPU."""

    _fields_ = [("gathers_per_s", ctypes.c_double), ("read_GBps", ctypes.c_double), ("copy_GBps", ctypes.c_double)]


class TuneResult(ctypes.Structure):
    """lb_tune_result: a candidate's schedule, resolved launch shape and mean milliseconds."""

    _fields_ = [("schedule", ctypes.c_int), ("tuning", _Tuning), ("ms", ctypes.c_float)]


_lib = None
_lock = threading.Lock()
_P = ctypes.c_void_p
_I = ctypes.c_int


def _declare(lib):
    lib.lb_status_string.restype = ctypes.c_char_p
    lib.lb_status_string.argtypes = [_I]
    lib.lb_version.restype = _I
    sigs = {
        "lb_spmv": [_I, _I, _I, _P, _P, _P, _I, _P, _P, _P],
        "lb_spmv_static": [_I, _I, _I, _P, _P, _P, _I, _P, _P, _P],
        "lb_partition": [_I, _I, _P, _I, _P, _P, _P],
        "lb_plan_create": [_I, _I, _I, _P, _I, ctypes.POINTER(_Tuning), _P, ctypes.POINTER(_P)],
        "lb_plan_info": [_P, ctypes.POINTER(_I), ctypes.POINTER(_Tuning), ctypes.POINTER(_I), ctypes.POINTER(_I)],
        "lb_plan_partition": [_P, _I, _P, _P, ctypes.POINTER(_I)],
        "lb_plan_tiles": [_P, _I, ctypes.POINTER(_I), ctypes.POINTER(_I)],
        "lb_spmv_planned": [_P, _P, _P, _I, _P, _P, _P],
        "lb_plan_build_transpose": [_P, _P, _P],
        "lb_plan_transpose": [_P, _P, _P, _P],
        "lb_spmv_t": [_P, _P, _I, _P, _P, _P],
        "lb_spmv_dvalues": [_P, _P, _P, _P, _P, _I, _P],
        "lb_spmv_planned_save": [_P, _P, _P, _I, _P, _P, _P, _P],
        "lb_spmv_dvalues_gathered": [_P, _P, _P, _P, _I, _P],
        "lb_spmv_backward": [_P, _P, _I, _P, _P, _P, _P, _I, _P],
        "lb_spmv_backward_scatter": [_P, _P, _P, _I, _P, _P, _P, _P, _I, _P],
        "lb_spmm_planned": [_P, _P, _P, _I, _I, _P, _P, _P],
        "lb_coo_row_offsets": [_I, _I, _P, _P, _P, _P],
        "lb_calibrate": [ctypes.POINTER(Calibration), _P],
        "lb_sssp": [_I, _I, _P, _P, _P, _I, _P, ctypes.POINTER(_I), _P],
        "lb_batched_plan_create": [_I, _P, _P, _P, _P, _I, ctypes.POINTER(_Tuning), _P, ctypes.POINTER(_P)],
        "lb_batched_plan_partition": [_P, _P, _P, ctypes.POINTER(_I)],
        "lb_batched_plan_info": [_P, ctypes.POINTER(_Tuning), ctypes.POINTER(_I), ctypes.POINTER(_I)],
        "lb_batched_plan_schedule": [_P, ctypes.POINTER(_I)],
        "lb_spmv_batched": [_P, _P, _P, _I, _P, _P, _P],
        "lb_validate_csr": [_I, _I, _I, _P, _P, _I, _P, _P],
        "lb_device_error": [ctypes.POINTER(_I), _I],
        "lb_set_profile_events": [_P, _P],
        "lb_tune": [_I, _I, _I, _P, _P, _P, _I, _P, _P, _I, _P, _I, ctypes.POINTER(_I), _P],
        "lb_tune_batched": [_I, _P, _P, _P, _P, _P, _P, _I, _P, _P, _I, _P, _I, ctypes.POINTER(_I), _P],
    }
    for name, args in sigs.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = _I
    lib.lb_tune_candidates.argtypes = []
    lib.lb_tune_candidates.restype = _I
    lib.lb_num_tiles.argtypes = [_I, _I, _I]
    lib.lb_num_tiles.restype = _I
    lib.lb_plan_destroy.argtypes = [_P]
    lib.lb_plan_destroy.restype = None
    lib.lb_batched_plan_destroy.argtypes = [_P]
    lib.lb_batched_plan_destroy.restype = None
    lib.lb_debug_fail_allocations_after.argtypes = [_I]
    lib.lb_debug_fail_allocations_after.restype = None
    lib.lb_debug_live_allocations.argtypes = []
    lib.lb_debug_live_allocations.restype = ctypes.c_longlong


def library_path() -> str:
    return _build.LIB


def ensure_loaded():
    """Build (if stale) and load liblbspmv.so; raises if that is impossible."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            lib = ctypes.CDLL(path)
            _declare(lib)
            _lib = lib
    return _lib


def _check(status: int, what: str):
    if status != LB_OK:
        raise LbError(status, what)


def _stream(stream=None) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def _ptr(t: torch.Tensor | None) -> int | None:
    return None if t is None else t.data_ptr()


def _need(t: torch.Tensor, dtype, name: str, numel: int | None = None):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    # The library works on the current device (its workspace, SM count and stream come from
    # it); a tensor on another device would be read through a foreign address.
    if t.device.index != torch.cuda.current_device():
        raise ValueError(
            f"{name} is on cuda:{t.device.index} but the current device is cuda:{torch.cuda.current_device()}"
        )
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, got {t.numel()}")


def _vdt(values: torch.Tensor) -> int:
    try:
        return _DTYPES[values.dtype]
    except KeyError:
        raise TypeError(f"values must be float32, bfloat16 or float16, got {values.dtype}") from None


def _dv_type(dvalues: torch.Tensor, values: torch.Tensor) -> int:
    """The values gradient's storage: float32, or the values' own 16-bit type."""
    if dvalues.dtype != torch.float32 and dvalues.dtype != values.dtype:
        raise TypeError(f"dvalues must be float32 or the values' type {values.dtype}, got {dvalues.dtype}")
    return _vdt(dvalues)


def _tuning(threads=0, items_per_thread=0, group_size=0):
    return _Tuning(int(threads), int(items_per_thread), int(group_size))


def num_tiles(m: int, nnz: int, tile_items: int) -> int:
    return int(ensure_loaded().lb_num_tiles(m, nnz, tile_items))


def spmv(row_offsets, col_idx, values, x, n: int | None = None, out=None, stream=None) -> torch.Tensor:
    """y = A x in one call (lb_spmv); the schedule follows the alpha/beta rule."""
    lib = ensure_loaded()
    m = row_offsets.numel() - 1
    nnz = col_idx.numel()
    n = x.numel() if n is None else n
    _need(row_offsets, torch.int32, "row_offsets")
    _need(col_idx, torch.int32, "col_idx")
    _need(values, None, "values", nnz)
    _need(x, torch.float32, "x", n)
    y = torch.empty(m, dtype=torch.float32, device=x.device) if out is None else out
    _need(y, torch.float32, "y", m)
    _check(
        lib.lb_spmv(m, n, nnz, _ptr(row_offsets), _ptr(col_idx), _ptr(values), _vdt(values), _ptr(x), _ptr(y), _stream(stream)),
        "lb_spmv",
    )
    return y


def spmv_static(row_offsets, col_idx, values, x, out, n: int | None = None, stream=None) -> torch.Tensor:
    """y = A x through lb_spmv_static: merge-path with the library's fixed static workspace,
    no device allocation (the caller provides ``out``).  Calls that overlap in time on one
    device race on that workspace; calls ordered on one stream are safe."""
    lib = ensure_loaded()
    m = row_offsets.numel() - 1
    nnz = col_idx.numel()
    n = x.numel() if n is None else n
    _need(row_offsets, torch.int32, "row_offsets")
    _need(col_idx, torch.int32, "col_idx")
    _need(values, None, "values", nnz)
    _need(x, torch.float32, "x", n)
    _need(out, torch.float32, "out", m)
    _check(
        lib.lb_spmv_static(
            m, n, nnz, _ptr(row_offsets), _ptr(col_idx), _ptr(values), _vdt(values), _ptr(x), _ptr(out), _stream(stream)
        ),
        "lb_spmv_static",
    )
    return out


def partition(row_offsets, nnz: int, tile_items: int, stream=None):
    """Merge-path tile boundaries as two int32 device tensors of G + 1 entries."""
    lib = ensure_loaded()
    m = row_offsets.numel() - 1
    _need(row_offsets, torch.int32, "row_offsets")
    G = num_tiles(m, nnz, tile_items)
    tr = torch.empty(G + 1, dtype=torch.int32, device=row_offsets.device)
    tn = torch.empty(G + 1, dtype=torch.int32, device=row_offsets.device)
    _check(lib.lb_partition(m, nnz, _ptr(row_offsets), tile_items, _ptr(tr), _ptr(tn), _stream(stream)), "lb_partition")
    return tr, tn


class Plan:
    """A sparsity structure prepared once: schedule, partition, carries, optional CSC view."""

    def __init__(self, row_offsets: torch.Tensor, n: int, nnz: int | None = None, schedule: str = "auto",
                 threads: int = 0, items_per_thread: int = 0, group_size: int = 0, stream=None):
        lib = ensure_loaded()
        _need(row_offsets, torch.int32, "row_offsets")
        self.m = row_offsets.numel() - 1
        self.n = int(n)
        self.nnz = int(row_offsets[-1].item()) if nnz is None else int(nnz)
        self.device = row_offsets.device
        self._h = _P()
        t = _tuning(threads, items_per_thread, group_size)
        _check(
            lib.lb_plan_create(self.m, self.n, self.nnz, _ptr(row_offsets), SCHEDULES[schedule], ctypes.byref(t),
                               _stream(stream), ctypes.byref(self._h)),
            "lb_plan_create",
        )
        self._has_t = False

    # -- introspection
    def info(self) -> dict:
        s, t, g, ti = _I(), _Tuning(), _I(), _I()
        _check(_lib.lb_plan_info(self._h, ctypes.byref(s), ctypes.byref(t), ctypes.byref(g), ctypes.byref(ti)), "lb_plan_info")
        return {
            "schedule": _SCHED_NAMES[s.value],
            "threads": t.threads,
            "items_per_thread": t.items_per_thread,
            "group_size": t.group_size,
            "num_tiles": g.value,
            "tile_items": ti.value,
        }

    def tiles(self, which: str = "rows") -> tuple[int, int]:
        """(num_tiles, tile_items) of one tile set: "rows" (the block-level passes), "merge"
        (the merge-path forward's warp tiles) or "transposed" (the transposed product's)."""
        g, ti = _I(), _I()
        _check(_lib.lb_plan_tiles(self._h, TILE_SETS[which], ctypes.byref(g), ctypes.byref(ti)), "lb_plan_tiles")
        return g.value, ti.value

    def partition(self, transposed: bool = False, which: str | None = None):
        """Host copy (tile_row, tile_nz) of a tile set: ``which`` as in ``tiles``; by default the
        "rows" set, or "transposed" with ``transposed=True``."""
        w = TILE_SETS[which if which is not None else ("transposed" if transposed else "rows")]
        g = _I()
        _check(_lib.lb_plan_partition(self._h, w, None, None, ctypes.byref(g)), "lb_plan_partition")
        tr = np.empty(g.value + 1, np.int32)
        tn = np.empty(g.value + 1, np.int32)
        _check(_lib.lb_plan_partition(self._h, w, tr.ctypes.data, tn.ctypes.data, ctypes.byref(g)), "lb_plan_partition")
        return tr, tn

    # -- forward
    def spmv(self, col_idx, values, x, out=None, stream=None, save_gathered=None) -> torch.Tensor:
        """y = A x.  With ``save_gathered`` (nnz float32), also x[col_idx[k]] for every nonzero
        (lb_spmv_planned_save; merge-path plans), for ``dvalues_gathered``."""
        _need(col_idx, torch.int32, "col_idx", self.nnz)
        _need(values, None, "values", self.nnz)
        _need(x, torch.float32, "x", self.n)
        y = torch.empty(self.m, dtype=torch.float32, device=x.device) if out is None else out
        _need(y, torch.float32, "y", self.m)
        if save_gathered is None:
            _check(_lib.lb_spmv_planned(self._h, _ptr(col_idx), _ptr(values), _vdt(values), _ptr(x), _ptr(y),
                                        _stream(stream)), "lb_spmv_planned")
        else:
            _need(save_gathered, torch.float32, "save_gathered", self.nnz)
            _check(_lib.lb_spmv_planned_save(self._h, _ptr(col_idx), _ptr(values), _vdt(values), _ptr(x), _ptr(y),
                                             _ptr(save_gathered), _stream(stream)), "lb_spmv_planned_save")
        return y

    def spmm(self, col_idx, values, B, out=None, stream=None) -> torch.Tensor:
        """C = A B (lb_spmm_planned): B float32 (n, kc) row-major, C float32 (m, kc)."""
        _need(col_idx, torch.int32, "col_idx", self.nnz)
        _need(values, None, "values", self.nnz)
        if B.dim() != 2 or B.shape[0] != self.n:
            raise ValueError(f"B must be ({self.n}, kc), got {tuple(B.shape)}")
        _need(B, torch.float32, "B")
        kc = B.shape[1]
        C = torch.empty((self.m, kc), dtype=torch.float32, device=B.device) if out is None else out
        if C.shape != (self.m, kc):
            raise ValueError(f"out must be ({self.m}, {kc})")
        _need(C, torch.float32, "out")
        _check(_lib.lb_spmm_planned(self._h, _ptr(col_idx), _ptr(values), _vdt(values), kc, _ptr(B), _ptr(C),
                                    _stream(stream)), "lb_spmm_planned")
        return C

    # -- backward
    def build_transpose(self, col_idx, stream=None):
        _need(col_idx, torch.int32, "col_idx", self.nnz)
        _check(_lib.lb_plan_build_transpose(self._h, _ptr(col_idx), _stream(stream)), "lb_plan_build_transpose")
        self._has_t = True

    @property
    def has_transpose(self) -> bool:
        return self._has_t

    def transpose(self):
        co = np.empty(self.n + 1, np.int32)
        ri = np.empty(max(self.nnz, 1), np.int32)
        perm = np.empty(max(self.nnz, 1), np.int32)
        _check(_lib.lb_plan_transpose(self._h, co.ctypes.data, ri.ctypes.data, perm.ctypes.data), "lb_plan_transpose")
        return co, ri[: self.nnz], perm[: self.nnz]

    def spmv_t(self, values, g, out=None, stream=None) -> torch.Tensor:
        _need(values, None, "values", self.nnz)
        _need(g, torch.float32, "g", self.m)
        dx = torch.empty(self.n, dtype=torch.float32, device=g.device) if out is None else out
        _need(dx, torch.float32, "dx", self.n)
        _check(_lib.lb_spmv_t(self._h, _ptr(values), _vdt(values), _ptr(g), _ptr(dx), _stream(stream)), "lb_spmv_t")
        return dx

    def dvalues(self, col_idx, g, x, out=None, stream=None, dtype=torch.float32) -> torch.Tensor:
        """dvalues[k] = g[row(k)] * x[col_idx[k]] gathering x; stored in ``out``'s type (else
        ``dtype``): float32, or bfloat16/float16 rounded to nearest even."""
        _need(col_idx, torch.int32, "col_idx", self.nnz)
        _need(g, torch.float32, "g", self.m)
        _need(x, torch.float32, "x", self.n)
        dv = torch.empty(self.nnz, dtype=dtype, device=g.device) if out is None else out
        _need(dv, None, "dvalues", self.nnz)
        _check(_lib.lb_spmv_dvalues(self._h, _ptr(col_idx), _ptr(g), _ptr(x), _ptr(dv), _vdt(dv), _stream(stream)),
               "lb_spmv_dvalues")
        return dv

    def backward(self, values, g, x_gathered, dx=None, dvalues=None, stream=None, dvalues_dtype=torch.float32):
        """(dx, dvalues) = (A^T g, g[row] * x_gathered) in two passes (lb_spmv_backward);
        needs ``build_transpose`` and x gathers saved by ``spmv(save_gathered=...)``.  dvalues
        is float32 or the values' 16-bit type (``dvalues``' own type, else ``dvalues_dtype``)."""
        _need(values, None, "values", self.nnz)
        _need(g, torch.float32, "g", self.m)
        _need(x_gathered, torch.float32, "x_gathered", self.nnz)
        dx = torch.empty(self.n, dtype=torch.float32, device=g.device) if dx is None else dx
        dvalues = torch.empty(self.nnz, dtype=dvalues_dtype, device=g.device) if dvalues is None else dvalues
        _need(dx, torch.float32, "dx", self.n)
        _need(dvalues, None, "dvalues", self.nnz)
        _check(_lib.lb_spmv_backward(self._h, _ptr(values), _vdt(values), _ptr(g), _ptr(x_gathered), _ptr(dx),
                                     _ptr(dvalues), _dv_type(dvalues, values), _stream(stream)), "lb_spmv_backward")
        return dx, dvalues

    def backward_scatter(self, col_idx, values, g, x_gathered=None, dx=None, dvalues=None, want_dvalues=True,
                         stream=None, dvalues_dtype=torch.float32):
        """(dx, dvalues) in one CSR-order pass without a CSC view (lb_spmv_backward_scatter):
        dx by float reductions into dx[col] (within tolerance, not bit-reproducible), dvalues
        as ``backward`` (bit-exact; needs ``x_gathered``).  dvalues is None when not wanted."""
        _need(col_idx, torch.int32, "col_idx", self.nnz)
        _need(values, None, "values", self.nnz)
        _need(g, torch.float32, "g", self.m)
        dx = torch.empty(self.n, dtype=torch.float32, device=g.device) if dx is None else dx
        _need(dx, torch.float32, "dx", self.n)
        if want_dvalues:
            _need(x_gathered, torch.float32, "x_gathered", self.nnz)
            dvalues = torch.empty(self.nnz, dtype=dvalues_dtype, device=g.device) if dvalues is None else dvalues
            _need(dvalues, None, "dvalues", self.nnz)
        else:
            dvalues = None
        _check(_lib.lb_spmv_backward_scatter(self._h, _ptr(col_idx), _ptr(values), _vdt(values), _ptr(g),
                                             _ptr(x_gathered) if x_gathered is not None else None, _ptr(dx),
                                             _ptr(dvalues) if dvalues is not None else None,
                                             _dv_type(dvalues, values) if dvalues is not None else 0,
                                             _stream(stream)),
               "lb_spmv_backward_scatter")
        return dx, dvalues

    def dvalues_gathered(self, g, x_gathered, out=None, stream=None, dtype=torch.float32) -> torch.Tensor:
        """dvalues[k] = g[row(k)] * x_gathered[k] (x gathers saved by ``spmv(save_gathered=...)``),
        stored in ``out``'s type (else ``dtype``), as ``dvalues``."""
        _need(g, torch.float32, "g", self.m)
        _need(x_gathered, torch.float32, "x_gathered", self.nnz)
        dv = torch.empty(self.nnz, dtype=dtype, device=g.device) if out is None else out
        _need(dv, None, "dvalues", self.nnz)
        _check(_lib.lb_spmv_dvalues_gathered(self._h, _ptr(g), _ptr(x_gathered), _ptr(dv), _vdt(dv), _stream(stream)),
               "lb_spmv_dvalues_gathered")
        return dv

    def close(self):
        if getattr(self, "_h", None) and self._h.value and _lib is not None:
            _lib.lb_plan_destroy(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class CscPlan:
    """y = A x for A given in CSC form: col_offsets (n + 1), row_idx (nnz) and values in CSC
    order.  A CSC matrix is its transpose in CSR form, so this is a Plan of A^T (n rows, m
    columns) with its CSC view, which is A in CSR, built once; y = A x is that plan's
    transposed product (lb_spmv_t): a streaming pass over A's columns scales each value by
    x[col] (x is read in column order), then the merge-path gather-sum over A's rows adds them
    up.  Merge-path serves any format with an atoms-per-tile count (Ch.4 Sec. "Merge-path load
    balancing"; CSC as a format, Ch.4 Sec. "Implementing Sparse Data Structures").  With A's
    columns sorted by row, the rows are summed in the order of A's CSR form, over the same
    partition and with the same products as the CSR forward."""

    def __init__(self, col_offsets: torch.Tensor, row_idx: torch.Tensor, m: int, nnz: int | None = None,
                 schedule: str = "merge_path", threads: int = 0, items_per_thread: int = 0, stream=None):
        self.plan = Plan(col_offsets, m, nnz, schedule=schedule, threads=threads, items_per_thread=items_per_thread,
                         stream=stream)
        self.plan.build_transpose(row_idx, stream=stream)
        self.m = int(m)
        self.n = self.plan.m
        self.nnz = self.plan.nnz

    def spmv(self, values, x, out=None, stream=None) -> torch.Tensor:
        """y (m floats) = A x, x: n floats; values FP32, BF16 or FP16 in CSC order."""
        return self.plan.spmv_t(values, x, out=out, stream=stream)

    def close(self):
        self.plan.close()


class BatchedPlan:
    """K CSR matrices run as one block-diagonal matrix in one launch: the global merge path
    (``schedule="merge_path"``, with the fixup) or a row per lane with long rows summed by
    the warp (``schedule="thread_mapped"``, no fixup)."""

    def __init__(self, ms, ns, nnzs, row_offsets_concat: torch.Tensor, threads: int = 0, items_per_thread: int = 0,
                 stream=None, schedule: str = "merge_path"):
        lib = ensure_loaded()
        _need(row_offsets_concat, torch.int32, "row_offsets_concat")
        self.ms = np.ascontiguousarray(ms, np.int32)
        self.ns = np.ascontiguousarray(ns, np.int32)
        self.nnzs = np.ascontiguousarray(nnzs, np.int32)
        self.count = int(self.ms.shape[0])
        self.total_rows = int(self.ms.astype(np.int64).sum())
        self.total_cols = int(self.ns.astype(np.int64).sum())
        self.total_nnz = int(self.nnzs.astype(np.int64).sum())
        self._h = _P()
        t = _tuning(threads, items_per_thread, 0)
        _check(
            lib.lb_batched_plan_create(self.count, self.ms.ctypes.data, self.ns.ctypes.data, self.nnzs.ctypes.data,
                                       _ptr(row_offsets_concat), SCHEDULES[schedule], ctypes.byref(t), _stream(stream),
                                       ctypes.byref(self._h)),
            "lb_batched_plan_create",
        )

    def info(self) -> dict:
        t, g, ti = _Tuning(), _I(), _I()
        _check(_lib.lb_batched_plan_info(self._h, ctypes.byref(t), ctypes.byref(g), ctypes.byref(ti)), "lb_batched_plan_info")
        s = _I()
        _check(_lib.lb_batched_plan_schedule(self._h, ctypes.byref(s)), "lb_batched_plan_schedule")
        return {"schedule": _SCHED_NAMES[s.value], "threads": t.threads, "items_per_thread": t.items_per_thread,
                "num_tiles": g.value, "tile_items": ti.value}

    def partition(self):
        g = _I()
        _check(_lib.lb_batched_plan_partition(self._h, None, None, ctypes.byref(g)), "lb_batched_plan_partition")
        tr = np.empty(g.value + 1, np.int32)
        tn = np.empty(g.value + 1, np.int32)
        _check(_lib.lb_batched_plan_partition(self._h, tr.ctypes.data, tn.ctypes.data, ctypes.byref(g)), "lb_batched_plan_partition")
        return tr, tn

    def spmv(self, col_idx, values, x, out=None, stream=None) -> torch.Tensor:
        _need(col_idx, torch.int32, "col_idx", self.total_nnz)
        _need(values, None, "values", self.total_nnz)
        _need(x, torch.float32, "x", self.total_cols)
        y = torch.empty(self.total_rows, dtype=torch.float32, device=x.device) if out is None else out
        _need(y, torch.float32, "y", self.total_rows)
        _check(_lib.lb_spmv_batched(self._h, _ptr(col_idx), _ptr(values), _vdt(values), _ptr(x), _ptr(y), _stream(stream)),
               "lb_spmv_batched")
        return y

    def close(self):
        if getattr(self, "_h", None) and self._h.value and _lib is not None:
            _lib.lb_batched_plan_destroy(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class SpMV(torch.autograd.Function):
    """y = A x with gradients for the values and for x.

    Backward: dx = A^T g by merge-path over the plan's CSC view (built on first use),
    dvalues = g[row] * x[col] per nonzero over the forward partition.  When the values need a
    gradient and the plan is merge-path, the forward saves x[col] of every nonzero (4 bytes per
    nonzero) and the backward streams them back instead of gathering x again; with both
    gradients wanted, one pass over the nonzeros forms dvalues and the scaled values for dx.
    With ``deterministic=False`` dx comes from ``Plan.backward_scatter`` instead: one pass, no
    CSC view, dx not bit-reproducible (within the same tolerance).
    """

    @staticmethod
    def forward(ctx, values, x, plan: Plan, col_idx, deterministic: bool = True):
        ctx.plan = plan
        ctx.deterministic = deterministic
        xg = None
        if ctx.needs_input_grad[0] and plan.info()["schedule"] == "merge_path":
            xg = torch.empty(plan.nnz, dtype=torch.float32, device=x.device)
        ctx.save_for_backward(values, x, col_idx, xg)
        return plan.spmv(col_idx, values.detach(), x.detach(), save_gathered=xg)

    @staticmethod
    def backward(ctx, g):
        values, x, col_idx, xg = ctx.saved_tensors
        plan = ctx.plan
        g = g.contiguous().float()
        dvals = dx = None
        # The values gradient takes the values' type, rounded in the library's kernels.
        dvt = values.dtype
        if not ctx.deterministic and ctx.needs_input_grad[1]:
            want_dv = ctx.needs_input_grad[0] and xg is not None
            dx, dvals = plan.backward_scatter(col_idx, values.detach(), g, xg, want_dvalues=want_dv,
                                              dvalues_dtype=dvt)
            if ctx.needs_input_grad[0] and dvals is None:
                dvals = plan.dvalues(col_idx, g, x.detach(), dtype=dvt)
            return dvals, dx, None, None, None
        if ctx.needs_input_grad[1] and not plan.has_transpose:
            plan.build_transpose(col_idx)
        if ctx.needs_input_grad[0] and ctx.needs_input_grad[1] and xg is not None:
            dx, dvals = plan.backward(values.detach(), g, xg, dvalues_dtype=dvt)  # both in two passes
        else:
            if ctx.needs_input_grad[0]:
                dvals = (plan.dvalues(col_idx, g, x.detach(), dtype=dvt) if xg is None
                         else plan.dvalues_gathered(g, xg, dtype=dvt))
            if ctx.needs_input_grad[1]:
                dx = plan.spmv_t(values.detach(), g)
        return dvals, dx, None, None, None


def spmv_autograd(plan: Plan, col_idx, values, x, deterministic: bool = True):
    """Differentiable y = A x (see ``SpMV``); ``deterministic=False`` takes dx from the
    one-pass scatter backward (no CSC view; not bit-reproducible)."""
    return SpMV.apply(values, x, plan, col_idx, deterministic)


def coo_row_offsets(row_idx, m: int, stream=None):
    """CSR row offsets (int32 device tensor of m + 1) of a row-sorted COO matrix, and the check
    mask (1: row out of range, 2: rows decrease; 0: valid); reading the mask synchronizes."""
    lib = ensure_loaded()
    _need(row_idx, torch.int32, "row_idx")
    ro = torch.empty(m + 1, dtype=torch.int32, device=row_idx.device)
    status = torch.zeros(1, dtype=torch.int32, device=row_idx.device)
    _check(lib.lb_coo_row_offsets(m, row_idx.numel(), _ptr(row_idx) if row_idx.numel() else None, _ptr(ro),
                                  _ptr(status), _stream(stream)), "lb_coo_row_offsets")
    return ro, int(status.item())


def sssp(row_offsets, col_idx, weights=None, source: int = 0, out=None, stream=None):
    """Shortest-path distances from `source` over a CSR graph (lb_sssp); weights None: unit
    weights (BFS levels).  Returns (dist float32 tensor, frontier iterations)."""
    lib = ensure_loaded()
    _need(row_offsets, torch.int32, "row_offsets")
    _need(col_idx, torch.int32, "col_idx")
    n = row_offsets.numel() - 1
    nnz = col_idx.numel()
    if weights is not None:
        _need(weights, torch.float32, "weights", nnz)
    dist = torch.empty(n, dtype=torch.float32, device=row_offsets.device) if out is None else out
    _need(dist, torch.float32, "dist", n)
    it = _I()
    _check(lib.lb_sssp(n, nnz, _ptr(row_offsets), _ptr(col_idx) if nnz else None, _ptr(weights), int(source),
                       _ptr(dist), ctypes.byref(it), _stream(stream)), "lb_sssp")
    return dist, it.value


def calibrate(stream=None) -> dict:
    """Measured ceilings of the current GPU (lb_calibrate): gathers per second and streaming
    read / copy GB/s."""
    lib = ensure_loaded()
    c = Calibration()
    _check(lib.lb_calibrate(ctypes.byref(c), _stream(stream)), "lb_calibrate")
    return {"gathers_per_s": c.gathers_per_s, "read_GBps": c.read_GBps, "copy_GBps": c.copy_GBps}


def validate_csr(row_offsets, col_idx, n: int, check_sorted: bool = True, stream=None) -> int:
    """Bit mask of problems found on the device (0 = valid); synchronizes to read it."""
    lib = ensure_loaded()
    m = row_offsets.numel() - 1
    nnz = col_idx.numel()
    status = torch.zeros(1, dtype=torch.int32, device=row_offsets.device)
    _check(lib.lb_validate_csr(m, n, nnz, _ptr(row_offsets), _ptr(col_idx) if nnz else None, int(check_sorted), _ptr(status),
                               _stream(stream)), "lb_validate_csr")
    return int(status.item())


def device_error(clear: bool = True) -> int:
    """The device error word (0, or LB_ERR_BAD_MATRIX after a malformed tile); synchronizes."""
    lib = ensure_loaded()
    s = _I()
    _check(lib.lb_device_error(ctypes.byref(s), int(clear)), "lb_device_error")
    return s.value


def set_profile_events(before: torch.cuda.Event | None, after: torch.cuda.Event | None):
    """Record `before`/`after` around every merge-path main kernel (None to stop)."""
    lib = ensure_loaded()
    b = before.cuda_event if before is not None else None
    a = after.cuda_event if after is not None else None
    _check(lib.lb_set_profile_events(b, a), "lb_set_profile_events")


def fail_allocations_after(count: int):
    """Test support: the library's next `count` device allocations proceed, later ones fail
    as if the device were full (LB_ERR_NO_MEMORY); a negative count removes the limit."""
    ensure_loaded().lb_debug_fail_allocations_after(int(count))


def live_allocations() -> int:
    """The library's device allocations currently held."""
    return int(ensure_loaded().lb_debug_live_allocations())
