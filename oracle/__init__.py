"""CPU oracle for load-balanced CSR SpMV -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference leg of
``bench.py`` may import this package.  The product path (``paper_2212_08964_gb300``)
never imports it and shares no code with it.

The arithmetic lives in ``oracle.c`` (plain C, FP64, one definition per function, each
citing the dissertation's section, algorithm or listing).  This module builds that
library with gcc, wraps it with ctypes, and adds two small pure-Python pieces used to
pin it: an explicit step-by-step merge of row ends and nonzeros (the merge that
Alg. alg:work-oriented's 2DSearch walks along), and the block-diagonal view of a batch.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i64 = ctypes.c_int64


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, OpenMP) unless it is up to date."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_max_threads.restype = ctypes.c_int
            lib.oracle_spmv_f64.argtypes = [_i64, _i32p, _i32p, _f64p, _f64p, _f64p, ctypes.c_int]
            lib.oracle_row_absdot.argtypes = [_i64, _i32p, _i32p, _f64p, _f64p, _f64p, ctypes.c_int]
            lib.oracle_merge_split.argtypes = [_i64, _i32p, _i64, ctypes.POINTER(_i64), ctypes.POINTER(_i64)]
            lib.oracle_num_tiles.argtypes = [_i64, _i64, _i64]
            lib.oracle_num_tiles.restype = _i64
            lib.oracle_partition.argtypes = [_i64, _i32p, _i64, _i32p, _i32p]
            lib.oracle_partition.restype = _i64
            lib.oracle_transpose.argtypes = [_i64, _i64, _i32p, _i32p, _i32p, _i32p, _i32p]
            lib.oracle_spmv_t_f64.argtypes = [_i64, _i64, _i32p, _i32p, _f64p, _f64p, _f64p, ctypes.c_int]
            lib.oracle_col_absdot.argtypes = [_i64, _i64, _i32p, _i32p, _f64p, _f64p, _f64p]
            lib.oracle_dvalues_f64.argtypes = [_i64, _i32p, _i32p, _f64p, _f64p, _f64p, ctypes.c_int]
            lib.oracle_spmm_f64.argtypes = [_i64, _i64, _i32p, _i32p, _f64p, _f64p, _f64p, ctypes.c_int]
            lib.oracle_spmm_absdot.argtypes = [_i64, _i64, _i32p, _i32p, _f64p, _f64p, _f64p, ctypes.c_int]
            lib.oracle_sssp_f64.argtypes = [_i64, _i32p, _i32p, ctypes.c_void_p, _i64, _f64p]
            lib.oracle_sssp_f64.restype = ctypes.c_int
            _lib = lib
    return _lib


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def spmv(ro, ci, v, x, threads: int = 0) -> np.ndarray:
    """y = A x in FP64 (Listing lst:spmv)."""
    ro = _c(ro, np.int32)
    m = ro.shape[0] - 1
    y = np.empty(m, np.float64)
    _load().oracle_spmv_f64(m, ro, _c(ci, np.int32), _c(v, np.float64), _c(x, np.float64), y, threads)
    return y


def spmm(ro, ci, v, B, threads: int = 0) -> np.ndarray:
    """C = A B in FP64, B dense n x kc (row-major): SpMV with a loop over B's columns."""
    ro = _c(ro, np.int32)
    B = np.ascontiguousarray(B, np.float64)
    m = ro.shape[0] - 1
    kc = B.shape[1]
    C = np.empty((m, kc), np.float64)
    _load().oracle_spmm_f64(m, kc, ro, _c(ci, np.int32), _c(v, np.float64), B.reshape(-1), C.reshape(-1), threads)
    return C


def spmm_absdot(ro, ci, v, B, threads: int = 0) -> np.ndarray:
    """sum_k |v_k||B[ci_k][j]| per entry of C."""
    ro = _c(ro, np.int32)
    B = np.ascontiguousarray(B, np.float64)
    m = ro.shape[0] - 1
    kc = B.shape[1]
    S = np.empty((m, kc), np.float64)
    _load().oracle_spmm_absdot(m, kc, ro, _c(ci, np.int32), _c(v, np.float64), B.reshape(-1), S.reshape(-1), threads)
    return S


def sssp(ro, ci, w, source: int) -> np.ndarray:
    """Shortest-path distances from `source` over a CSR graph (Dijkstra, FP64); w None: unit
    weights (BFS levels).  +inf for unreachable vertices."""
    ro = _c(ro, np.int32)
    n = ro.shape[0] - 1
    dist = np.empty(n, np.float64)
    wp = None
    if w is not None:
        w = _c(w, np.float64)
        wp = w.ctypes.data_as(ctypes.c_void_p)
    rc = _load().oracle_sssp_f64(n, ro, _c(ci, np.int32), wp, int(source), dist)
    if rc != 0:
        raise ValueError(f"oracle_sssp_f64 failed ({rc})")
    return dist


def row_absdot(ro, ci, v, x, threads: int = 0) -> np.ndarray:
    """sum_j |a_ij||x_j| per row."""
    ro = _c(ro, np.int32)
    m = ro.shape[0] - 1
    s = np.empty(m, np.float64)
    _load().oracle_row_absdot(m, ro, _c(ci, np.int32), _c(v, np.float64), _c(x, np.float64), s, threads)
    return s


def merge_split(ro, d: int):
    """(i, j) = split(d) by the counting definition."""
    ro = _c(ro, np.int32)
    i, j = _i64(), _i64()
    _load().oracle_merge_split(ro.shape[0] - 1, ro, int(d), ctypes.byref(i), ctypes.byref(j))
    return int(i.value), int(j.value)


def num_tiles(m: int, nnz: int, T: int) -> int:
    return int(_load().oracle_num_tiles(m, nnz, T))


def partition(ro, T: int):
    """Tile boundaries (tile_row, tile_nz), G+1 entries each, for tiles of T work items."""
    ro = _c(ro, np.int32)
    m = ro.shape[0] - 1
    nnz = int(ro[-1]) if m > 0 else 0
    G = num_tiles(m, nnz, T)
    tr = np.empty(G + 1, np.int32)
    tn = np.empty(G + 1, np.int32)
    _load().oracle_partition(m, ro, int(T), tr, tn)
    return tr, tn


def transpose(ro, ci, n: int):
    """Stable CSR -> CSC: (col_offsets[n+1], row_idx[nnz], perm[nnz])."""
    ro = _c(ro, np.int32)
    m = ro.shape[0] - 1
    nnz = int(ro[-1]) if m > 0 else 0
    co = np.empty(n + 1, np.int32)
    ri = np.empty(max(nnz, 1), np.int32)
    perm = np.empty(max(nnz, 1), np.int32)
    _load().oracle_transpose(m, n, ro, _c(ci, np.int32), co, ri, perm)
    return co, ri[:nnz], perm[:nnz]


def spmv_t(ro, ci, v, g, n: int, threads: int = 0) -> np.ndarray:
    """dx = A^T g in FP64, each column summed in CSC order."""
    ro = _c(ro, np.int32)
    m = ro.shape[0] - 1
    dx = np.empty(n, np.float64)
    _load().oracle_spmv_t_f64(m, n, ro, _c(ci, np.int32), _c(v, np.float64), _c(g, np.float64), dx, threads)
    return dx


def col_absdot(ro, ci, v, g, n: int) -> np.ndarray:
    """sum_i |a_ij||g_i| per column."""
    ro = _c(ro, np.int32)
    s = np.empty(n, np.float64)
    _load().oracle_col_absdot(ro.shape[0] - 1, n, ro, _c(ci, np.int32), _c(v, np.float64), _c(g, np.float64), s)
    return s


def dvalues(ro, ci, g, x, threads: int = 0) -> np.ndarray:
    """dv_k = g[row(k)] x[ci_k] in FP64."""
    ro = _c(ro, np.int32)
    m = ro.shape[0] - 1
    nnz = int(ro[-1]) if m > 0 else 0
    dv = np.empty(max(nnz, 1), np.float64)
    _load().oracle_dvalues_f64(m, ro, _c(ci, np.int32), _c(g, np.float64), _c(x, np.float64), dv, threads)
    return dv[:nnz]


# ---------------------------------------------------------------------------------------
# Pure-Python pieces (small inputs only).

def explicit_merge(ro):
    """Walk the merge of row ends and nonzero indices one item at a time.

    Returns the merged sequence as a list of ("R", r) / ("N", k).  At each step the next
    row end R_r (key ro[r+1]) is taken when ro[r+1] <= k for the next nonzero k, i.e. when
    the row has no nonzeros left; otherwise nonzero k is taken (Alg. alg:work-oriented:
    a row's nonzeros are consumed while k < offsets[row + 1], then the row's output).
    """
    ro = [int(v) for v in ro]
    m = len(ro) - 1
    nnz = ro[-1] if m > 0 else 0
    r, k, out = 0, 0, []
    while r < m or k < nnz:
        if r < m and (k >= nnz or ro[r + 1] <= k):
            out.append(("R", r))
            r += 1
        else:
            out.append(("N", k))
            k += 1
    return out


def block_diagonal_offsets(ms, nnzs, row_offsets_concat) -> np.ndarray:
    """Row offsets of the block-diagonal matrix diag(A_0, ..., A_{K-1}).

    Matrix i's local offsets (m_i+1 entries starting at 0) are shifted by the number of
    nonzeros of the matrices before it; the leading zero of every matrix after the first
    is dropped.
    """
    parts = [np.zeros(1, np.int64)]
    ro_pos = 0
    nz_base = 0
    for m, nnz in zip(ms, nnzs):
        m, nnz = int(m), int(nnz)
        local = np.asarray(row_offsets_concat[ro_pos : ro_pos + m + 1], np.int64)
        parts.append(local[1:] + nz_base)
        ro_pos += m + 1
        nz_base += nnz
    return np.concatenate(parts).astype(np.int32)


def batched_spmv(b, x_concat, threads: int = 0):
    """Per-matrix oracle SpMV of a batch, concatenated (y_i = A_i x_i)."""
    ys = []
    x_pos = 0
    for i in range(b.count):
        a = b.matrix(i)
        ys.append(spmv(a.row_offsets, a.col_idx, a.values, x_concat[x_pos : x_pos + a.n], threads))
        x_pos += a.n
    return np.concatenate(ys) if ys else np.zeros(0)


def batched_row_absdot(b, x_concat, threads: int = 0):
    out = []
    x_pos = 0
    for i in range(b.count):
        a = b.matrix(i)
        out.append(row_absdot(a.row_offsets, a.col_idx, a.values, x_concat[x_pos : x_pos + a.n], threads))
        x_pos += a.n
    return np.concatenate(out) if out else np.zeros(0)


def loss(ro, ci, v, x, t) -> float:
    """L = 1/2 ||A x - t||^2 in FP64."""
    r = spmv(ro, ci, v, x) - np.asarray(t, np.float64)
    return 0.5 * float(r @ r)
