"""Autotuner: schedule and launch shape per matrix-shape class, chosen by measurement.

The dissertation chooses between its schedules with a fixed rule of matrix size (Ch.4 Sec.
"Improved Performance Response": merge-path unless rows or columns are below 500 and the
nonzeros below 10000).  The rule cannot see row-length skew or the hardware it runs on.  This
module keeps a table from *shape classes* to the schedule and launch shape that measured
fastest for that class (``lb_tune`` in the library times every candidate on the device); a
matrix of a class already in the table gets the recorded winner, any other matrix gets the
dissertation's rule (``"auto"``).

A shape class is computed on the host from the row lengths:

* ``size``: log2 of the work items m + nnz (rounded down);
* ``mean``: log2 of the mean row length nnz / m, in half-octave steps;
* ``skew``: the longest row over the mean row length, bucketed to 1, 4, 32, 256 and above;
* ``lrb``: the logarithmic radix bin (Ch.3 Sec. "Binning and Reordering") of row lengths that
  holds the most nonzeros;
* ``dtype``: the value type.

Without a table entry, ``choose_by_roofline`` picks the schedule family that a roofline model
of the measured ceilings (``lbspmv.calibrate``) predicts fastest.

Batches are classed by the batch count and total work (log2), and the dominant member class.
The table is a plain dict that round-trips through JSON (``save`` / ``load``).

``build_table`` tunes the standard synthetic workloads (FP32, BF16 and FP16 values, and the
batch of 4096 matrices); ``python -m paper_2212_08964_gb300.autotune --out PATH`` runs it on the current
GPU.  The package ships the table measured on a GB300 (``default_table``).
"""
from __future__ import annotations

import ctypes
import json
import math
import os

import numpy as np

from . import lbspmv

__all__ = ["shape_class", "lrb_bins", "batch_class", "Table", "tune", "tune_batched", "choose", "plan_for", "batched_plan_for", "predict",
           "choose_by_roofline", "build_table", "default_table", "DEFAULT_TABLE", "STANDARD_WORKLOADS"]

_SKEW_EDGES = (1.5, 4.0, 32.0, 256.0)
# Loaded latency of one dependent gather, for the critical path of row-per-thread schedules.
_GATHER_LATENCY_S = 1.0e-6
_DTYPE_NAMES = {0: "f32", 1: "bf16", 2: "f16"}


def _row_lengths(row_offsets) -> np.ndarray:
    ro = np.asarray(row_offsets, dtype=np.int64)
    return np.diff(ro)


def lrb_bins(row_offsets) -> np.ndarray:
    """Logarithmic radix binning of the rows (Ch.3 Sec. "Binning and Reordering"): the share
    of the nonzeros held by rows of length in [2^b, 2^(b+1)), for b = 0..31 (empty rows hold
    none)."""
    lengths = _row_lengths(row_offsets)
    nz = lengths[lengths > 0]
    out = np.zeros(32)
    if nz.size:
        b = np.floor(np.log2(nz)).astype(np.int64)
        np.add.at(out, b, nz.astype(np.float64))
        out /= out.sum()
    return out


def shape_class(row_offsets, dtype: str = "f32") -> str:
    """Class key of a CSR matrix from its (host) row offsets: work size, mean row length, skew,
    the LRB bin holding the most nonzeros, and the value type."""
    lengths = _row_lengths(row_offsets)
    m = int(lengths.shape[0])
    nnz = int(lengths.sum()) if m else 0
    size = int(math.floor(math.log2(m + nnz))) if m + nnz > 0 else 0
    mean = nnz / m if m else 0.0
    mean_b = int(math.floor(2.0 * math.log2(mean))) if mean > 0 else -99
    skew = (float(lengths.max()) / mean) if mean > 0 else 0.0
    skew_b = sum(1 for e in _SKEW_EDGES if skew >= e)
    lrb = int(np.argmax(lrb_bins(row_offsets))) if nnz else -1
    return f"size{size}-mean{mean_b}-skew{skew_b}-lrb{lrb}-{dtype}"


def predict(row_offsets, n: int, calibration: dict, value_bytes: int = 4) -> dict:
    """Roofline estimate of the SpMV time of each schedule family from the measured ceilings
    (``lbspmv.calibrate()``), in seconds.

    - Streamed bytes: values and column indices per nonzero, offsets and y per row.
    - Work-oriented schedules (merge path, nonzero splitting) are bound by the larger of the
      sector requests (one per random gather plus the streamed bytes / 32) at the measured
      gather rate, and the streamed bytes at the measured read bandwidth.  Nonzero splitting
      also clears y.
    - Row-per-thread and row-per-warp schedules pay the same, or the critical path of their
      longest row of dependent gathers (per thread, or per lane of a warp), whichever is longer.
    """
    lengths = _row_lengths(row_offsets)
    m = int(lengths.shape[0])
    nnz = int(lengths.sum()) if m else 0
    streamed = nnz * (value_bytes + 4) + 8 * m + 4
    rate = float(calibration["gathers_per_s"])
    bw = float(calibration["read_GBps"]) * 1e9
    balanced = max((nnz + streamed / 32.0) / rate, streamed / bw)
    longest = int(lengths.max()) if m else 0
    return {
        "merge_path": balanced,
        "nonzero_split": balanced + 4.0 * m / bw,
        "thread_mapped": max(balanced, longest * _GATHER_LATENCY_S),
        "warp_mapped": max(balanced, math.ceil(longest / 32) * _GATHER_LATENCY_S),
    }


def choose_by_roofline(row_offsets, n: int, calibration: dict, value_bytes: int = 4) -> str:
    """The schedule family with the smallest ``predict`` time (ties go to merge path)."""
    t = predict(row_offsets, n, calibration, value_bytes)
    return min(t, key=lambda k: (t[k], k != "merge_path"))


def batch_class(ms, nnzs, row_offsets_concat, dtype: str = "f32") -> str:
    """Class key of a batch: count and total work (log2), and the class of the member holding
    the most work."""
    ms = np.asarray(ms, np.int64)
    nnzs = np.asarray(nnzs, np.int64)
    count = int(ms.shape[0])
    work = ms + nnzs
    total = int(work.sum())
    big = int(np.argmax(work)) if count else 0
    start = int((ms[:big] + 1).sum())
    member = shape_class(np.asarray(row_offsets_concat)[start: start + int(ms[big]) + 1], dtype) if count else "none"
    c = int(math.floor(math.log2(count))) if count else 0
    t = int(math.floor(math.log2(total))) if total else 0
    return f"batch{c}-work{t}-[{member}]"


class Table:
    """Shape class -> winning configuration, with the measured candidates."""

    def __init__(self, entries: dict | None = None):
        self.entries: dict[str, dict] = dict(entries or {})

    def record(self, key: str, results: list[dict]):
        if not results:
            raise ValueError("no tuning results to record")
        best = min(results, key=lambda r: r["ms"])
        self.entries[key] = {"best": {k: best[k] for k in ("schedule", "threads", "items_per_thread", "group_size")},
                             "ms": best["ms"], "candidates": results}

    def lookup(self, key: str) -> dict | None:
        e = self.entries.get(key)
        return dict(e["best"]) if e else None

    def save(self, path: str):
        tmp = path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(self.entries, f, indent=1, sort_keys=True)
        os.replace(tmp, path)

    @classmethod
    def load(cls, path: str) -> "Table":
        with open(path) as f:
            return cls(json.load(f))


def _results(buf, count: int) -> list[dict]:
    names = {v: k for k, v in lbspmv.SCHEDULES.items()}
    out = []
    for i in range(count):
        r = buf[i]
        out.append({"schedule": names[r.schedule], "threads": r.tuning.threads,
                    "items_per_thread": r.tuning.items_per_thread, "group_size": r.tuning.group_size,
                    "ms": float(r.ms)})
    return out


def tune(row_offsets, col_idx, values, x, n: int | None = None, reps: int = 20, table: Table | None = None,
         stream=None) -> list[dict]:
    """Time every schedule and launch shape on this matrix (device tensors); returns the
    candidates fastest first and, with ``table``, records the winner for the matrix's class."""
    import torch

    lib = lbspmv.ensure_loaded()
    m = row_offsets.numel() - 1
    nnz = col_idx.numel()
    n = x.numel() if n is None else int(n)
    y = torch.empty(m, dtype=torch.float32, device=x.device)
    cap = int(lib.lb_tune_candidates())
    buf = (lbspmv.TuneResult * cap)()
    cnt = ctypes.c_int()
    lbspmv._check(lib.lb_tune(m, n, nnz, row_offsets.data_ptr(), col_idx.data_ptr(), values.data_ptr(),
                              lbspmv._vdt(values), x.data_ptr(), y.data_ptr(), int(reps), buf, cap, ctypes.byref(cnt),
                              lbspmv._stream(stream)), "lb_tune")
    res = _results(buf, cnt.value)
    if table is not None:
        dt = _DTYPE_NAMES[lbspmv._vdt(values)]
        table.record(shape_class(row_offsets.cpu().numpy(), dt), res)
    return res


def tune_batched(ms, ns, nnzs, row_offsets_concat, col_idx_concat, values_concat, x_concat, reps: int = 10,
                 table: Table | None = None, stream=None) -> list[dict]:
    """Time the batch schedules on this batch (thread-mapped rows, and the global merge path at
    every launch shape); with ``table``, record the winner for the batch's class."""
    import torch

    lib = lbspmv.ensure_loaded()
    ms32 = np.ascontiguousarray(ms, np.int32)
    ns32 = np.ascontiguousarray(ns, np.int32)
    nz32 = np.ascontiguousarray(nnzs, np.int32)
    y = torch.empty(int(ms32.astype(np.int64).sum()), dtype=torch.float32, device=x_concat.device)
    cap = int(lib.lb_tune_candidates())
    buf = (lbspmv.TuneResult * cap)()
    cnt = ctypes.c_int()
    lbspmv._check(lib.lb_tune_batched(int(ms32.shape[0]), ms32.ctypes.data, ns32.ctypes.data, nz32.ctypes.data,
                                      row_offsets_concat.data_ptr(), col_idx_concat.data_ptr(),
                                      values_concat.data_ptr(), lbspmv._vdt(values_concat), x_concat.data_ptr(),
                                      y.data_ptr(), int(reps), buf, cap, ctypes.byref(cnt), lbspmv._stream(stream)),
                  "lb_tune_batched")
    res = _results(buf, cnt.value)
    if table is not None:
        dt = _DTYPE_NAMES[lbspmv._vdt(values_concat)]
        table.record(batch_class(ms, nnzs, row_offsets_concat.cpu().numpy(), dt), res)
    return res


# The table measured on a GB300 (sm_103a) by ``build_table`` over ``STANDARD_WORKLOADS``.
DEFAULT_TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tables", "gb300_sm103.json")
STANDARD_WORKLOADS = ("powerlaw_4k", "powerlaw_4m", "stencil7_160", "lognormal_1m", "powerlaw_8m")


def default_table() -> Table | None:
    """The shipped GB300 table, or None when it is absent."""
    return Table.load(DEFAULT_TABLE) if os.path.exists(DEFAULT_TABLE) else None


def build_table(workloads=STANDARD_WORKLOADS, dtypes=("f32", "bf16", "f16"), batched=("batched_4096", "batched_grid_1024"), reps: int = 10,
                table: Table | None = None, log=None) -> Table:
    """Tune every workload in every value type (and every batch) on the current GPU and
    record the winners by shape class."""
    import torch

    from . import synth

    table = Table() if table is None else table
    torch_dt = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}
    for name in workloads:
        a = synth.workload(name)
        x = torch.from_numpy(synth.uniform_pm1(np.random.default_rng(0), a.n)).cuda()
        ro, ci = torch.from_numpy(a.row_offsets).cuda(), torch.from_numpy(a.col_idx).cuda()
        for dt in dtypes:
            v = torch.from_numpy(a.values).cuda().to(torch_dt[dt])
            res = tune(ro, ci, v, x, a.n, reps=reps, table=table)
            if log:
                log(f"{name} {dt}: {res[0]['schedule']} ({res[0]['threads']}, {res[0]['items_per_thread']}, "
                    f"{res[0]['group_size']}) {res[0]['ms'] * 1e3:.1f} us")
        del ro, ci, v, x, a
    for name in batched:
        b = synth.workload(name)
        xs = torch.from_numpy(synth.uniform_pm1(np.random.default_rng(0), int(b.ns.sum()))).cuda()
        res = tune_batched(b.ms, b.ns, b.nnzs, torch.from_numpy(b.row_offsets).cuda(),
                           torch.from_numpy(b.col_idx).cuda(), torch.from_numpy(b.values).cuda(), xs, reps=reps,
                           table=table)
        if log:
            log(f"{name}: {res[0]['schedule']} ({res[0]['threads']}, {res[0]['items_per_thread']}) "
                f"{res[0]['ms'] * 1e3:.1f} us")
    return table


def choose(row_offsets, table: Table | None, dtype: str = "f32") -> dict:
    """The configuration for a matrix: the table's winner for its class, else the
    dissertation's size rule (schedule "auto")."""
    best = table.lookup(shape_class(row_offsets, dtype)) if table is not None else None
    return best if best is not None else {"schedule": "auto", "threads": 0, "items_per_thread": 0, "group_size": 0}


def plan_for(row_offsets, n: int, table: Table | None, dtype: str = "f32", stream=None) -> "lbspmv.Plan":
    """A Plan built with ``choose``'s configuration (row_offsets: int32 device tensor)."""
    cfg = choose(row_offsets.cpu().numpy(), table, dtype)
    return lbspmv.Plan(row_offsets, n, schedule=cfg["schedule"], threads=cfg["threads"],
                       items_per_thread=cfg["items_per_thread"], group_size=cfg["group_size"], stream=stream)


def batched_plan_for(ms, ns, nnzs, row_offsets_concat, table: Table | None, dtype: str = "f32",
                     stream=None) -> "lbspmv.BatchedPlan":
    """A BatchedPlan with the table's schedule and shape for the batch's class (the global
    merge path at the default shape when the class is not in the table)."""
    best = table.lookup(batch_class(ms, nnzs, row_offsets_concat.cpu().numpy(), dtype)) if table is not None else None
    if best is None or best["schedule"] not in ("merge_path", "thread_mapped"):
        best = {"schedule": "merge_path", "threads": 0, "items_per_thread": 0}
    return lbspmv.BatchedPlan(ms, ns, nnzs, row_offsets_concat, threads=best["threads"],
                              items_per_thread=best["items_per_thread"], schedule=best["schedule"], stream=stream)


if __name__ == "__main__":
    import argparse

    p = argparse.ArgumentParser(description="Tune the standard workloads on this GPU and write the table.")
    p.add_argument("--out", default=DEFAULT_TABLE)
    p.add_argument("--reps", type=int, default=10)
    args = p.parse_args()
    os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
    t = build_table(reps=args.reps, log=lambda msg: print(msg, flush=True))
    t.save(args.out)
    print(f"wrote {len(t.entries)} classes to {args.out}")
