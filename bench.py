#!/usr/bin/env python
"""Benchmark: load-balanced CSR SpMV forward + backward on GB300.

One step is one training pass of y = A x (as the autograd function runs it) over the large
power-law matrix (m = n = 4,194,304, ~64M nonzeros, Pareto row lengths with exponent 1.3,
rows up to 500k), with the plan (merge-path partition, CSC view) built once per structure:

  forward   y  = A x      lb_spmv_planned_save: persistent merge-path SpMV + carry fixup, also
                          saving x[col] of every nonzero for the values gradient
  backward  dv = g . x    lb_spmv_backward: one CSR-order pass over the forward partition forms
            dx = A^T g    dvalues and the scaled values v * g[row] in L2-sized buckets of CSC
                          order; a merge-path gather-sum over the CSC view + fixup forms dx

The partition alone and the one-shot lb_spmv (partition + SpMV + fixup every call) are timed
separately and reported under config.components_us.

``value`` is whole-job algorithmic GB/s: bytes = nnz*(value+index) + offsets + x + y for each
of the three passes (counting every dense vector once), divided by the device time of the
timed steps, summed over ranks.  ``--impl reference`` times the FP64 CPU oracle on the same
workload instead (this project's reference arm).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
       (N > 1 under torchrun: independent replicas, one per GPU, weak scaling)
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CSR SpMV GB/s as % of GB300 HBM peak; fwd+bwd and batched vs plain"
UNIT = "GB/s"
WORKLOAD = "powerlaw_4m"
FALLBACK_HBM_GBS = 6800.0
NOMINAL_HBM_GBS = 8000.0  # GB300 HBM3e, nominal


def parse_args(argv=None):
    p = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=1000)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", default=WORKLOAD)
    p.add_argument("--scale", type=float, default=1.0,
                   help="shrink the workload's m, n and nnz together (small cases for profiler captures)")
    p.add_argument("--no-cpu-baseline", action="store_true", help="skip the oracle timing leg")
    p.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    p.add_argument("--no-secondary", action="store_true",
                   help="skip the secondary lines (BF16/FP16 step, batched vs per-matrix)")
    p.add_argument("--spmm-only", action="store_true",
                   help="time only SpMM on the workload and print its line (small cases for profiler captures)")
    p.add_argument("--batched-only", action="store_true",
                   help="time only the two batch classes and print their line (for profiler captures)")
    return p.parse_args(argv)


# ------------------------------------------------------------------------------------------
# Algorithmic bytes (the method's minimum traffic; every dense vector counted once).


def spmv_bytes(m: int, n: int, nnz: int, value_bytes: int = 4) -> int:
    return nnz * (value_bytes + 4) + 4 * (m + 1) + 4 * n + 4 * m


def dvalues_bytes(m: int, n: int, nnz: int) -> int:
    # reads col_idx and writes dvalues per nonzero; reads offsets, g and x once.
    return nnz * (4 + 4) + 4 * (m + 1) + 4 * m + 4 * n


def step_bytes(m, n, nnz, value_bytes=4):
    fwd = spmv_bytes(m, n, nnz, value_bytes)
    bwd_t = spmv_bytes(n, m, nnz, value_bytes)
    dv = dvalues_bytes(m, n, nnz)
    return fwd, bwd_t, dv


def measured_hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash(files=("lb_merge.cuh", "lb_warp.cuh", "lb_internal.cuh")) -> str:
    """Hash of a kernel's source files with comments and blank space removed, so a recorded
    DRAM-traffic figure is used only while the code it was measured on is unchanged."""
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2212_08964_gb300", "csrc", f)) as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def recorded_traffic(workload: str, kernel: str):
    """DRAM bytes per launch of `kernel` from a committed ncu summary, if the kernel's source
    files have not changed since it was captured; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        e = d.get(workload, {}).get(kernel)
        if e and e.get("kernel_source_hash") == kernel_source_hash(tuple(e["sources"])):
            return float(e["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


# ------------------------------------------------------------------------------------------
# Clocks during the timed region.


class ClockSampler:
    """nvidia-smi samples (every 20 ms, timestamped) around the timed region.

    The sampler starts before the timed region and the region begins only after its first
    sample has arrived, so nvidia-smi's start-up does not eat the region.  `mark_start` and
    `mark_end` bracket the timed steps; `hold(step)` keeps running the same step, untimed, for
    `hold_s` seconds afterwards, so that a timed region shorter than a few sampling periods
    still has clocks recorded under the same load.  The summary reports the samples inside the
    timed region and those of the whole loaded window (region + hold) separately; `sm_mhz` and
    `reasons` come from the region when it holds at least three samples, else from the window,
    and `basis` says which.
    """

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    PERIOD_MS = 20

    def __init__(self, gpu_index: int, hold_s: float = 0.3):
        self.gpu = gpu_index
        self.proc = None
        self.path = None
        self.hold_s = hold_s
        self.t_start = self.t_end = self.t_hold = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", str(self.PERIOD_MS)], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            deadline = time.time() + 5.0  # wait (bounded) for the first sample
            while time.time() < deadline and self.proc.poll() is None:
                if os.path.getsize(self.path) > 0:
                    break
                time.sleep(0.01)
        except Exception:
            self.proc = None
        return self

    def mark_start(self):
        self.t_start = time.time()

    def mark_end(self):
        self.t_end = time.time()

    def hold(self, step, sync):
        """Run `step` (untimed) for hold_s seconds under the sampler."""
        if self.proc is None:
            return
        t = time.time()
        while time.time() - t < self.hold_s:
            for _ in range(8):
                step()
            sync()
        self.t_hold = time.time()

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    @staticmethod
    def _stamp(text):
        import datetime

        try:
            return datetime.datetime.strptime(text.strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            return None

    def summary(self):
        if self.proc is None or not self.path:
            return None
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 10:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        half = self.PERIOD_MS / 2000.0

        def pick(t0, t1):
            if t0 is None or t1 is None:
                return []
            return [r for r in rows if (ts := self._stamp(r[0])) is not None and t0 - half <= ts <= t1 + half]

        def stats(sel):
            sm = [float(r[2]) for r in sel if r[2].replace(".", "").isdigit()]
            smax = [float(r[3]) for r in sel if r[3].replace(".", "").isdigit()]
            reasons = sorted({names[i] for r in sel for i in range(4) if r[6 + i].lower() == "active"})
            return (float(np.median(sm)) if sm else None, max(smax) if smax else None, reasons, len(sel))

        region = pick(self.t_start, self.t_end)
        window = pick(self.t_start, self.t_hold if self.t_hold is not None else self.t_end)
        basis, sel = ("timed region", region) if len(region) >= 3 else ("timed region + untimed hold of the same step",
                                                                          window)
        sm, smax, reasons, n = stats(sel)
        w_sm, _, w_reasons, w_n = stats(window)
        all_reasons = sorted(set(reasons) | set(w_reasons))
        return {"sm_mhz": sm, "sm_max_mhz": smax, "reasons": all_reasons, "samples": len(region),
                "window_samples": w_n, "window_sm_mhz": w_sm, "basis": basis,
                "period_ms": self.PERIOD_MS, "hold_s": self.hold_s}


# ------------------------------------------------------------------------------------------
# Distributed plumbing (one process per GPU; replicas, no data-path collective).


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        backend = "nccl" if _cuda_ok() else "gloo"
        dist.init_process_group(backend)
    return rank, world, local


def _cuda_ok():
    try:
        import torch

        return torch.cuda.is_available()
    except Exception:
        return False


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(value: float, world: int) -> float:
    if world == 1:
        return value
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------------------------------
# CPU oracle timing (the baseline leg and the reference arm).


def oracle_step_time(a, x64, g64, v64, threads=0, budget_s=12.0, max_steps=None):
    """Mean seconds of one oracle fwd + bwd step (oracle as it stands) over a bounded run."""
    import oracle

    oracle.build()
    times = []
    t_start = time.perf_counter()
    while True:
        t0 = time.perf_counter()
        oracle.spmv(a.row_offsets, a.col_idx, v64, x64, threads)
        oracle.spmv_t(a.row_offsets, a.col_idx, v64, g64, a.n, threads)
        oracle.dvalues(a.row_offsets, a.col_idx, g64, x64, threads)
        times.append(time.perf_counter() - t0)
        if max_steps is not None and len(times) >= max_steps:
            break
        if max_steps is None and time.perf_counter() - t_start > budget_s:
            break
    return float(np.mean(times)), len(times)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


# ------------------------------------------------------------------------------------------


def make_inputs(workload: str, scale: float = 1.0):
    from paper_2212_08964_gb300 import synth

    a = synth.workload(workload, scale)
    rng = np.random.default_rng(1234)
    x = synth.uniform_pm1(rng, a.n)
    g = synth.uniform_pm1(rng, a.m)
    return a, x, g


def row_sample(a, m_s: int):
    """The leading m_s rows of a CSR matrix (all columns)."""
    from paper_2212_08964_gb300 import synth

    m_s = max(1, min(a.m, m_s))
    nz = int(a.row_offsets[m_s])
    return synth.CSR(m_s, a.n, a.row_offsets[: m_s + 1].copy(), a.col_idx[:nz], a.values[:nz])


def run_reference(args, budget_s: float = 150.0):
    rank, world, _ = dist_setup(args)
    if rank != 0:
        return 0
    a, x, g = make_inputs(args.workload, args.scale)
    import oracle

    cores = oracle.max_threads()
    x64, g64 = x.astype(np.float64), g.astype(np.float64)
    t_full, _ = oracle_step_time(a, x64, g64, a.values.astype(np.float64), max_steps=1)
    K, W = max(args.steps, 1), max(args.warmup, 0)
    per_step = budget_s / (K + W)
    if t_full <= per_step:
        s, sample = a, f"full {args.workload} fwd+bwd per step"
    else:
        s = row_sample(a, int(a.m * per_step / t_full))
        sample = f"leading {s.m} of {a.m} rows ({s.nnz} nonzeros) of {args.workload}, fwd+bwd per step"
    v64 = s.values.astype(np.float64)
    if W:
        oracle_step_time(s, x64, g64[: s.m], v64, max_steps=W)
    sec, steps = oracle_step_time(s, x64, g64[: s.m], v64, max_steps=K)
    fwd, bwd, dv = step_bytes(s.m, s.n, s.nnz)
    value = (fwd + bwd + dv) / sec / 1e9
    line = {
        "impl": "reference",
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": steps, "warmup": W,
        "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded power-law CSR)",
        "config": {"workload": f"{workload_name(args)} fwd+bwd", "m": a.m, "n": a.n, "nnz": a.nnz},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def workload_name(args) -> str:
    return args.workload if args.scale == 1.0 else f"{args.workload} scaled by {args.scale:g}"


def run_ours(args):
    import torch

    from paper_2212_08964_gb300 import lbspmv as lb

    rank, world, local = dist_setup(args)
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (the CUDA library is the only compute path)")
    torch.cuda.set_device(local)
    lb.ensure_loaded()
    if args.batched_only:
        if rank == 0:
            print(json.dumps({"batched": run_batched(lb, torch, torch.device("cuda", local))}))
        return 0
    a, x, g = make_inputs(args.workload, args.scale)
    dev = torch.device("cuda", local)
    ro = torch.from_numpy(a.row_offsets).to(dev)
    ci = torch.from_numpy(a.col_idx).to(dev)
    v = torch.from_numpy(a.values).to(dev)
    xd = torch.from_numpy(x).to(dev)
    gd = torch.from_numpy(g).to(dev)
    y = torch.empty(a.m, device=dev)
    dx = torch.empty(a.n, device=dev)
    dv = torch.empty(a.nnz, device=dev)
    xg = torch.empty(a.nnz, device=dev)
    plan = lb.Plan(ro, a.n, a.nnz, schedule="merge_path")
    if args.spmm_only:
        if rank == 0:
            print(json.dumps({"workload": args.workload, "scale": args.scale, "nnz": int(a.nnz),
                              "spmm": run_spmm(lb, torch, dev, a, plan, ci, v, xd, y)}))
        return 0
    plan.build_transpose(ci)
    info = plan.info()
    torch.cuda.synchronize()

    # The values gradient in the values' type, as the autograd function stores it.
    dv_of = {torch.float32: dv, torch.bfloat16: torch.empty(a.nnz, dtype=torch.bfloat16, device=dev),
             torch.float16: torch.empty(a.nnz, dtype=torch.float16, device=dev)}

    def step(vals, xx, gg):
        # The training step of y = A x under autograd: forward (saving x[col] per nonzero for
        # the values gradient), then dx = A^T g and dvalues = g[row] * x[col] together.
        plan.spmv(ci, vals, xx, out=y, save_gathered=xg)
        plan.backward(vals, gg, xg, dx=dx, dvalues=dv_of[vals.dtype])

    launches_per_step = 2 + 3
    fwd_b, bwd_t_b, dv_b = step_bytes(a.m, a.n, a.nnz)
    total_b = fwd_b + bwd_t_b + dv_b

    for _ in range(max(args.warmup, 3)):
        step(v, xd, gd)
    K = max(args.steps, 1)
    mk = lambda: [torch.cuda.Event(enable_timing=True) for _ in range(K)]  # noqa: E731
    evf_b, evf_a, evt_b, evt_a, evd_b, evd_a = mk(), mk(), mk(), mk(), mk(), mk()
    for e in evf_b + evf_a + evt_b + evt_a + evd_b + evd_a:  # create the events before the timed region
        e.record()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        clocks.mark_start()
        t0.record()
        for i in range(K):
            # The same step, with events around each pass's main kernel (recorded by the library
            # on the launching stream for the merge-path kernels).
            lb.set_profile_events(evf_b[i], evf_a[i])
            plan.spmv(ci, v, xd, out=y, save_gathered=xg)
            evd_b[i].record()  # the CSR-order backward pass runs first in lb_spmv_backward
            lb.set_profile_events(evt_b[i], evt_a[i])
            plan.backward(v, gd, xg, dx=dx, dvalues=dv)
            lb.set_profile_events(None, None)
        t1.record()
        torch.cuda.synchronize()
        clocks.mark_end()
        lb.set_profile_events(None, None)
        clocks.hold(lambda: step(v, xd, gd), torch.cuda.synchronize)
    lb.set_profile_events(None, None)
    barrier(world)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / K
    ms_max = max_over_ranks(ms, world)
    mean_ms = lambda b, e: float(np.mean([x.elapsed_time(y_) for x, y_ in zip(b, e)]))  # noqa: E731
    # Backward bytes: the CSR-order pass reads values, saved gathers and row offsets and writes
    # dvalues and the scaled values; the gather-sum streams CSC offsets and positions, gathers
    # the scaled values and writes dx.  Both counted at their minimum (every array once).
    vb = 4
    csr_b = a.nnz * (vb + 4 + 4 + 4) + 4 * (a.m + 1) + 4 * a.m
    gs_b = a.nnz * (4 + 4) + 4 * (a.n + 1) + 4 * a.n
    # Per kernel: mean time, algorithmic bytes (the hot-path step's minimum: each array once),
    # the bytes it moves beyond them (the forward's saved gathers, the CSR-order pass's bucket
    # positions: plan or step data that the minimum leaves out), and its random gathers.
    kern = {
        "merge_spmv_kernel<plain> (y = A x, saving x[col])": (mean_ms(evf_b, evf_a), fwd_b),
        "csr_backward_kernel (dvalues, v*g[row] into CSC buckets)": (mean_ms(evd_b, evt_b), csr_b),
        "merge_spmv_kernel<gather-sum> (dx = A^T g)": (mean_ms(evt_b, evt_a), gs_b),
    }
    extra = {
        "merge_spmv_kernel<plain> (y = A x, saving x[col])": 4 * a.nnz,
        # more than one 2^23-entry bucket: the pass reads a bucket position per nonzero
        "csr_backward_kernel (dvalues, v*g[row] into CSC buckets)": 4 * a.nnz if a.nnz > (1 << 23) else 0,
        "merge_spmv_kernel<gather-sum> (dx = A^T g)": 0,
    }
    gathers = {
        "merge_spmv_kernel<plain> (y = A x, saving x[col])": a.nnz,
        "csr_backward_kernel (dvalues, v*g[row] into CSC buckets)": 0,
        "merge_spmv_kernel<gather-sum> (dx = A^T g)": a.nnz,
    }
    assert lb.device_error() == 0

    peak, peak_kind = measured_hbm_peak()
    calib = lb.calibrate() if rank == 0 else None
    kernels = {}
    for k, (t, b) in kern.items():
        kernels[k] = {"avg_launch_ms": t, "algorithmic_bytes_per_launch": b, "extra_bytes_per_launch": extra[k],
                      "achieved_GBps": b / (t * 1e-3) / 1e9, "frac": b / (t * 1e-3) / 1e9 / peak,
                      "random_gathers_per_launch": gathers[k], "gathers_per_s": gathers[k] / (t * 1e-3)}
        if calib and gathers[k]:
            kernels[k]["frac_of_gather_ceiling"] = kernels[k]["gathers_per_s"] / calib["gathers_per_s"]
    dom = max(kern, key=lambda k: kern[k][0])
    dom_ms, dom_b = kern[dom]
    achieved = dom_b / (dom_ms * 1e-3) / 1e9
    value = total_b * world / (ms_max * 1e-3) / 1e9

    # Components outside the timed step: the partition (once per structure in a plan) and the
    # one-shot lb_spmv, which recomputes the partition on every call.
    merge_tiles, merge_items = plan.tiles("merge")
    part_tr = torch.empty(merge_tiles + 1, dtype=torch.int32, device=dev)
    part_tn = torch.empty_like(part_tr)
    comp = {
        "partition_us": 1e3 * _time(torch, lambda: lb._lib.lb_partition(a.m, a.nnz, ro.data_ptr(), merge_items,
                                                                         part_tr.data_ptr(), part_tn.data_ptr(),
                                                                         torch.cuda.current_stream().cuda_stream), 20),
        "forward_oneshot_lb_spmv_us": 1e3 * _time(torch, lambda: lb.spmv(ro, ci, v, xd, out=y), 20),
        "forward_planned_us": 1e3 * _time(torch, lambda: plan.spmv(ci, v, xd, out=y), 20),
        "dvalues_gathering_x_us": 1e3 * _time(torch, lambda: plan.dvalues(ci, gd, xd, out=dv), 20),
        "spmv_t_us": 1e3 * _time(torch, lambda: plan.spmv_t(v, gd, out=dx), 20),
    }

    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": max(args.warmup, 3),
        "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded power-law CSR, uniform[-1,1] values, x and g)",
        "config": {
            "workload": f"{workload_name(args)} fwd+bwd", "m": a.m, "n": a.n, "nnz": a.nnz,
            "schedule": info["schedule"], "threads": info["threads"], "items_per_thread": info["items_per_thread"],
            "num_tiles": info["num_tiles"], "parallelism": f"replicas x{world}",
            "step": "plan built once per structure (partition, CSC view); per step: forward saving x[col], "
                    "then dvalues and dx = A^T g (CSR-order pass + merge-path gather-sum over the CSC view)",
            "l2": f"no flush: each step streams {total_b / 1e9:.2f} GB of inputs, above the 129 MB L2",
            "bytes_per_step": {"forward": fwd_b, "backward_dx": bwd_t_b, "backward_dvalues": dv_b},
            "components_us": comp,
        },
        "roofline": {
            "bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_kind": peak_kind, "traffic": recorded_traffic(args.workload, dom) if args.scale == 1.0 else None,
            "algorithmic_bytes_per_launch": dom_b, "extra_bytes_per_launch": extra[dom], "avg_launch_ms": dom_ms,
            "frac_of_nominal_8000": achieved / NOMINAL_HBM_GBS,
        },
        "kernels": kernels,
        "calibration": calib,
        "roofline_gathers": None if not calib else {
            "bound": "random 4-byte gathers (one 32-byte L1-to-L2 sector request each)",
            "kernels": {k: {"gathers_per_s": kernels[k]["gathers_per_s"],
                            "frac": kernels[k]["gathers_per_s"] / calib["gathers_per_s"]}
                        for k in kernels if gathers[k]},
            "peak": calib["gathers_per_s"], "unit": "gathers/s",
            "peak_kind": "measured by lb_calibrate in this run (random 4-byte gathers from a 16 MB vector)"},
        "gpu_launches": launches_per_step * K,
        "clocks": clocks.summary(),
    }
    result["roofline"]["frac_of"] = f"of {peak_kind}"

    # End to end through the public API with host buffers: per step, H2D of the values, x and
    # g from pinned memory, the step, then the D2H read of y, dx and dvalues.  Steps run as a
    # two-slot pipeline on three streams: step i's inputs arrive while step i - 1 computes and
    # step i - 2's results go back, so the two link directions and the kernels overlap.  Every
    # step's copies are inside the timed region; a serial run (one stream) is timed beside it.
    if not args.no_e2e:
        h_v = torch.from_numpy(a.values).pin_memory()
        h_x = torch.from_numpy(x).pin_memory()
        h_g = torch.from_numpy(g).pin_memory()
        slots = []
        for _ in range(2):
            slots.append({
                "v": torch.empty_like(v), "x": torch.empty_like(xd), "g": torch.empty_like(gd),
                "y": torch.empty_like(y), "dx": torch.empty_like(dx), "dv": torch.empty_like(dv),
                "oy": torch.empty(a.m, pin_memory=True), "odx": torch.empty(a.n, pin_memory=True),
                "odv": torch.empty(a.nnz, pin_memory=True),
                "in_ready": torch.cuda.Event(), "in_free": torch.cuda.Event(),
                "out_ready": torch.cuda.Event(), "out_free": torch.cuda.Event()})
        cs = torch.cuda.current_stream()
        h2d_s, d2h_s = torch.cuda.Stream(), torch.cuda.Stream()

        def e2e_pipelined(steps):
            for sl in slots:  # every slot starts free
                sl["in_free"].record(cs)
                sl["out_free"].record(cs)
            for i in range(steps):
                sl = slots[i % 2]
                with torch.cuda.stream(h2d_s):
                    h2d_s.wait_event(sl["in_free"])
                    sl["v"].copy_(h_v, non_blocking=True)
                    sl["x"].copy_(h_x, non_blocking=True)
                    sl["g"].copy_(h_g, non_blocking=True)
                    sl["in_ready"].record(h2d_s)
                cs.wait_event(sl["in_ready"])
                cs.wait_event(sl["out_free"])
                plan.spmv(ci, sl["v"], sl["x"], out=sl["y"], save_gathered=xg)
                plan.backward(sl["v"], sl["g"], xg, dx=sl["dx"], dvalues=sl["dv"])
                sl["in_free"].record(cs)
                sl["out_ready"].record(cs)
                with torch.cuda.stream(d2h_s):
                    d2h_s.wait_event(sl["out_ready"])
                    sl["oy"].copy_(sl["y"], non_blocking=True)
                    sl["odx"].copy_(sl["dx"], non_blocking=True)
                    sl["odv"].copy_(sl["dv"], non_blocking=True)
                    sl["out_free"].record(d2h_s)
            cs.wait_stream(d2h_s)

        def e2e_serial():
            sl = slots[0]
            sl["v"].copy_(h_v, non_blocking=True)
            sl["x"].copy_(h_x, non_blocking=True)
            sl["g"].copy_(h_g, non_blocking=True)
            plan.spmv(ci, sl["v"], sl["x"], out=sl["y"], save_gathered=xg)
            plan.backward(sl["v"], sl["g"], xg, dx=sl["dx"], dvalues=sl["dv"])
            sl["oy"].copy_(sl["y"], non_blocking=True)
            sl["odx"].copy_(sl["dx"], non_blocking=True)
            sl["odv"].copy_(sl["dv"], non_blocking=True)

        def timed_e2e(run):
            torch.cuda.synchronize()
            barrier(world)
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record(cs)
            run()
            s1.record(cs)
            torch.cuda.synchronize()
            barrier(world)
            return s0.elapsed_time(s1)

        Ke = max(2, min(K, 50))
        e2e_pipelined(2)  # warm-up
        e_ms = max_over_ranks(timed_e2e(lambda: e2e_pipelined(Ke)) / Ke, world)
        # The host copies of the last step's results equal the device results.
        last = slots[(Ke - 1) % 2]
        assert torch.equal(last["oy"], last["y"].cpu()) and torch.equal(last["odv"], last["dv"].cpu())
        e2e_serial()
        serial_ms = max_over_ranks(timed_e2e(lambda: [e2e_serial() for _ in range(Ke)]) / Ke, world)
        h2d = (a.values.nbytes + x.nbytes + g.nbytes)
        d2h = 4 * (a.m + a.n + a.nnz)
        # The link alone: the same copies with no kernels, both directions at once.
        sl = slots[0]

        def link_only():
            with torch.cuda.stream(h2d_s):
                h2d_s.wait_stream(cs)
                sl["v"].copy_(h_v, non_blocking=True)
                sl["x"].copy_(h_x, non_blocking=True)
                sl["g"].copy_(h_g, non_blocking=True)
            with torch.cuda.stream(d2h_s):
                d2h_s.wait_stream(cs)
                sl["oy"].copy_(sl["y"], non_blocking=True)
                sl["odx"].copy_(sl["dx"], non_blocking=True)
                sl["odv"].copy_(sl["dv"], non_blocking=True)
            cs.wait_stream(h2d_s)
            cs.wait_stream(d2h_s)

        link_only()
        link_ms = max_over_ranks(timed_e2e(lambda: [link_only() for _ in range(Ke)]) / Ke, world)
        result["e2e"] = {"value": total_b * world / (e_ms * 1e-3) / 1e9, "unit": UNIT, "h2d_bytes_per_step": h2d,
                         "d2h_bytes_per_step": d2h, "ms_per_step": e_ms, "steps": Ke,
                         "mode": "two-slot pipeline: H2D, compute and D2H on three streams",
                         "serial_one_stream": {"value": total_b * world / (serial_ms * 1e-3) / 1e9,
                                               "ms_per_step": serial_ms},
                         "link_only_ms_per_step": link_ms, "link_GBps": (h2d + d2h) / (link_ms * 1e-3) / 1e9}
        del slots

    if rank == 0 and not args.no_secondary:
        # The same step captured once in a CUDA graph and replayed (no host work per step).
        gs = torch.cuda.Stream()
        gs.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(gs):
            step(v, xd, gd)
        torch.cuda.current_stream().wait_stream(gs)
        torch.cuda.synchronize()
        g_step = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g_step):
            step(v, xd, gd)
        result["graph_step_ms"] = _time(torch, g_step.replay, 50)
        del g_step
        # The metric's second half: BF16/FP16 values against FP32 on this step, and the batched
        # form (one persistent launch in a CUDA graph) against one call per matrix.
        def step_ms(vals):
            return _time(torch, lambda: step(vals, xd, gd), 20)

        f32_ms = step_ms(v)
        mixed = {"f32_step_ms": f32_ms}
        for name, dt, vbytes in (("bf16", torch.bfloat16, 2), ("f16", torch.float16, 2)):
            ms_ = step_ms(v.to(dt))
            mixed[f"{name}_step_ms"] = ms_
            mixed[f"{name}_speedup_vs_f32"] = f32_ms / ms_
        mixed["tuned_" + args.workload] = run_tuned_precision(lb, torch, a, ro, ci, v, xd, gd, y, dx, dv, xg)
        mixed["stencil7_160_forward"] = run_stencil_precision(lb, torch, dev)
        mixed["powerlaw_8m_forward"] = run_c5(lb, torch, dev)
        result["mixed_precision"] = mixed

        # The opt-in backward without a CSC view: dx by float reductions into dx[col] in the
        # CSR-order pass (not bit-reproducible), dvalues as in the step above.
        def scatter_step():
            plan.spmv(ci, v, xd, out=y, save_gathered=xg)
            plan.backward_scatter(ci, v, gd, xg, dx=dx, dvalues=dv)

        sc_ms = _time(torch, scatter_step, 20)
        sc_bwd = _time(torch, lambda: plan.backward_scatter(ci, v, gd, xg, dx=dx, dvalues=dv), 20)
        det_bwd = _time(torch, lambda: plan.backward(v, gd, xg, dx=dx, dvalues=dv), 20)
        result["backward_scatter"] = {
            "step_ms": sc_ms, "step_GBps": total_b / (sc_ms * 1e-3) / 1e9, "speedup_vs_step": f32_ms / sc_ms,
            "backward_ms": sc_bwd, "deterministic_backward_ms": det_bwd,
            "note": "opt-in lb_spmv_backward_scatter: dx by float reductions in L2, not bit-reproducible; "
                    "no CSC view"}
        result["batched"] = run_batched(lb, torch, dev)
        result["differentiable"] = run_differentiable(lb, torch, dev)
        result["small_4k"] = run_small(lb, torch, dev)
        result["spmm"] = run_spmm(lb, torch, dev, a, plan, ci, v, xd, y)
        result["sssp"] = run_sssp(lb, torch, dev, a, ro, ci)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle

        cores = oracle.max_threads()
        sec, steps = oracle_step_time(a, x.astype(np.float64), g.astype(np.float64), a.values.astype(np.float64))
        result["cpu_baseline"] = {"value": total_b / sec / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
                                  "sample": f"{steps} full fwd+bwd steps of {args.workload} (FP64 C oracle, OpenMP)"}
        # The same oracle on one host core, over the leading eighth of the rows (one step).
        s = row_sample(a, a.m // 8)
        sec1, _ = oracle_step_time(s, x.astype(np.float64), g[: s.m].astype(np.float64),
                                   s.values.astype(np.float64), threads=1, max_steps=1)
        b1 = sum(step_bytes(s.m, s.n, s.nnz))
        result["cpu_baseline"]["single_thread"] = {
            "value": b1 / sec1 / 1e9, "unit": UNIT, "cores": 1,
            "sample": f"one fwd+bwd step over the leading {s.m} rows ({s.nnz} nonzeros) of {args.workload}"}
    if rank == 0:
        print(json.dumps(result), flush=True)
    return 0


def _tuned_plan(lb, torch, a, ro, dtype_name):
    """A plan with the shipped GB300 table's configuration for the matrix's class and value
    type (the size rule when the class is not in the table), and that configuration."""
    from paper_2212_08964_gb300 import autotune

    cfg = autotune.choose(a.row_offsets, autotune.default_table(), dtype_name)
    plan = lb.Plan(ro, a.n, a.nnz, schedule=cfg["schedule"], threads=cfg["threads"],
                   items_per_thread=cfg["items_per_thread"], group_size=cfg["group_size"])
    info = plan.info()
    return plan, [info["schedule"], info["threads"], info["items_per_thread"], info["group_size"]]


_DTYPES = (("f32", "float32", 4), ("bf16", "bfloat16", 2), ("f16", "float16", 2))


def run_tuned_precision(lb, torch, a, ro, ci, v, xd, gd, y, dx, dv, xg):
    """The step and the forward with each value type in the autotuned configuration of its
    class (the shipped GB300 table): the shape that wins for narrow values differs."""
    out = {}
    for name, tname, _ in _DTYPES:
        plan, shape = _tuned_plan(lb, torch, a, ro, name)
        plan.build_transpose(ci)
        vd = v.to(getattr(torch, tname))
        dvd = dv if vd.dtype == torch.float32 else torch.empty(a.nnz, dtype=vd.dtype, device=dv.device)

        def step():
            plan.spmv(ci, vd, xd, out=y, save_gathered=xg)
            plan.backward(vd, gd, xg, dx=dx, dvalues=dvd)

        out[name] = {"config": shape, "forward_ms": _time(torch, lambda: plan.spmv(ci, vd, xd, out=y), 20),
                     "forward_save_ms": _time(torch, lambda: plan.spmv(ci, vd, xd, out=y, save_gathered=xg), 20),
                     "backward_ms": _time(torch, lambda: plan.backward(vd, gd, xg, dx=dx, dvalues=dvd), 20),
                     "step_ms": _time(torch, step, 20)}
        del dvd
        del plan
    for name in ("bf16", "f16"):
        out[f"{name}_forward_speedup_vs_f32"] = out["f32"]["forward_ms"] / out[name]["forward_ms"]
        out[f"{name}_step_speedup_vs_f32"] = out["f32"]["step_ms"] / out[name]["step_ms"]
    return out


def run_c5(lb, torch, dev):
    """The mixed-precision configuration: the 8M-row power-law matrix (128M nonzeros), the
    forward with FP32, BF16 and FP16 values, in the default merge-path shape and in each value
    type's autotuned configuration."""
    from paper_2212_08964_gb300 import synth

    out = {}
    a = synth.workload("powerlaw_8m")
    x = torch.from_numpy(synth.uniform_pm1(np.random.default_rng(6), a.n)).to(dev)
    ro, ci = torch.from_numpy(a.row_offsets).to(dev), torch.from_numpy(a.col_idx).to(dev)
    y = torch.empty(a.m, device=dev)
    out["workload"] = f"powerlaw_8m: m = n = {a.m}, nnz = {a.nnz}"
    base = lb.Plan(ro, a.n, a.nnz, schedule="merge_path")
    for name, tname, vb in _DTYPES:
        v = torch.from_numpy(a.values).to(dev).to(getattr(torch, tname))
        ms = _time(torch, lambda: base.spmv(ci, v, x, out=y), 20)
        plan, shape = _tuned_plan(lb, torch, a, ro, name)
        ms_t = _time(torch, lambda: plan.spmv(ci, v, x, out=y), 20)
        byts = spmv_bytes(a.m, a.n, a.nnz, vb)
        out[name] = {"default_ms": ms, "tuned_config": shape, "tuned_ms": ms_t, "tuned_GBps": byts / (ms_t * 1e-3) / 1e9}
        del plan, v
    for name in ("bf16", "f16"):
        out[f"{name}_speedup_vs_f32_tuned"] = out["f32"]["tuned_ms"] / out[name]["tuned_ms"]
        out[f"{name}_speedup_vs_f32_default_shape"] = out["f32"]["default_ms"] / out[name]["default_ms"]
    return out


def run_small(lb, torch, dev):
    """The small configuration (m = n = 4096, about 64k nonzeros), which launch latency bounds:
    one planned forward per schedule, captured 50 times in a CUDA graph and replayed, in
    microseconds per call, with the schedule the size rule picks."""
    from paper_2212_08964_gb300 import synth

    a = synth.workload("powerlaw_4k")
    x = torch.from_numpy(synth.uniform_pm1(np.random.default_rng(1), a.n)).to(dev)
    ro, ci, v = (torch.from_numpy(t).to(dev) for t in (a.row_offsets, a.col_idx, a.values))
    y = torch.empty(a.m, device=dev)
    out = {"workload": f"powerlaw_4k: m = n = {a.m}, nnz = {a.nnz}",
           "rule_choice": lb.Plan(ro, a.n, a.nnz, schedule="auto").info()["schedule"]}
    for sched in ("merge_path", "thread_mapped", "warp_mapped", "block_mapped", "nonzero_split"):
        plan = lb.Plan(ro, a.n, a.nnz, schedule=sched)
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            plan.spmv(ci, v, x, out=y)  # first call outside the capture
        torch.cuda.current_stream().wait_stream(s)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            for _ in range(50):
                plan.spmv(ci, v, x, out=y)
        out[f"{sched}_us"] = 1e3 * _time(torch, graph.replay, 20) / 50
        del graph, plan
    return out


def run_differentiable(lb, torch, dev):
    """The differentiable SpMV on the 1M-row log-normal matrix: the library step (forward saving
    x[col], then dx and dvalues) with g given, and the autograd training step of the loss
    0.5 ||A x - t||^2 (the loss and g = y - t are two small torch ops; the SpMV forward and
    backward are the library's).  Bytes as for the main step."""
    from paper_2212_08964_gb300 import synth

    a = synth.workload("lognormal_1m")
    rng = np.random.default_rng(4)
    x = torch.from_numpy(synth.uniform_pm1(rng, a.n)).to(dev)
    t = torch.from_numpy(synth.uniform_pm1(rng, a.m)).to(dev)
    g = torch.from_numpy(synth.uniform_pm1(rng, a.m)).to(dev)
    ro, ci = torch.from_numpy(a.row_offsets).to(dev), torch.from_numpy(a.col_idx).to(dev)
    v = torch.from_numpy(a.values).to(dev)
    plan = lb.Plan(ro, a.n, a.nnz, schedule="merge_path")
    plan.build_transpose(ci)
    y = torch.empty(a.m, device=dev)
    dx = torch.empty(a.n, device=dev)
    dv = torch.empty(a.nnz, device=dev)
    xg = torch.empty(a.nnz, device=dev)

    def step():
        plan.spmv(ci, v, x, out=y, save_gathered=xg)
        plan.backward(v, g, xg, dx=dx, dvalues=dv)

    vt = v.clone().requires_grad_(True)
    xt = x.clone().requires_grad_(True)

    def train_step():
        vt.grad = None
        xt.grad = None
        yy = lb.spmv_autograd(plan, ci, vt, xt)
        loss = 0.5 * torch.sum((yy - t) ** 2)
        loss.backward()

    fwd_b, bwd_t_b, dv_b = step_bytes(a.m, a.n, a.nnz)
    total = fwd_b + bwd_t_b + dv_b
    ms = _time(torch, step, 50)
    ms_train = _time(torch, train_step, 50)
    return {"workload": f"lognormal_1m: m = n = {a.m}, nnz = {a.nnz}", "bytes_per_step": total,
            "step_ms": ms, "step_GBps": total / (ms * 1e-3) / 1e9,
            "autograd_train_step_ms": ms_train, "autograd_train_step_GBps": total / (ms_train * 1e-3) / 1e9}


def run_stencil_precision(lb, torch, dev):
    """The balanced contrast: the 7-point stencil on a 160^3 grid (4.1M rows, 28.5M nonzeros),
    whose gathers hit neighbouring sectors, so the pass is bound by streaming the matrix and
    narrower values pay off.  Forward with FP32, BF16 and FP16 values, thread-mapped (the
    schedule the autotuner picks for this class) and merge-path."""
    from paper_2212_08964_gb300 import synth

    a = synth.workload("stencil7_160")
    x = torch.from_numpy(synth.uniform_pm1(np.random.default_rng(3), a.n)).to(dev)
    ro, ci = torch.from_numpy(a.row_offsets).to(dev), torch.from_numpy(a.col_idx).to(dev)
    y = torch.empty(a.m, device=dev)
    out = {"workload": f"stencil7_160: m = n = {a.m}, nnz = {a.nnz}"}
    for sched in ("thread_mapped", "merge_path"):
        plan = lb.Plan(ro, a.n, a.nnz, schedule=sched)
        for name, dt, vb in (("f32", torch.float32, 4), ("bf16", torch.bfloat16, 2), ("f16", torch.float16, 2)):
            v = torch.from_numpy(a.values).to(dev).to(dt)
            ms = _time(torch, lambda: plan.spmv(ci, v, x, out=y), 30)
            out[f"{sched}_{name}"] = {"ms": ms, "GBps": spmv_bytes(a.m, a.n, a.nnz, vb) / (ms * 1e-3) / 1e9}
        out[f"{sched}_bf16_speedup_vs_f32"] = out[f"{sched}_f32"]["ms"] / out[f"{sched}_bf16"]["ms"]
    return out


def run_spmm(lb, torch, dev, a, plan, ci, v, xd, y):
    """SpMM C = A B on the same matrix with B of 4, 8, 16 and 32 columns (kc = 4 runs the quad
    warp kernel, 8 and 16 the wide warp kernel, 32 the block kernel), against kc SpMV calls.
    Bytes: nonzeros (value + index), row offsets, B and C once each."""
    out = {}
    spmv_ms = _time(torch, lambda: plan.spmv(ci, v, xd, out=y), 20)
    for kc in (4, 8, 16, 32):
        B = torch.rand(a.n, kc, device=dev) * 2 - 1
        C = torch.empty(a.m, kc, device=dev)
        ms = _time(torch, lambda: plan.spmm(ci, v, B, out=C), 10)
        byts = a.nnz * 8 + 4 * (a.m + 1) + 4 * kc * (a.n + a.m)
        out[f"kc{kc}"] = {"ms": ms, "GBps": byts / (ms * 1e-3) / 1e9, "GFLOPs": 2.0 * a.nnz * kc / (ms * 1e-3) / 1e9,
                          "speedup_vs_kc_spmv_calls": kc * spmv_ms / ms}
        del B, C
    return out


def run_sssp(lb, torch, dev, a, ro, ci):
    """SSSP and BFS from vertex 0 over the same matrix read as a directed graph (integer
    weights 1..99, then unit weights), wall time per run including the per-iteration host
    synchronizations; edges/s counts the graph's edges."""
    w = torch.randint(1, 100, (a.nnz,), device=dev, generator=torch.Generator(device=dev).manual_seed(7)).float()
    out = {}
    for name, wt in (("sssp", w), ("bfs", None)):
        lb.sssp(ro, ci, wt, 0)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        reps = 3
        for _ in range(reps):
            dist, iters = lb.sssp(ro, ci, wt, 0)
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) / reps * 1e3
        out[name] = {"ms": ms, "iterations": iters, "edges_per_s": a.nnz / (ms * 1e-3),
                     "reachable": int(torch.isfinite(dist).sum().item())}
    return out


def _graph_ms(torch, fn, reps=20):
    """Mean ms of one call of fn replayed from a CUDA graph (fn's first call runs outside
    the capture: kernel attributes are set there)."""
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        fn()
    torch.cuda.current_stream().wait_stream(s)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        fn()
    return _time(torch, graph.replay, reps)


def run_batched(lb, torch, dev):
    """Two batch classes, each as one launch replayed from a CUDA graph under both batch
    schedules (the global merge path; thread-mapped rows with long rows summed by the warp)
    and in the shipped table's choice for its class; batched_4096 also against one planned
    call per matrix (the plain per-matrix form)."""
    from paper_2212_08964_gb300 import autotune, synth

    table = autotune.default_table()
    out = {}
    for name in ("batched_4096", "batched_grid_1024"):
        b = synth.workload(name)
        xs = torch.from_numpy(synth.uniform_pm1(np.random.default_rng(5), int(b.ns.sum()))).to(dev)
        bci, bv = torch.from_numpy(b.col_idx).to(dev), torch.from_numpy(b.values).to(dev)
        bro = torch.from_numpy(b.row_offsets).to(dev)
        yb = torch.empty(int(b.ms.sum()), device=dev)
        total = sum(spmv_bytes(int(m), int(n), int(z)) for m, n, z in zip(b.ms, b.ns, b.nnzs))
        r = {"workload": f"{name}: {b.count} matrices, {int(b.ms.sum())} rows, {int(b.nnzs.sum())} nonzeros",
             "bytes": total}
        for sched in ("merge_path", "thread_mapped"):
            bp = lb.BatchedPlan(b.ms, b.ns, b.nnzs, bro, schedule=sched)
            ms_b = _graph_ms(torch, lambda: bp.spmv(bci, bv, xs, out=yb))
            r[sched] = {"graph_ms": ms_b, "graph_GBps": total / (ms_b * 1e-3) / 1e9,
                        "launches": 2 if sched == "merge_path" else 1}
            bp.close()
        bp = autotune.batched_plan_for(b.ms, b.ns, b.nnzs, bro, table)
        info = bp.info()
        ms_t = _graph_ms(torch, lambda: bp.spmv(bci, bv, xs, out=yb))
        r["tuned"] = {"schedule": info["schedule"], "shape": [info["threads"], info["items_per_thread"]],
                      "graph_ms": ms_t, "graph_GBps": total / (ms_t * 1e-3) / 1e9}
        if name == "batched_4096":
            plans, views = [], []
            ro_pos = nz_pos = x_pos = y_pos = 0
            for i in range(b.count):
                m, n, z = int(b.ms[i]), int(b.ns[i]), int(b.nnzs[i])
                p = lb.Plan(bro[ro_pos: ro_pos + m + 1], n, z, schedule="auto")
                plans.append(p)
                views.append((bci[nz_pos: nz_pos + z], bv[nz_pos: nz_pos + z], xs[x_pos: x_pos + n],
                              yb[y_pos: y_pos + m]))
                ro_pos += m + 1
                nz_pos += z
                x_pos += n
                y_pos += m

            def per_matrix():
                for p, (c_, v_, x_, y_) in zip(plans, views):
                    p.spmv(c_, v_, x_, out=y_)

            ms_p = _time(torch, per_matrix, 3)
            r["per_matrix_ms"] = ms_p
            r["per_matrix_GBps"] = total / (ms_p * 1e-3) / 1e9
            r["per_matrix_launches"] = 2 * b.count
            r["tuned_speedup_vs_per_matrix"] = ms_p / ms_t
            for p in plans:
                p.close()
        out[name] = r
        del b, bci, bv, bro, yb, xs
    return out


def _time(torch, fn, reps):
    for _ in range(3):
        fn()
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(reps):
        fn()
    e.record()
    torch.cuda.synchronize()
    return s.elapsed_time(e) / reps


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
