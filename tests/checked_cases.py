"""Cases run against the range-checked build (liblbspmv_checked.so), in a process of their
own with LBSPMV_CHECKED=1 (tests/test_gpu_checked.py starts it).

1. Valid inputs through every schedule and pass (merge path forward with and without saved
   gathers, the backward over the CSC view and by float reductions, thread-, warp-, block-
   and group-mapped, nonzero splitting, batched, SpMM, SSSP): results match the oracle and no
   range check fires.
2. A column index outside [0, n) planted in the inputs: each kernel that gathers by column
   (merge path, the mapped schedules, nonzero splitting, SpMM, the scattered backward, dvalues
   gathering x) skips the access and records LB_ERR_OUT_OF_RANGE; nothing reads outside x.
"""
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "tests"))

import oracle  # noqa: E402
from gpu_helpers import check_bound, dev, to_dev, vec, workload  # noqa: E402
from paper_2212_08964_gb300 import lbspmv as lb  # noqa: E402
from paper_2212_08964_gb300 import synth  # noqa: E402

OUT_OF_RANGE = -8


def rows_ok(got, a, x):
    check_bound(got.cpu().numpy(), oracle.spmv(a.row_offsets, a.col_idx, a.values, x),
                oracle.row_absdot(a.row_offsets, a.col_idx, a.values, x), 1e-5)


def valid_inputs():
    a = workload("powerlaw_4k")
    ro, ci, v = to_dev(a)
    x, g = vec(a.n, 1), vec(a.m, 2)
    xd, gd = dev(x), dev(g)
    for sched in ["merge_path", "thread_mapped", "warp_mapped", "block_mapped", "group_mapped", "nonzero_split"]:
        plan = lb.Plan(ro, a.n, a.nnz, schedule=sched)
        rows_ok(plan.spmv(ci, v, xd), a, x)
        plan.close()
    plan = lb.Plan(ro, a.n, a.nnz, schedule="merge_path")
    plan.build_transpose(ci)
    xg = torch.empty(a.nnz, device="cuda")
    rows_ok(plan.spmv(ci, v, xd, save_gathered=xg), a, x)
    dx, dv = torch.empty(a.n, device="cuda"), torch.empty(a.nnz, device="cuda")
    plan.backward(v, gd, xg, dx=dx, dvalues=dv)
    dx_ref = oracle.spmv_t(a.row_offsets, a.col_idx, a.values, g, a.n)
    dx_scale = oracle.col_absdot(a.row_offsets, a.col_idx, a.values, g, a.n)
    check_bound(dx.cpu().numpy(), dx_ref, dx_scale, 1e-5, "columns")
    dv_ref = oracle.dvalues(a.row_offsets, a.col_idx, g, x).astype(np.float32)
    assert np.array_equal(dv.cpu().numpy(), dv_ref)
    plan.backward_scatter(ci, v, gd, xg, dx=dx, dvalues=dv)
    check_bound(dx.cpu().numpy(), dx_ref, dx_scale, 1e-5, "columns")
    assert np.array_equal(plan.dvalues(ci, gd, xd).cpu().numpy(), dv_ref)
    B = np.random.default_rng(3).uniform(-1, 1, (a.n, 8)).astype(np.float32)
    C = plan.spmm(ci, v, dev(B))
    check_bound(C.cpu().numpy(), oracle.spmm(a.row_offsets, a.col_idx, a.values, B),
                oracle.spmm_absdot(a.row_offsets, a.col_idx, a.values, B), 1e-5)
    plan.close()
    b = synth.batched_powerlaw(16, 64, 2048, 20_000, 1.5, seed=5)
    xb = vec(int(b.ns.sum()), 4)
    bp = lb.BatchedPlan(b.ms, b.ns, b.nnzs, dev(b.row_offsets))
    yb = bp.spmv(dev(b.col_idx), dev(b.values), dev(xb))
    check_bound(yb.cpu().numpy(), oracle.batched_spmv(b, xb), oracle.batched_row_absdot(b, xb), 1e-5)
    bp.close()
    w = np.random.default_rng(5).integers(1, 100, a.nnz).astype(np.float32)
    dist, _ = lb.sssp(ro, ci, dev(w), 0)
    ref = oracle.sssp(a.row_offsets, a.col_idx, w.astype(np.float64), 0)
    got = dist.cpu().numpy().astype(np.float64)
    fin = np.isfinite(ref)
    assert np.array_equal(np.isinf(got), ~fin) and np.array_equal(got[fin], ref[fin])
    assert lb.device_error() == 0, "a range check fired on valid inputs"


def planted_column():
    a = workload("powerlaw_4k")
    ro, ci, v = to_dev(a)
    bad = a.col_idx.copy()
    bad[a.nnz // 3] = a.n + 7
    bad[a.nnz // 2] = -3
    bci = dev(bad)
    xd, gd = dev(vec(a.n, 1)), dev(vec(a.m, 2))
    runs = {}
    for sched in ["merge_path", "thread_mapped", "warp_mapped", "block_mapped", "group_mapped", "nonzero_split"]:
        plan = lb.Plan(ro, a.n, a.nnz, schedule=sched)
        plan.spmv(bci, v, xd)
        runs[sched] = lb.device_error()
        if sched == "merge_path":
            plan.spmm(bci, v, dev(np.ones((a.n, 4), np.float32)))
            runs["spmm"] = lb.device_error()
            plan.dvalues(bci, gd, xd)
            runs["dvalues"] = lb.device_error()
            xg = torch.zeros(a.nnz, device="cuda")
            plan.backward_scatter(bci, v, gd, xg, want_dvalues=False)
            runs["backward_scatter"] = lb.device_error()
        plan.close()
    assert all(s == OUT_OF_RANGE for s in runs.values()), runs
    assert lb.device_error() == 0


if __name__ == "__main__":
    assert os.environ.get("LBSPMV_CHECKED") == "1"
    lb.ensure_loaded()
    assert lb.library_path().endswith("liblbspmv_checked.so"), lb.library_path()
    valid_inputs()
    planted_column()
    print("checked build: valid inputs match the oracle; planted columns recorded as out of range")
