"""Out-of-memory paths on the GPU, with the failure injected on the host: the library's n-th
device allocation is made to fail (lb_debug_fail_allocations_after) for every n up to the
first success.  Each failing call must report LB_ERR_NO_MEMORY, hand back no plan, hold no
allocation afterwards, and leave the library usable: the next call without the limit matches
the oracle."""
import numpy as np
import pytest
import torch

from gpu_helpers import check_bound, dev, to_dev, vec, workload

pytestmark = pytest.mark.gpu

NO_MEMORY = -4


def _no_memory(exc: Exception) -> bool:
    return getattr(exc, "status", None) == NO_MEMORY or "LB_ERR_NO_MEMORY" in str(exc)


def _fail_each_allocation(lb, make, limit=40):
    """Run make() with the n-th allocation failing, n = 0, 1, ...; returns the first success
    and how many allocations it needed."""
    torch.cuda.synchronize()
    live = lb.live_allocations()
    for n in range(limit):
        lb.fail_allocations_after(n)
        try:
            obj = make()
        except Exception as exc:  # noqa: BLE001 - the binding raises LbError
            assert _no_memory(exc), exc
            torch.cuda.synchronize()
            assert lb.live_allocations() == live, f"allocation {n}: a failed call kept device memory"
            continue
        finally:
            lb.fail_allocations_after(-1)
        return obj, n
    raise AssertionError("no success within the allocation limit")


@pytest.mark.parametrize("schedule", ["merge_path", "nonzero_split"])
def test_plan_and_transpose_out_of_memory(lb, orc, schedule):
    a = workload("powerlaw_4k")
    ro, ci, v = to_dev(a)
    plan, n_plan = _fail_each_allocation(lb, lambda: lb.Plan(ro, a.n, a.nnz, schedule=schedule))
    assert n_plan >= 4

    def with_transpose():
        plan.build_transpose(ci)
        return plan

    _, n_t = _fail_each_allocation(lb, with_transpose)
    assert n_t >= 1
    x, g = vec(a.n, 1), vec(a.m, 2)
    y = plan.spmv(ci, v, dev(x))
    dx = plan.spmv_t(v, dev(g))
    torch.cuda.synchronize()
    check_bound(y.cpu().numpy(), orc.spmv(a.row_offsets, a.col_idx, a.values, x),
                orc.row_absdot(a.row_offsets, a.col_idx, a.values, x), 1e-5)
    check_bound(dx.cpu().numpy(), orc.spmv_t(a.row_offsets, a.col_idx, a.values, g, a.n),
                orc.col_absdot(a.row_offsets, a.col_idx, a.values, g, a.n), 1e-5, "columns")
    plan.close()
    assert lb.device_error() == 0


def test_one_shot_and_batched_out_of_memory(lb, orc):
    a = workload("powerlaw_4m", 0.01)  # merge path by the size rule
    ro, ci, v = to_dev(a)
    x = vec(a.n, 3)
    y, n_one = _fail_each_allocation(lb, lambda: lb.spmv(ro, ci, v, dev(x)))
    assert n_one == 1  # the one-shot call's single workspace
    torch.cuda.synchronize()
    check_bound(y.cpu().numpy(), orc.spmv(a.row_offsets, a.col_idx, a.values, x),
                orc.row_absdot(a.row_offsets, a.col_idx, a.values, x), 1e-5)

    from paper_2212_08964_gb300 import synth

    b = synth.batched_powerlaw(12, 64, 2048, 15_000, 1.5, seed=9)
    bro = dev(b.row_offsets)
    bp, n_b = _fail_each_allocation(lb, lambda: lb.BatchedPlan(b.ms, b.ns, b.nnzs, bro))
    assert n_b >= 4
    xb = vec(int(b.ns.sum()), 4)
    yb = bp.spmv(dev(b.col_idx), dev(b.values), dev(xb))
    torch.cuda.synchronize()
    check_bound(yb.cpu().numpy(), orc.batched_spmv(b, xb), orc.batched_row_absdot(b, xb), 1e-5)
    bp.close()
    assert lb.device_error() == 0


def test_calls_documented_to_allocate_nothing(lb, orc):
    """With every allocation failing, the calls the header documents as allocation-free
    still succeed: the planned forward (with and without saved gathers), the transposed
    product, the backward, dvalues and lb_validate_csr."""
    a = workload("powerlaw_4k")
    ro, ci, v = to_dev(a)
    plan = lb.Plan(ro, a.n, a.nnz, schedule="merge_path")
    plan.build_transpose(ci)
    x, g = dev(vec(a.n, 5)), dev(vec(a.m, 6))
    y, dx, dv, xg = (torch.empty(a.m, device="cuda"), torch.empty(a.n, device="cuda"),
                     torch.empty(a.nnz, device="cuda"), torch.empty(a.nnz, device="cuda"))
    torch.cuda.synchronize()
    lb.fail_allocations_after(0)
    try:
        plan.spmv(ci, v, x, out=y)
        plan.spmv(ci, v, x, out=y, save_gathered=xg)
        plan.spmv_t(v, g, out=dx)
        plan.backward(v, g, xg, dx=dx, dvalues=dv)
        plan.dvalues(ci, g, x, out=dv)
        assert lb.validate_csr(ro, ci, a.n) == 0
        torch.cuda.synchronize()
    finally:
        lb.fail_allocations_after(-1)
    xh = x.cpu().numpy()
    check_bound(y.cpu().numpy(), orc.spmv(a.row_offsets, a.col_idx, a.values, xh),
                orc.row_absdot(a.row_offsets, a.col_idx, a.values, xh), 1e-5)
    plan.close()
