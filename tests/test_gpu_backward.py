"""Backward on the GPU vs the oracle: the CSC plan (stable transpose and its partition)
bit-exact; dx = A^T g within 1e-5 * sum_i |a_ij||g_i| per column; dvalues = g[row] x[col]
bit-exact (one rounding of an exact product); autograd end to end."""
import numpy as np
import pytest
import torch

from golden.fixtures import load
from gpu_helpers import check_bound, dev, rounded, to_dev, vec, workload
from paper_2212_08964_gb300 import synth

pytestmark = pytest.mark.gpu

TOL32 = 1e-5


def _plan_with_t(lb, a, schedule="merge_path", dtype=torch.float32, **tune):
    ro, ci, v = to_dev(a, dtype)
    plan = lb.Plan(ro, a.n, a.nnz, schedule=schedule, **tune)
    plan.build_transpose(ci)
    return plan, ci, v


def _cases():
    f = load("worked_example_4x4.txt")
    worked = synth.CSR(4, 4, f["row_offsets"].astype(np.int32), f["col_idx"].astype(np.int32), f["values"].astype(np.float32))
    rng = np.random.default_rng(11)
    # Columns concentrated in a few: long columns and many empty ones.
    skew = synth.csr_from_row_lengths(rng, 300, rng.integers(0, 40, 5000))
    wide = synth.csr_from_row_lengths(rng, 70_000, rng.integers(0, 9, 3000))  # n > 2^16: three radix passes
    return {"worked": worked, "powerlaw_4k": workload("powerlaw_4k"), "skew": skew, "wide": wide,
            "stencil_small": synth.stencil7_csr(12, seed=3)}


@pytest.mark.parametrize("name", ["worked", "powerlaw_4k", "skew", "wide", "stencil_small"])
def test_transpose_and_its_partition_bit_exact(lb, orc, name):
    a = _cases()[name]
    plan, _, _ = _plan_with_t(lb, a)
    co, ri, perm = plan.transpose()
    oco, ori, operm = orc.transpose(a.row_offsets, a.col_idx, a.n)
    assert np.array_equal(co, oco) and np.array_equal(ri, ori) and np.array_equal(perm, operm)
    tr, tn = plan.partition(transposed=True)
    assert plan.tiles("transposed")[0] == len(tr) - 1
    otr, otn = orc.partition(oco, plan.tiles("transposed")[1])
    assert np.array_equal(tr, otr) and np.array_equal(tn, otn)


@pytest.mark.parametrize("name", ["worked", "powerlaw_4k", "skew", "wide", "stencil_small"])
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_spmv_t_and_dvalues(lb, orc, name, dtype):
    a = _cases()[name]
    plan, ci, v = _plan_with_t(lb, a, dtype=dtype)
    g = vec(a.m, 201)
    x = vec(a.n, 202)
    dx = plan.spmv_t(v, dev(g))
    dv = plan.dvalues(ci, dev(g), dev(x))
    torch.cuda.synchronize()
    vals = a.values if dtype == torch.float32 else rounded(a.values, dtype)
    ref = orc.spmv_t(a.row_offsets, a.col_idx, vals, g, a.n)
    scale = orc.col_absdot(a.row_offsets, a.col_idx, vals, g, a.n)
    check_bound(dx.cpu().numpy(), ref, scale, TOL32, "columns")
    dv_ref = orc.dvalues(a.row_offsets, a.col_idx, g, x).astype(np.float32)
    assert np.array_equal(dv.cpu().numpy(), dv_ref)


@pytest.mark.parametrize("name", ["worked", "powerlaw_4k", "skew", "wide", "stencil_small"])
@pytest.mark.parametrize("shape", [(256, 8), (128, 16), (512, 8)])
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_saved_gathers(lb, orc, name, shape, dtype):
    """The forward that saves x[col] per nonzero: y unchanged bit for bit, the saved gathers
    equal x[col] exactly, and dvalues from them equal the oracle's products exactly."""
    a = _cases()[name]
    ro, ci, v = to_dev(a, dtype)
    plan = lb.Plan(ro, a.n, a.nnz, schedule="merge_path", threads=shape[0], items_per_thread=shape[1])
    x = vec(a.n, 205)
    g = vec(a.m, 206)
    xd = dev(x)
    y0 = plan.spmv(ci, v, xd)
    xg = torch.full((a.nnz,), float("nan"), device="cuda")
    y1 = plan.spmv(ci, v, xd, save_gathered=xg)
    dv = plan.dvalues_gathered(dev(g), xg)
    torch.cuda.synchronize()
    assert torch.equal(y0, y1)
    assert np.array_equal(xg.cpu().numpy(), x[a.col_idx])
    dv_ref = orc.dvalues(a.row_offsets, a.col_idx, g, x).astype(np.float32)
    assert np.array_equal(dv.cpu().numpy(), dv_ref)


def test_saved_gathers_unaligned_views(lb, orc):
    """Column indices and the saved-gather buffer at element offsets 1..3 (16-byte alignment
    differs between them), through the scalar-store path."""
    a = workload("powerlaw_4k")
    x = vec(a.n, 207)
    g = vec(a.m, 208)
    for off_c, off_g in [(1, 0), (0, 3), (2, 1), (3, 3)]:
        ci_buf = torch.zeros(a.nnz + 4, dtype=torch.int32, device="cuda")
        ci_buf[off_c: off_c + a.nnz] = dev(a.col_idx)
        ci = ci_buf[off_c: off_c + a.nnz]
        xg_buf = torch.full((a.nnz + 4,), float("nan"), device="cuda")
        xg = xg_buf[off_g: off_g + a.nnz]
        plan = lb.Plan(dev(a.row_offsets), a.n, a.nnz, schedule="merge_path")
        plan.spmv(ci, dev(a.values), dev(x), save_gathered=xg)
        dv = plan.dvalues_gathered(dev(g), xg)
        torch.cuda.synchronize()
        assert np.array_equal(xg.cpu().numpy(), x[a.col_idx])
        assert torch.isnan(xg_buf[:off_g]).all() and torch.isnan(xg_buf[off_g + a.nnz:]).all()
        assert np.array_equal(dv.cpu().numpy(), orc.dvalues(a.row_offsets, a.col_idx, g, x).astype(np.float32))


@pytest.mark.parametrize("name", ["worked", "powerlaw_4k", "skew", "wide", "stencil_small"])
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16, torch.float16])
@pytest.mark.parametrize("bucket_shift", [None, "10", "12"])
def test_two_pass_backward(lb, orc, monkeypatch, name, dtype, bucket_shift):
    """lb_spmv_backward: dx and dvalues from one CSR-order pass plus the gather-sum, equal bit
    for bit to lb_spmv_t and lb_spmv_dvalues_gathered, and to the oracle within tolerance."""
    if bucket_shift:
        monkeypatch.setenv("LBSPMV_VALUE_BUCKET_SHIFT", bucket_shift)
    a = _cases()[name]
    plan, ci, v = _plan_with_t(lb, a, dtype=dtype)
    x = vec(a.n, 211)
    g = vec(a.m, 212)
    xg = torch.empty(a.nnz, device="cuda")
    plan.spmv(ci, v, dev(x), save_gathered=xg)
    dx, dv = plan.backward(v, dev(g), xg)
    dx2 = plan.spmv_t(v, dev(g))
    dv2 = plan.dvalues_gathered(dev(g), xg)
    torch.cuda.synchronize()
    assert torch.equal(dx, dx2) and torch.equal(dv, dv2)
    vals = a.values if dtype == torch.float32 else rounded(a.values, dtype)
    check_bound(dx.cpu().numpy(), orc.spmv_t(a.row_offsets, a.col_idx, vals, g, a.n),
                orc.col_absdot(a.row_offsets, a.col_idx, vals, g, a.n), TOL32, "columns")
    assert np.array_equal(dv.cpu().numpy(), orc.dvalues(a.row_offsets, a.col_idx, g, x).astype(np.float32))


def test_two_pass_backward_unaligned_views(lb, orc):
    """Values, saved gathers and dvalues at element offsets that break 16-byte alignment."""
    a = workload("powerlaw_4k")
    x = vec(a.n, 213)
    g = vec(a.m, 214)
    ro, ci, _ = to_dev(a)
    plan = lb.Plan(ro, a.n, a.nnz, schedule="merge_path")
    plan.build_transpose(ci)
    ref_dx = orc.spmv_t(a.row_offsets, a.col_idx, a.values, g, a.n)
    scale = orc.col_absdot(a.row_offsets, a.col_idx, a.values, g, a.n)
    ref_dv = orc.dvalues(a.row_offsets, a.col_idx, g, x).astype(np.float32)
    for dtype in (torch.float32, torch.bfloat16):
        for off_v, off_x, off_d in [(1, 0, 0), (0, 2, 0), (0, 0, 3), (3, 1, 2)]:
            vb = torch.zeros(a.nnz + 4, dtype=dtype, device="cuda")
            vb[off_v: off_v + a.nnz] = dev(a.values, dtype)
            v = vb[off_v: off_v + a.nnz]
            xgb = torch.zeros(a.nnz + 4, device="cuda")
            xg = xgb[off_x: off_x + a.nnz]
            dvb = torch.full((a.nnz + 4,), float("nan"), device="cuda")
            dvv = dvb[off_d: off_d + a.nnz]
            plan.spmv(ci, v, dev(x), save_gathered=xg)
            dx, _ = plan.backward(v, dev(g), xg, dvalues=dvv)
            torch.cuda.synchronize()
            assert np.array_equal(dvv.cpu().numpy(), ref_dv)
            assert torch.isnan(dvb[:off_d]).all() and torch.isnan(dvb[off_d + a.nnz:]).all()
            vals = a.values if dtype == torch.float32 else rounded(a.values, dtype)
            check_bound(dx.cpu().numpy(), orc.spmv_t(a.row_offsets, a.col_idx, vals, g, a.n),
                        orc.col_absdot(a.row_offsets, a.col_idx, vals, g, a.n), TOL32, "columns")


@pytest.mark.parametrize("sched", ["merge_path", "thread_mapped", "warp_mapped"])
@pytest.mark.parametrize("deterministic", [True, False])
def test_autograd_function(lb, orc, sched, deterministic):
    """Both gradients through the autograd function; deterministic=False takes dx from the
    scatter backward and builds no CSC view."""
    a = workload("powerlaw_4k")
    ro, ci, v = to_dev(a)
    plan = lb.Plan(ro, a.n, a.nnz, schedule=sched)
    x = vec(a.n, 203)
    g = vec(a.m, 204)
    vt = v.clone().requires_grad_(True)
    xt = dev(x).requires_grad_(True)
    y = lb.spmv_autograd(plan, ci, vt, xt, deterministic=deterministic)
    y.backward(dev(g))
    torch.cuda.synchronize()
    assert plan.has_transpose == deterministic
    ref_dx = orc.spmv_t(a.row_offsets, a.col_idx, a.values, g, a.n)
    scale = orc.col_absdot(a.row_offsets, a.col_idx, a.values, g, a.n)
    check_bound(xt.grad.cpu().numpy(), ref_dx, scale, TOL32, "columns")
    assert np.array_equal(vt.grad.cpu().numpy(), orc.dvalues(a.row_offsets, a.col_idx, g, x).astype(np.float32))


def test_autograd_quadratic_loss_gradient(lb, orc):
    """L = 1/2 ||A x - t||^2 on the finite-difference-sized log-normal matrix: GPU gradients
    against the oracle's (which finite differences pin in the CPU tests)."""
    a = synth.lognormal_csr(256, 256, 2.5, 1.2, seed=4, l_max=256)
    rng = np.random.default_rng(12)
    x = rng.uniform(-1, 1, a.n).astype(np.float32)
    t = rng.uniform(-1, 1, a.m).astype(np.float32)
    ro, ci, v = to_dev(a)
    plan = lb.Plan(ro, a.n, a.nnz, schedule="merge_path")
    vt = v.clone().requires_grad_(True)
    xt = dev(x).requires_grad_(True)
    y = lb.spmv_autograd(plan, ci, vt, xt)
    loss = 0.5 * ((y - dev(t)) ** 2).sum()
    loss.backward()
    torch.cuda.synchronize()
    g = orc.spmv(a.row_offsets, a.col_idx, a.values, x) - t
    dx = orc.spmv_t(a.row_offsets, a.col_idx, a.values, g, a.n)
    dv = orc.dvalues(a.row_offsets, a.col_idx, g, x)
    # g on the GPU carries the forward's error (<= 1e-5 * sum|a||x| per row) into both
    # gradients, so the bound scale is |g| + sum|a||x| per row.
    ys = orc.row_absdot(a.row_offsets, a.col_idx, a.values, x)
    gs = np.abs(g) + ys
    sdx = orc.col_absdot(a.row_offsets, a.col_idx, a.values, gs, a.n)
    check_bound(xt.grad.cpu().numpy(), dx, sdx, 2e-5, "columns")
    rows = np.repeat(np.arange(a.m), a.row_lengths())
    sdv = gs[rows] * np.abs(x[a.col_idx])
    check_bound(vt.grad.cpu().numpy(), dv, sdv, 2e-5, "nonzeros")


def test_full_size_lognormal_1m(lb, orc):
    """The differentiable configuration at full size: forward, dx and dvalues."""
    a = workload("lognormal_1m")
    plan, ci, v = _plan_with_t(lb, a)
    x = vec(a.n, 4)
    g = vec(a.m, 5)
    y = plan.spmv(ci, v, dev(x))
    dx = plan.spmv_t(v, dev(g))
    dv = plan.dvalues(ci, dev(g), dev(x))
    torch.cuda.synchronize()
    ref_y = orc.spmv(a.row_offsets, a.col_idx, a.values, x)
    check_bound(y.cpu().numpy(), ref_y, orc.row_absdot(a.row_offsets, a.col_idx, a.values, x), TOL32)
    ref_dx = orc.spmv_t(a.row_offsets, a.col_idx, a.values, g, a.n)
    mx, med = check_bound(dx.cpu().numpy(), ref_dx, orc.col_absdot(a.row_offsets, a.col_idx, a.values, g, a.n), TOL32, "columns")
    print(f"lognormal_1m dx: max rel err {mx:.3e} median {med:.3e}")
    assert np.array_equal(dv.cpu().numpy(), orc.dvalues(a.row_offsets, a.col_idx, g, x).astype(np.float32))
    co, ri, perm = plan.transpose()
    oco, ori, operm = orc.transpose(a.row_offsets, a.col_idx, a.n)
    assert np.array_equal(co, oco) and np.array_equal(ri, ori) and np.array_equal(perm, operm)


def test_full_size_powerlaw_4m_backward(lb, orc):
    """Backward on the large power-law matrix, as the benchmark's step runs it."""
    a = workload("powerlaw_4m")
    plan, ci, v = _plan_with_t(lb, a)
    x = vec(a.n, 1)
    g = vec(a.m, 3)
    xg = torch.empty(a.nnz, device="cuda")
    y = plan.spmv(ci, v, dev(x), save_gathered=xg)
    dx, dv = plan.backward(v, dev(g), xg)
    dv2 = plan.dvalues(ci, dev(g), dev(x))
    torch.cuda.synchronize()
    ref_y = orc.spmv(a.row_offsets, a.col_idx, a.values, x)
    check_bound(y.cpu().numpy(), ref_y, orc.row_absdot(a.row_offsets, a.col_idx, a.values, x), TOL32)
    ref_dx = orc.spmv_t(a.row_offsets, a.col_idx, a.values, g, a.n)
    mx, med = check_bound(dx.cpu().numpy(), ref_dx, orc.col_absdot(a.row_offsets, a.col_idx, a.values, g, a.n), TOL32, "columns")
    print(f"powerlaw_4m dx: max rel err {mx:.3e} median {med:.3e}")
    dv_ref = orc.dvalues(a.row_offsets, a.col_idx, g, x).astype(np.float32)
    assert np.array_equal(dv.cpu().numpy(), dv_ref)
    assert torch.equal(dv, dv2)


def test_bucketed_value_permutation(lb, orc, monkeypatch):
    """Small value buckets (2^10 CSC entries) force the bucketed path on a small matrix."""
    monkeypatch.setenv("LBSPMV_VALUE_BUCKET_SHIFT", "10")
    a = workload("powerlaw_4k")
    for dtype in (torch.float32, torch.bfloat16, torch.float16):
        plan, ci, v = _plan_with_t(lb, a, dtype=dtype)
        g = vec(a.m, 205)
        dx1 = plan.spmv_t(v, dev(g))
        dx2 = plan.spmv_t(v, dev(g))
        torch.cuda.synchronize()
        assert torch.equal(dx1, dx2)
        vals = a.values if dtype == torch.float32 else rounded(a.values, dtype)
        ref = orc.spmv_t(a.row_offsets, a.col_idx, vals, g, a.n)
        check_bound(dx1.cpu().numpy(), ref, orc.col_absdot(a.row_offsets, a.col_idx, vals, g, a.n), TOL32, "columns")
        co, ri, perm = plan.transpose()
        oco, ori, operm = orc.transpose(a.row_offsets, a.col_idx, a.n)
        assert np.array_equal(perm, operm) and np.array_equal(ri, ori)


@pytest.mark.parametrize("name", ["worked", "powerlaw_4k", "skew", "wide", "stencil_small"])
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16, torch.float16])
def test_backward_scatter(lb, orc, name, dtype):
    """lb_spmv_backward_scatter, with no CSC view: dx within tolerance of the oracle (its
    additions into a column come in no fixed order), dvalues bit-exact; dx alone as well."""
    a = _cases()[name]
    ro, ci, v = to_dev(a, dtype)
    plan = lb.Plan(ro, a.n, a.nnz, schedule="merge_path")
    x, g = vec(a.n, 241), vec(a.m, 242)
    xg = torch.empty(a.nnz, device="cuda")
    plan.spmv(ci, v, dev(x), save_gathered=xg)
    dx, dv = plan.backward_scatter(ci, v, dev(g), xg)
    dx2, none = plan.backward_scatter(ci, v, dev(g), want_dvalues=False)
    torch.cuda.synchronize()
    assert none is None
    vals = a.values if dtype == torch.float32 else rounded(a.values, dtype)
    ref = orc.spmv_t(a.row_offsets, a.col_idx, vals, g, a.n)
    scale = orc.col_absdot(a.row_offsets, a.col_idx, vals, g, a.n)
    check_bound(dx.cpu().numpy(), ref, scale, TOL32, "columns")
    check_bound(dx2.cpu().numpy(), ref, scale, TOL32, "columns")
    assert np.array_equal(dv.cpu().numpy(), orc.dvalues(a.row_offsets, a.col_idx, g, x).astype(np.float32))
    assert lb.device_error() == 0


def test_backward_scatter_unaligned_and_empty(lb, orc):
    """Column indices, values and saved gathers at offsets that break 16-byte alignment; and a
    matrix without nonzeros (dx all zero)."""
    a = workload("powerlaw_4k")
    x, g = vec(a.n, 243), vec(a.m, 244)
    ro = dev(a.row_offsets)
    ci_buf = torch.zeros(a.nnz + 4, dtype=torch.int32, device="cuda")
    ci_buf[1: 1 + a.nnz] = dev(a.col_idx)
    v_buf = torch.zeros(a.nnz + 4, device="cuda")
    v_buf[3: 3 + a.nnz] = dev(a.values)
    ci, v = ci_buf[1: 1 + a.nnz], v_buf[3: 3 + a.nnz]
    plan = lb.Plan(ro, a.n, a.nnz, schedule="merge_path")
    xg_buf = torch.zeros(a.nnz + 4, device="cuda")
    xg = xg_buf[2: 2 + a.nnz]
    plan.spmv(ci, v, dev(x), save_gathered=xg)
    dx, dv = plan.backward_scatter(ci, v, dev(g), xg)
    torch.cuda.synchronize()
    check_bound(dx.cpu().numpy(), orc.spmv_t(a.row_offsets, a.col_idx, a.values, g, a.n),
                orc.col_absdot(a.row_offsets, a.col_idx, a.values, g, a.n), TOL32, "columns")
    assert np.array_equal(dv.cpu().numpy(), orc.dvalues(a.row_offsets, a.col_idx, g, x).astype(np.float32))
    empty = lb.Plan(torch.zeros(6, dtype=torch.int32, device="cuda"), 9, 0, schedule="merge_path")
    dx0 = torch.full((9,), 7.0, device="cuda")
    empty.backward_scatter(torch.zeros(0, dtype=torch.int32, device="cuda"), torch.zeros(0, device="cuda"),
                           torch.ones(5, device="cuda"), want_dvalues=False, dx=dx0)
    torch.cuda.synchronize()
    assert torch.equal(dx0, torch.zeros(9, device="cuda"))


def test_training_step_in_a_cuda_graph(lb, orc):
    """Forward saving its gathers plus the two-pass backward, captured once in a CUDA graph and
    replayed: the same bits as eager calls (no allocation or synchronization inside)."""
    a = workload("lognormal_1m", 0.1)
    plan, ci, v = _plan_with_t(lb, a)
    x, g = dev(vec(a.n, 221)), dev(vec(a.m, 222))
    y, dx = torch.empty(a.m, device="cuda"), torch.empty(a.n, device="cuda")
    dv, xg = torch.empty(a.nnz, device="cuda"), torch.empty(a.nnz, device="cuda")

    def step():
        plan.spmv(ci, v, x, out=y, save_gathered=xg)
        plan.backward(v, g, xg, dx=dx, dvalues=dv)

    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        step()  # first calls outside the capture (kernel attributes, occupancy queries)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    ref = (y.clone(), dx.clone(), dv.clone())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    for t in (y, dx, dv):
        t.zero_()
    graph.replay()
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(y, ref[0]) and torch.equal(dx, ref[1]) and torch.equal(dv, ref[2])
    check_bound(dx.cpu().numpy(), orc.spmv_t(a.row_offsets, a.col_idx, a.values, vec(a.m, 222), a.n),
                orc.col_absdot(a.row_offsets, a.col_idx, a.values, vec(a.m, 222), a.n), TOL32, "columns")


def _dv16(ref_f64, dtype):
    """The oracle's dvalues as the library stores them in a 16-bit type: the exact product of
    two FP32 numbers rounded to FP32 (what FP32 arithmetic gives), then to nearest even."""
    return torch.from_numpy(ref_f64.astype(np.float32)).to(dtype)


@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float16])
@pytest.mark.parametrize("name", ["powerlaw_4k", "skew", "worked"])
def test_values_gradient_in_the_values_type(lb, orc, name, dtype):
    """dvalues stored in the 16-bit values' own type by every entry point that forms it (the
    two-pass backward, the scattered backward, from saved gathers and gathering x), bit-exact
    against the oracle's product rounded the same way; another 16-bit type is refused."""
    a = _cases()[name]
    plan, ci, v = _plan_with_t(lb, a, dtype=dtype)
    x = vec(a.n, 231)
    g = vec(a.m, 232)
    xg = torch.empty(a.nnz, device="cuda")
    plan.spmv(ci, v, dev(x), save_gathered=xg)
    ref = _dv16(orc.dvalues(a.row_offsets, a.col_idx, g, x), dtype)
    dx32, dv32 = plan.backward(v, dev(g), xg)
    dx, dv = plan.backward(v, dev(g), xg, dvalues_dtype=dtype)
    _, dvs = plan.backward_scatter(ci, v, dev(g), xg, dvalues_dtype=dtype)
    dvg = plan.dvalues_gathered(dev(g), xg, dtype=dtype)
    dvx = plan.dvalues(ci, dev(g), dev(x), dtype=dtype)
    torch.cuda.synchronize()
    assert torch.equal(dx, dx32)
    for got in (dv, dvs, dvg, dvx):
        assert got.dtype == dtype and torch.equal(got.cpu(), ref)
    assert torch.equal(dv.cpu(), dv32.cpu().to(dtype))
    with pytest.raises(TypeError):
        plan.backward(v, dev(g), xg, dvalues_dtype=torch.float16 if dtype == torch.bfloat16 else torch.bfloat16)
    # A 16-bit gradient one element off a 16-byte boundary takes the element-wise stores.
    buf = torch.full((a.nnz + 1,), float("nan"), dtype=dtype, device="cuda")
    plan.backward(v, dev(g), xg, dvalues=buf[1:])
    torch.cuda.synchronize()
    assert torch.equal(buf[1:].cpu(), ref) and torch.isnan(buf[:1]).all()


@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float16])
@pytest.mark.parametrize("deterministic", [True, False])
def test_autograd_values_gradient_16bit(lb, orc, dtype, deterministic):
    """With 16-bit values, the autograd function's values gradient arrives in that type from
    the library's kernels, equal to the oracle's product rounded to nearest even."""
    a = workload("powerlaw_4k")
    ro, ci, v = to_dev(a, dtype)
    plan = lb.Plan(ro, a.n, a.nnz, schedule="merge_path")
    x = vec(a.n, 233)
    g = vec(a.m, 234)
    vt = v.clone().requires_grad_(True)
    xt = dev(x).requires_grad_(True)
    y = lb.spmv_autograd(plan, ci, vt, xt, deterministic=deterministic)
    y.backward(dev(g))
    torch.cuda.synchronize()
    assert vt.grad.dtype == dtype
    assert torch.equal(vt.grad.cpu(), _dv16(orc.dvalues(a.row_offsets, a.col_idx, g, x), dtype))
