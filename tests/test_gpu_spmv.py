"""Forward SpMV on the GPU (every schedule, every merge-path shape, FP32/BF16/FP16) vs the
FP64 oracle: exact where the arithmetic is exact, else |y - y_ref| <= tol * sum_j |a_ij||x_j|
per row (tol 1e-5 for FP32 values; 8e-3 for BF16/FP16 values against the unrounded values)."""
import numpy as np
import pytest
import torch

from golden.fixtures import load
from gpu_helpers import check_bound, dev, rounded, to_dev, vec, workload
from paper_2212_08964_gb300 import synth

pytestmark = pytest.mark.gpu

TOL32 = 1e-5
TOL16 = 8e-3


def _run(lb, a, x, schedule="merge_path", dtype=torch.float32, **tune):
    ro, ci, v = to_dev(a, dtype)
    plan = lb.Plan(ro, a.n, a.nnz, schedule=schedule, **tune)
    y = plan.spmv(ci, v, dev(x))
    torch.cuda.synchronize()
    return y.cpu().numpy(), plan


def _ref(orc, a, x, values=None):
    v = a.values if values is None else values
    return orc.spmv(a.row_offsets, a.col_idx, v, x), orc.row_absdot(a.row_offsets, a.col_idx, v, x)


def test_worked_example_exact(lb):
    f = load("worked_example_4x4.txt")
    a = synth.CSR(4, 4, f["row_offsets"].astype(np.int32), f["col_idx"].astype(np.int32), f["values"].astype(np.float32))
    for sched in ["merge_path", "thread_mapped", "warp_mapped", "block_mapped", "group_mapped", "nonzero_split"]:
        y, _ = _run(lb, a, f["x"].astype(np.float32), sched)
        assert np.array_equal(y, f["y"]), sched


@pytest.mark.parametrize("shape", [(128, 16), (256, 8), (256, 16), (384, 8), (512, 8)])
def test_merge_path_shapes_powerlaw_4k(lb, orc, shape):
    a = workload("powerlaw_4k")
    x = vec(a.n, 101)
    y, _ = _run(lb, a, x, "merge_path", threads=shape[0], items_per_thread=shape[1])
    ref, scale = _ref(orc, a, x)
    mx, med = check_bound(y, ref, scale, TOL32)
    print(f"merge {shape}: max rel err {mx:.3e} median {med:.3e}")


@pytest.mark.parametrize("shape", [(128, 16), (256, 8), (256, 16), (384, 8), (512, 8)])
def test_merge_path_many_tiles_per_cta(lb, orc, shape):
    """Enough tiles that every persistent CTA cycles through all stages and both product
    buffers several times (the small matrices above give most CTAs a single tile)."""
    a = synth.powerlaw_csr(300_000, 300_000, 6_000_000, 1.4, 50_000, seed=33)
    x = vec(a.n, 110)
    y, plan = _run(lb, a, x, "merge_path", threads=shape[0], items_per_thread=shape[1])
    assert plan.info()["num_tiles"] > 1000  # several tiles for every resident CTA
    ref, scale = _ref(orc, a, x)
    check_bound(y, ref, scale, TOL32)


@pytest.mark.parametrize("sched,tune", [
    ("thread_mapped", {}), ("warp_mapped", {}), ("block_mapped", {"threads": 128}), ("block_mapped", {"threads": 256}),
    ("group_mapped", {"group_size": 4}), ("group_mapped", {"group_size": 8}), ("group_mapped", {"group_size": 16}),
    ("group_mapped", {"group_size": 32}),
])
def test_mapped_schedules_powerlaw_4k(lb, orc, sched, tune):
    a = workload("powerlaw_4k")
    x = vec(a.n, 102)
    y, plan = _run(lb, a, x, sched, **tune)
    assert plan.info()["schedule"] == sched
    ref, scale = _ref(orc, a, x)
    check_bound(y, ref, scale, TOL32)


@pytest.mark.parametrize("sched", ["merge_path", "thread_mapped", "warp_mapped", "block_mapped", "group_mapped", "nonzero_split"])
def test_exact_special_cases(lb, sched):
    rng = np.random.default_rng(5)
    n = 3000
    x = vec(n, 103)
    eye = synth.from_dense(np.eye(n, dtype=np.float32))
    y, _ = _run(lb, eye, x, sched)
    assert np.array_equal(y, x)
    d = synth.uniform_pm1(rng, n)
    d[d == 0] = 0.25
    dg = synth.CSR(n, n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), d)
    y, _ = _run(lb, dg, x, sched)
    assert np.array_equal(y, d * x)  # one rounding of the exact product
    p = rng.permutation(n).astype(np.int32)
    pm = synth.CSR(n, n, np.arange(n + 1, dtype=np.int32), p, np.ones(n, np.float32))
    y, _ = _run(lb, pm, x, sched)
    assert np.array_equal(y, x[p])


@pytest.mark.parametrize("sched", ["merge_path", "thread_mapped", "warp_mapped", "block_mapped", "group_mapped", "nonzero_split"])
def test_integer_values_bit_exact(lb, orc, sched):
    rng = np.random.default_rng(6)
    a = synth.powerlaw_csr(20_000, 20_000, 300_000, 1.3, 20_000, seed=31)
    a.values = rng.integers(-8, 9, size=a.nnz).astype(np.float32)
    x = rng.integers(-8, 9, size=a.n).astype(np.float32)
    y, _ = _run(lb, a, x, sched)
    ref = orc.spmv(a.row_offsets, a.col_idx, a.values, x)
    assert np.abs(ref).max() < 2**24
    assert np.array_equal(y.astype(np.float64), ref)


def test_long_rows_spanning_many_tiles(lb, orc):
    n = 1_200_000
    rng = np.random.default_rng(7)
    lengths = np.array([5, 1_000_000, 0, 7, 300_000, 1, 0, 0, 2])
    a = synth.csr_from_row_lengths(rng, n, lengths)
    x = vec(n, 104)
    ref, scale = _ref(orc, a, x)
    for shape in [(256, 8), (128, 16), (512, 8)]:
        y, plan = _run(lb, a, x, "merge_path", threads=shape[0], items_per_thread=shape[1])
        assert plan.info()["num_tiles"] > 100
        check_bound(y, ref, scale, TOL32)
    # A single row holding every nonzero.
    one = synth.csr_from_row_lengths(rng, n, np.array([n]))
    ref1, sc1 = _ref(orc, one, x)
    y1, _ = _run(lb, one, x, "merge_path")
    check_bound(y1, ref1, sc1, TOL32)


def test_empty_rows_and_no_nonzeros(lb, orc):
    rng = np.random.default_rng(8)
    lengths = np.where(rng.random(40_000) < 0.7, 0, rng.integers(1, 60, 40_000))
    a = synth.csr_from_row_lengths(rng, 5000, lengths)
    x = vec(a.n, 105)
    ref, scale = _ref(orc, a, x)
    for sched in ["merge_path", "thread_mapped", "warp_mapped", "block_mapped", "group_mapped", "nonzero_split"]:
        y, _ = _run(lb, a, x, sched)
        check_bound(y, ref, scale, TOL32)
        assert np.all(y[lengths == 0] == 0)
    empty = synth.CSR(777, 10, np.zeros(778, np.int32), np.zeros(0, np.int32), np.zeros(0, np.float32))
    y = torch.full((777,), 5.0, device="cuda")
    lb.spmv(dev(empty.row_offsets), dev(empty.col_idx), dev(empty.values), dev(vec(10, 1)), out=y)
    plan = lb.Plan(dev(empty.row_offsets), 10, 0, schedule="merge_path")
    y2 = plan.spmv(dev(empty.col_idx), dev(empty.values), dev(vec(10, 1)))
    torch.cuda.synchronize()
    assert torch.all(y == 0) and torch.all(y2 == 0)


def test_unaligned_pointers(lb, orc):
    """Sliced views put every array at an odd element offset (not 16-byte aligned)."""
    a = workload("powerlaw_4k")
    x = vec(a.n, 106)
    ref, scale = _ref(orc, a, x)
    for off in (1, 2, 3):
        ro_b = dev(np.concatenate([np.zeros(off, np.int32), a.row_offsets]))[off:]
        ci_b = dev(np.concatenate([np.zeros(off, np.int32), a.col_idx]))[off:]
        for dtype in (torch.float32, torch.bfloat16):
            v_b = dev(np.concatenate([np.zeros(off, np.float32), a.values]), dtype)[off:]
            x_b = dev(np.concatenate([np.zeros(off, np.float32), x]))[off:]
            y_b = torch.zeros(a.m + off, device="cuda")[off:]
            lb.spmv(ro_b, ci_b, v_b, x_b, out=y_b)
            plan = lb.Plan(ro_b, a.n, a.nnz, schedule="merge_path")
            y_p = plan.spmv(ci_b, v_b, x_b)
            torch.cuda.synchronize()
            if dtype == torch.float32:
                check_bound(y_b.cpu().numpy(), ref, scale, TOL32)
                check_bound(y_p.cpu().numpy(), ref, scale, TOL32)
            else:
                r16, s16 = _ref(orc, a, x, rounded(a.values, dtype))
                check_bound(y_b.cpu().numpy(), r16, s16, TOL32)
                check_bound(y_p.cpu().numpy(), r16, s16, TOL32)


def test_auto_rule_and_plain_call(lb, orc):
    small = synth.powerlaw_csr(300, 300, 2000, 1.5, 300, seed=41)
    ro, ci, v = to_dev(small)
    plan = lb.Plan(ro, small.n, small.nnz)
    assert plan.info()["schedule"] in ("thread_mapped", "group_mapped")
    big = workload("powerlaw_4k")
    rb, cb, vb = to_dev(big)
    assert lb.Plan(rb, big.n, big.nnz).info()["schedule"] == "merge_path"
    for a, (r, c, vv) in ((small, (ro, ci, v)), (big, (rb, cb, vb))):
        x = vec(a.n, 107)
        y = lb.spmv(r, c, vv, dev(x))
        torch.cuda.synchronize()
        ref, scale = _ref(orc, a, x)
        check_bound(y.cpu().numpy(), ref, scale, TOL32)


@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float16])
@pytest.mark.parametrize("sched", ["merge_path", "thread_mapped", "warp_mapped", "block_mapped", "nonzero_split"])
def test_half_precision_values(lb, orc, dtype, sched):
    a = workload("powerlaw_4k")
    x = vec(a.n, 108)
    y, _ = _run(lb, a, x, sched, dtype)
    ref32, s32 = _ref(orc, a, x)
    mx, med = check_bound(y, ref32, s32, TOL16)
    r16, s16 = _ref(orc, a, x, rounded(a.values, dtype))
    check_bound(y, r16, s16, TOL32)
    print(f"{dtype} {sched}: vs FP32 values max {mx:.3e} median {med:.3e}")


def test_deterministic(lb):
    a = workload("powerlaw_4k")
    ro, ci, v = to_dev(a)
    x = dev(vec(a.n, 109))
    for sched in ["merge_path", "thread_mapped", "warp_mapped", "block_mapped", "group_mapped", "nonzero_split"]:
        plan = lb.Plan(ro, a.n, a.nnz, schedule=sched)
        y1 = plan.spmv(ci, v, x)
        y2 = plan.spmv(ci, v, x)
        torch.cuda.synchronize()
        assert torch.equal(y1, y2), sched


def test_validate_csr(lb):
    a = synth.powerlaw_csr(2000, 1500, 20_000, 1.4, 1500, seed=51)
    ro, ci = a.row_offsets.copy(), a.col_idx.copy()
    assert lb.validate_csr(dev(ro), dev(ci), a.n) == 0
    bad = ro.copy()
    bad[0] = 1
    assert lb.validate_csr(dev(bad), dev(ci), a.n) & 1
    bad = ro.copy()
    bad[10] = bad[11] + 5
    assert lb.validate_csr(dev(bad), dev(ci), a.n) & 2
    bad = ro.copy()
    bad[-1] -= 1
    assert lb.validate_csr(dev(bad), dev(ci), a.n) & 4
    badc = ci.copy()
    last = int(ro[int(np.argmax(np.diff(ro) >= 1)) + 1]) - 1  # last entry of a non-empty row
    badc[last] = a.n
    assert lb.validate_csr(dev(ro), dev(badc), a.n) == 8
    badc = ci.copy()
    r = int(np.argmax(np.diff(ro) >= 2))
    badc[ro[r]], badc[ro[r] + 1] = badc[ro[r] + 1], badc[ro[r]]
    assert lb.validate_csr(dev(ro), dev(badc), a.n) == 16
    assert lb.validate_csr(dev(ro), dev(badc), a.n, check_sorted=False) == 0
    # Rows longer than 32 entries are walked by a whole warp: errors deep inside one.
    r = int(np.argmax(np.diff(ro) >= 64))
    assert ro[r + 1] - ro[r] >= 64
    badc = ci.copy()
    badc[ro[r + 1] - 1] = a.n  # out of range at the row's end, still increasing
    assert lb.validate_csr(dev(ro), dev(badc), a.n) == 8
    badc = ci.copy()
    badc[ro[r] + 40] = -1  # out of range and below its predecessor
    assert lb.validate_csr(dev(ro), dev(badc), a.n) == 8 | 16
    badc = ci.copy()
    badc[ro[r] + 33], badc[ro[r] + 34] = badc[ro[r] + 34], badc[ro[r] + 33]
    assert lb.validate_csr(dev(ro), dev(badc), a.n) == 16
    badc = ci.copy()
    badc[ro[r + 1] - 1] = badc[ro[r + 1] - 2]  # a repeated column at the row's end
    assert lb.validate_csr(dev(ro), dev(badc), a.n) == 16


# ------------------------------------------------------------------ full sizes


def test_full_size_powerlaw_4m(lb, orc):
    """The large power-law configuration in the benchmark's launch shape."""
    a = workload("powerlaw_4m")
    x = vec(a.n, 1)
    ro, ci, v = to_dev(a)
    plan = lb.Plan(ro, a.n, a.nnz, schedule="merge_path")
    y1 = plan.spmv(ci, v, dev(x))
    y2 = plan.spmv(ci, v, dev(x))
    torch.cuda.synchronize()
    assert torch.equal(y1, y2)
    ref, scale = _ref(orc, a, x)
    mx, med = check_bound(y1.cpu().numpy(), ref, scale, TOL32)
    print(f"powerlaw_4m FP32: max rel err {mx:.3e} median {med:.3e}")
    assert lb.device_error() == 0
    y3 = lb.Plan(ro, a.n, a.nnz, schedule="nonzero_split").spmv(ci, v, dev(x))
    torch.cuda.synchronize()
    check_bound(y3.cpu().numpy(), ref, scale, TOL32)


def test_full_size_stencil(lb, orc):
    a = workload("stencil7_160")
    x = vec(a.n, 2)
    y, _ = _run(lb, a, x)
    ref, scale = _ref(orc, a, x)
    check_bound(y, ref, scale, TOL32)
    ai = synth.stencil7_csr(160, seed=3, integer_values=True)
    xi = np.random.default_rng(9).integers(-8, 9, size=ai.n).astype(np.float32)
    yi, _ = _run(lb, ai, xi)
    assert np.array_equal(yi.astype(np.float64), orc.spmv(ai.row_offsets, ai.col_idx, ai.values, xi))


def _tuned_shape(a, dtype_name):
    """The merge-path shape the shipped autotuner table records for this matrix's class."""
    from paper_2212_08964_gb300 import autotune

    cfg = autotune.choose(a.row_offsets, autotune.default_table(), dtype_name)
    if cfg["schedule"] != "merge_path":
        return None
    return cfg["threads"], cfg["items_per_thread"]


@pytest.mark.parametrize("shape", ["default", "tuned"])
def test_full_size_powerlaw_8m_f32(lb, orc, shape):
    """The mixed-precision configuration's FP32-value run (the baseline its BF16/FP16 errors
    are compared with): 1e-5 * sum|a||x| per row in the default and the tuned launch shape."""
    a = workload("powerlaw_8m")
    x = vec(a.n, 6)
    tune = {}
    if shape == "tuned":
        ts = _tuned_shape(a, "f32")
        if ts is not None:
            tune = {"threads": ts[0], "items_per_thread": ts[1]}
    y, _ = _run(lb, a, x, "merge_path", torch.float32, **tune)
    ref, scale = _ref(orc, a, x)
    mx, med = check_bound(y, ref, scale, TOL32)
    print(f"powerlaw_8m FP32 ({shape} {tune}): max {mx:.3e} median {med:.3e}")
    assert lb.device_error() == 0


@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float16])
@pytest.mark.parametrize("shape", [(256, 8), (128, 16)])
def test_full_size_powerlaw_8m_half(lb, orc, dtype, shape):
    """BF16/FP16 values at full size, in the default shape and the narrow-value tuned one."""
    a = workload("powerlaw_8m")
    x = vec(a.n, 6)
    y, _ = _run(lb, a, x, "merge_path", dtype, threads=shape[0], items_per_thread=shape[1])
    ref32, s32 = _ref(orc, a, x)
    mx, med = check_bound(y, ref32, s32, TOL16)
    r16, s16 = _ref(orc, a, x, rounded(a.values, dtype))
    mx16, med16 = check_bound(y, r16, s16, TOL32)
    print(f"powerlaw_8m {dtype} {shape}: vs FP32 values max {mx:.3e} median {med:.3e}; "
          f"vs rounded values max {mx16:.3e} median {med16:.3e}")


@pytest.mark.parametrize("name", ["powerlaw_4k", "stencil", "empty_rows", "few_columns"])
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
@pytest.mark.parametrize("bucket_shift", [None, "10"])
def test_csc_input(lb, orc, monkeypatch, name, dtype, bucket_shift):
    """y = A x from A in CSC form (the oracle's stable transpose of the CSR matrix): within
    tolerance of the oracle, and bit-equal to the CSR forward on the same matrix, whose
    partition, products and summation order it shares."""
    if bucket_shift:
        monkeypatch.setenv("LBSPMV_VALUE_BUCKET_SHIFT", bucket_shift)
    rng = np.random.default_rng(17)
    if name == "powerlaw_4k":
        a = workload("powerlaw_4k")
    elif name == "stencil":
        a = synth.stencil7_csr(9, seed=3)
    elif name == "empty_rows":
        lengths = rng.integers(0, 4, 5000)
        lengths[:100] = 0
        lengths[-300:] = 0
        a = synth.csr_from_row_lengths(rng, 700, lengths)
    else:  # many rows over few columns: long columns, and empty ones
        a = synth.csr_from_row_lengths(rng, 40, rng.integers(0, 12, 20000))
    co, ri, perm = orc.transpose(a.row_offsets, a.col_idx, a.n)
    vals = a.values if dtype == torch.float32 else rounded(a.values, dtype)
    v_csc = dev(a.values[perm]).to(dtype)
    x = vec(a.n, 71)
    cp = lb.CscPlan(dev(co), dev(ri), a.m)
    y = cp.spmv(v_csc, dev(x))
    plan = lb.Plan(dev(a.row_offsets), a.n, a.nnz, schedule="merge_path")
    y_csr = plan.spmv(dev(a.col_idx), dev(a.values).to(dtype), dev(x))
    torch.cuda.synchronize()
    check_bound(y.cpu().numpy(), orc.spmv(a.row_offsets, a.col_idx, vals, x),
                orc.row_absdot(a.row_offsets, a.col_idx, vals, x), TOL32)
    assert torch.equal(y, y_csr)
    assert lb.device_error() == 0


@pytest.mark.parametrize("name", ["powerlaw_4k", "stencil", "empty_rows"])
def test_coo_input(lb, orc, name):
    """COO (row-sorted) to CSR offsets bit-exact against counting; the COO matrix then runs
    through the plain entry point; unsorted and out-of-range rows are reported."""
    if name == "powerlaw_4k":
        a = workload("powerlaw_4k")
    elif name == "stencil":
        a = synth.stencil7_csr(9, seed=3)
    else:
        rng = np.random.default_rng(3)
        lengths = rng.integers(0, 4, 5000)
        lengths[:100] = 0
        lengths[-300:] = 0
        a = synth.csr_from_row_lengths(rng, 700, lengths)
    rows = np.repeat(np.arange(a.m, dtype=np.int32), a.row_lengths())
    ro, status = lb.coo_row_offsets(dev(rows), a.m)
    assert status == 0
    counted = np.array([np.count_nonzero(rows < r) for r in range(a.m + 1)], dtype=np.int32)
    assert np.array_equal(ro.cpu().numpy(), counted)
    assert np.array_equal(counted, a.row_offsets)
    x = vec(a.n, 61)
    y = lb.spmv(ro, dev(a.col_idx), dev(a.values), dev(x), n=a.n)
    torch.cuda.synchronize()
    check_bound(y.cpu().numpy(), orc.spmv(a.row_offsets, a.col_idx, a.values, x),
                orc.row_absdot(a.row_offsets, a.col_idx, a.values, x), TOL32)
    if rows.size > 2:
        bad = rows.copy()
        bad[1], bad[-1] = bad[-1], bad[1]
        assert lb.coo_row_offsets(dev(bad), a.m)[1] & 2
        bad = rows.copy()
        bad[-1] = a.m
        assert lb.coo_row_offsets(dev(bad), a.m)[1] & 1


def test_calibrate(lb):
    """The measured ceilings are positive and in the range this part can reach."""
    c = lb.calibrate()
    assert 1e10 < c["gathers_per_s"] < 5e12
    assert 100 < c["read_GBps"] < 20000
    assert 100 < c["copy_GBps"] < 20000


def test_one_row_spanning_thousands_of_tiles(lb, orc):
    """A 5M-entry row between two short rows: its partial sums are carried out of ~2500 tiles
    and combined by one fixup run."""
    rng = np.random.default_rng(123)
    a = synth.csr_from_row_lengths(rng, 6_000_000, np.array([3, 5_000_000, 2]))
    x = vec(a.n, 124)
    ro, ci, v = to_dev(a)
    plan = lb.Plan(ro, a.n, a.nnz, schedule="merge_path")
    assert plan.info()["num_tiles"] > 2000
    y = plan.spmv(ci, v, dev(x))
    y1 = lb.spmv(ro, ci, v, dev(x))
    y2 = lb.Plan(ro, a.n, a.nnz, schedule="nonzero_split").spmv(ci, v, dev(x))
    torch.cuda.synchronize()
    scale = orc.row_absdot(a.row_offsets, a.col_idx, a.values, x)
    ref = orc.spmv(a.row_offsets, a.col_idx, a.values, x)
    check_bound(y.cpu().numpy(), ref, scale, TOL32)
    check_bound(y2.cpu().numpy(), ref, scale, TOL32)
    assert torch.equal(y, y1)
