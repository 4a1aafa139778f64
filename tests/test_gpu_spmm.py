"""SpMM C = A B on the GPU against the FP64 oracle: every entry within 1e-5 * sum_k |a||b|
(BF16/FP16 values against the oracle on the rounded values); columns of B from 1 to 160 (the
wide warp kernel at 8 and 16 columns, the quad warp kernel up to 4, the block kernel with one
and two column passes, vector and scalar paths); rows spanning many tiles, empty rows, empty
matrices; determinism."""
import numpy as np
import pytest
import torch

from gpu_helpers import dev, rounded, to_dev, workload
from paper_2212_08964_gb300 import synth

pytestmark = pytest.mark.gpu

TOL32 = 1e-5


def _long_rows():
    """Power-law body plus rows of 5k-20k nonzeros (each spans 20-80 warp tiles of 248
    items, more than one 32-tile probe of the fixup) and runs of empty rows."""
    rng = np.random.default_rng(71)
    lengths = rng.integers(0, 12, 6000)
    lengths[[5, 6, 7, 3000, 5999]] = [20000, 0, 9000, 5000, 12000]
    lengths[100:180] = 0
    return synth.csr_from_row_lengths(rng, 30000, lengths)


def _cases():
    return {"powerlaw_4k": workload("powerlaw_4k"), "long_rows": _long_rows(),
            "stencil": synth.stencil7_csr(10, seed=3)}


def _check(C, ref, scale, tol):
    err = np.abs(C.astype(np.float64) - ref)
    bad = err > tol * scale
    assert not bad.any(), f"{int(bad.sum())} entries exceed; worst {float((err / np.maximum(scale, 1e-300)).max()):.3e}"


@pytest.mark.parametrize("name", ["powerlaw_4k", "long_rows", "stencil"])
@pytest.mark.parametrize("kc", [1, 3, 4, 8, 12, 16, 17, 24, 32, 64, 160])
def test_spmm_vs_oracle(lb, orc, name, kc):
    a = _cases()[name]
    ro, ci, v = to_dev(a)
    plan = lb.Plan(ro, a.n, a.nnz, schedule="merge_path")
    B = np.random.default_rng(kc).uniform(-1, 1, (a.n, kc)).astype(np.float32)
    C = plan.spmm(ci, v, dev(B))
    torch.cuda.synchronize()
    ref = orc.spmm(a.row_offsets, a.col_idx, a.values, B)
    _check(C.cpu().numpy(), ref, orc.spmm_absdot(a.row_offsets, a.col_idx, a.values, B), TOL32)
    C2 = plan.spmm(ci, v, dev(B))
    torch.cuda.synchronize()
    assert torch.equal(C, C2)
    assert lb.device_error() == 0


@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float16])
@pytest.mark.parametrize("kc", [4, 8, 16, 24])
def test_spmm_half_values(lb, orc, dtype, kc):
    """16-bit values through every SpMM kernel: quad warp (4), wide warp (8, 16), block (24)."""
    a = _long_rows()
    ro, ci, v = to_dev(a, dtype)
    plan = lb.Plan(ro, a.n, a.nnz, schedule="merge_path")
    B = np.random.default_rng(5).uniform(-1, 1, (a.n, kc)).astype(np.float32)
    C = plan.spmm(ci, v, dev(B))
    torch.cuda.synchronize()
    vals = rounded(a.values, dtype)
    _check(C.cpu().numpy(), orc.spmm(a.row_offsets, a.col_idx, vals, B),
           orc.spmm_absdot(a.row_offsets, a.col_idx, vals, B), TOL32)


def test_spmm_unaligned_and_degenerate(lb, orc):
    a = workload("powerlaw_4k")
    ro, ci, v = to_dev(a)
    plan = lb.Plan(ro, a.n, a.nnz, schedule="merge_path")
    kc = 8
    B = np.random.default_rng(9).uniform(-1, 1, (a.n, kc)).astype(np.float32)
    Bbuf = torch.zeros(a.n * kc + 1, device="cuda")
    Bbuf[1:] = dev(B.reshape(-1))
    Bv = Bbuf[1:].view(a.n, kc)  # 4-byte offset: the scalar path
    C = plan.spmm(ci, v, Bv)
    torch.cuda.synchronize()
    _check(C.cpu().numpy(), orc.spmm(a.row_offsets, a.col_idx, a.values, B),
           orc.spmm_absdot(a.row_offsets, a.col_idx, a.values, B), TOL32)
    # B and C 16 bytes off a 32-byte boundary: kc = 8 leaves the wide kernel for the block
    # kernel, kc = 4 keeps the quad warp kernel's vector path; 4 bytes off, kc = 4 takes its
    # scalar path.
    for kc2, off in [(8, 4), (4, 4), (4, 1)]:
        B2 = np.random.default_rng(10 + kc2 + off).uniform(-1, 1, (a.n, kc2)).astype(np.float32)
        Bb = torch.zeros(a.n * kc2 + off, device="cuda")
        Bb[off:] = dev(B2.reshape(-1))
        Cb = torch.zeros(a.m * kc2 + off, device="cuda")
        plan.spmm(ci, v, Bb[off:].view(a.n, kc2), out=Cb[off:].view(a.m, kc2))
        torch.cuda.synchronize()
        _check(Cb[off:].view(a.m, kc2).cpu().numpy(), orc.spmm(a.row_offsets, a.col_idx, a.values, B2),
               orc.spmm_absdot(a.row_offsets, a.col_idx, a.values, B2), TOL32)
    # No nonzeros: C = 0.  No columns: nothing to do.
    e = synth.CSR(5, 7, np.zeros(6, np.int32), np.zeros(0, np.int32), np.zeros(0, np.float32))
    pe = lb.Plan(dev(e.row_offsets), 7, 0, schedule="merge_path")
    Ce = torch.full((5, 3), float("nan"), device="cuda")
    pe.spmm(torch.zeros(0, dtype=torch.int32, device="cuda"), torch.zeros(0, device="cuda"),
            torch.zeros(7, 3, device="cuda"), out=Ce)
    torch.cuda.synchronize()
    assert (Ce == 0).all()


def test_spmm_large_powerlaw(lb, orc):
    """A quarter-size power-law matrix (1M rows, 16M nonzeros) with 8 columns."""
    a = workload("powerlaw_4m", 0.25)
    ro, ci, v = to_dev(a)
    plan = lb.Plan(ro, a.n, a.nnz, schedule="merge_path")
    B = np.random.default_rng(8).uniform(-1, 1, (a.n, 8)).astype(np.float32)
    C = plan.spmm(ci, v, dev(B))
    torch.cuda.synchronize()
    _check(C.cpu().numpy(), orc.spmm(a.row_offsets, a.col_idx, a.values, B),
           orc.spmm_absdot(a.row_offsets, a.col_idx, a.values, B), TOL32)


@pytest.mark.parametrize("shape,kc", [((128, 16), 2), ((128, 16), 4), ((512, 8), 3), ((128, 16), 8), ((128, 16), 12)])
def test_spmm_other_plan_shapes(lb, orc, shape, kc):
    """Plans of other merge-path shapes.  kc <= 4 runs over 248-item warp tiles: a partition of
    its own, built on the first call, for plans whose warp tiles differ (128 x 16), else the
    plan's (512 x 8).  Wider B runs over the plan's block tiles."""
    a = _long_rows()
    ro, ci, v = to_dev(a)
    plan = lb.Plan(ro, a.n, a.nnz, schedule="merge_path", threads=shape[0], items_per_thread=shape[1])
    B = np.random.default_rng(kc + 100).uniform(-1, 1, (a.n, kc)).astype(np.float32)
    for _ in range(2):
        C = plan.spmm(ci, v, dev(B))
        torch.cuda.synchronize()
        _check(C.cpu().numpy(), orc.spmm(a.row_offsets, a.col_idx, a.values, B),
               orc.spmm_absdot(a.row_offsets, a.col_idx, a.values, B), TOL32)
    assert lb.device_error() == 0
