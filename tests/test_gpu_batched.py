"""Batched SpMV (many matrices, one launch) vs per-matrix oracle runs, under both batch
schedules (the global merge path, and thread-mapped rows with long rows summed by the warp);
the global partition bit-exact against the block-diagonal counting definition; CUDA-graph
replay."""
import numpy as np
import pytest
import torch

from gpu_helpers import check_bound, dev, vec, workload
from paper_2212_08964_gb300 import synth

pytestmark = pytest.mark.gpu

TOL32 = 1e-5


def _batch_with_degenerates():
    """Small batch including empty matrices, matrices without nonzeros and one-row matrices."""
    rng = np.random.default_rng(21)
    mats = []
    for i in range(40):
        kind = i % 8
        if kind == 0:
            mats.append(synth.CSR(0, int(rng.integers(0, 5)), np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0, np.float32)))
        elif kind == 1:
            m = int(rng.integers(1, 30))
            mats.append(synth.CSR(m, 7, np.zeros(m + 1, np.int32), np.zeros(0, np.int32), np.zeros(0, np.float32)))
        elif kind == 2:
            n = int(rng.integers(1, 5000))
            mats.append(synth.csr_from_row_lengths(rng, n, np.array([n])))
        else:
            m = int(rng.integers(1, 3000))
            n = int(rng.integers(1, 3000))
            mats.append(synth.csr_from_row_lengths(rng, n, np.minimum(rng.integers(0, 80, m), n)))
    return synth.BatchedCSR(
        np.array([a.m for a in mats], np.int64), np.array([a.n for a in mats], np.int64),
        np.array([a.nnz for a in mats], np.int64), np.concatenate([a.row_offsets for a in mats]),
        np.concatenate([a.col_idx for a in mats]), np.concatenate([a.values for a in mats]))


def _plan(lb, b, **tune):
    return lb.BatchedPlan(b.ms, b.ns, b.nnzs, dev(b.row_offsets), **tune)


@pytest.mark.parametrize("shape", [(256, 8), (128, 16), (512, 8)])
def test_batched_partition_bit_exact(lb, orc, shape):
    b = _batch_with_degenerates()
    plan = _plan(lb, b, threads=shape[0], items_per_thread=shape[1])
    tr, tn = plan.partition()
    ro_g = orc.block_diagonal_offsets(b.ms, b.nnzs, b.row_offsets)
    T = plan.info()["tile_items"]
    assert T == 32 * shape[1] - 8  # warp tiles of the merge-path kernel
    otr, otn = orc.partition(ro_g, T)
    assert np.array_equal(tr, otr) and np.array_equal(tn, otn)


@pytest.mark.parametrize("schedule", ["merge_path", "thread_mapped"])
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16, torch.float16])
def test_batched_vs_oracle(lb, orc, dtype, schedule):
    b = _batch_with_degenerates()
    x = vec(int(b.ns.sum()), 301)
    plan = _plan(lb, b, schedule=schedule)
    assert plan.info()["schedule"] == schedule
    y = plan.spmv(dev(b.col_idx), dev(b.values, dtype), dev(x))
    torch.cuda.synchronize()
    vals = b.values if dtype == torch.float32 else torch.from_numpy(b.values).to(dtype).float().numpy()
    bb = synth.BatchedCSR(b.ms, b.ns, b.nnzs, b.row_offsets, b.col_idx, vals)
    ref = orc.batched_spmv(bb, x)
    scale = orc.batched_row_absdot(bb, x)
    check_bound(y.cpu().numpy(), ref, scale, TOL32)


@pytest.mark.parametrize("schedule", ["merge_path", "thread_mapped"])
def test_batched_cuda_graph_replay(lb, orc, schedule):
    b = workload("batched_4096", 0.05)
    x = vec(int(b.ns.sum()), 302)
    plan = _plan(lb, b, schedule=schedule)
    ci, v, xd = dev(b.col_idx), dev(b.values), dev(x)
    y = torch.empty(int(b.ms.sum()), device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        plan.spmv(ci, v, xd, out=y)  # warm-up outside capture (sets kernel attributes)
    torch.cuda.current_stream().wait_stream(s)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        plan.spmv(ci, v, xd, out=y)
    y.zero_()
    graph.replay()
    torch.cuda.synchronize()
    ref = orc.batched_spmv(b, x)
    check_bound(y.cpu().numpy(), ref, orc.batched_row_absdot(b, x), TOL32)
    y1 = y.clone()
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(y, y1)


@pytest.mark.parametrize("schedule", ["merge_path", "thread_mapped"])
def test_full_size_batched_4096(lb, orc, schedule):
    b = workload("batched_4096")
    x = vec(int(b.ns.sum()), 5)
    plan = _plan(lb, b, schedule=schedule)
    y = plan.spmv(dev(b.col_idx), dev(b.values), dev(x))
    torch.cuda.synchronize()
    ref = orc.batched_spmv(b, x)
    mx, med = check_bound(y.cpu().numpy(), ref, orc.batched_row_absdot(b, x), TOL32)
    print(f"batched_4096 {schedule}: max rel err {mx:.3e} median {med:.3e}")
    ro_g = orc.block_diagonal_offsets(b.ms, b.nnzs, b.row_offsets)
    tr, tn = plan.partition()
    otr, otn = orc.partition(ro_g, plan.info()["tile_items"])
    assert np.array_equal(tr, otr) and np.array_equal(tn, otn)


def test_thread_mapped_batch_long_rows_and_single_matrix(lb, orc):
    """Rows far longer than the warp's share (summed by the whole warp), next to rows of one
    nonzero and empty rows, in a batch of one matrix and in a batch of many."""
    rng = np.random.default_rng(23)
    lens = np.concatenate([rng.integers(0, 3, 200), [5000, 33, 9, 8, 0, 70000], rng.integers(0, 3, 100)])
    one = synth.csr_from_row_lengths(rng, 80_000, lens)
    for mats in ([one], [one, synth.csr_from_row_lengths(rng, 50, rng.integers(0, 12, 700)), one]):
        b = synth.BatchedCSR(
            np.array([a.m for a in mats], np.int64), np.array([a.n for a in mats], np.int64),
            np.array([a.nnz for a in mats], np.int64), np.concatenate([a.row_offsets for a in mats]),
            np.concatenate([a.col_idx for a in mats]), np.concatenate([a.values for a in mats]))
        x = vec(int(b.ns.sum()), 303)
        plan = _plan(lb, b, schedule="thread_mapped")
        y = plan.spmv(dev(b.col_idx), dev(b.values), dev(x))
        torch.cuda.synchronize()
        check_bound(y.cpu().numpy(), orc.batched_spmv(b, x), orc.batched_row_absdot(b, x), TOL32)


@pytest.mark.parametrize("schedule", ["merge_path", "thread_mapped"])
def test_batched_grid(lb, orc, schedule):
    """The batch of 2-D Laplacians of uneven size (regular short rows) under both schedules."""
    b = workload("batched_grid_1024", 0.1)
    x = vec(int(b.ns.sum()), 304)
    plan = _plan(lb, b, schedule=schedule)
    y = plan.spmv(dev(b.col_idx), dev(b.values), dev(x))
    torch.cuda.synchronize()
    check_bound(y.cpu().numpy(), orc.batched_spmv(b, x), orc.batched_row_absdot(b, x), TOL32)
