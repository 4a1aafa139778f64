"""SSSP and BFS on the GPU against the Dijkstra oracle: integer weights (exact in FP32 sums)
and unit weights (BFS levels) compared exactly; real weights within the rounding of an FP32
path sum; unreachable vertices, sources without out-edges, self loops, long chains."""
import numpy as np
import pytest
import torch

from gpu_helpers import dev, workload
from paper_2212_08964_gb300 import synth

pytestmark = pytest.mark.gpu


def _graph(name):
    rng = np.random.default_rng(91)
    if name == "powerlaw_4k":
        return workload("powerlaw_4k")
    if name == "sparse_random":  # many vertices unreachable, some without out-edges
        return synth.csr_from_row_lengths(rng, 20000, rng.integers(0, 3, 20000))
    if name == "chain":  # 0 -> 1 -> ... -> 2999: one vertex per iteration
        n = 3000
        ro = np.arange(n + 1, dtype=np.int32).clip(max=n - 1)
        ro[-1] = n - 1
        ci = np.arange(1, n, dtype=np.int32)
        return synth.CSR(n, n, ro, ci, np.ones(n - 1, np.float32))
    if name == "self_loops":
        a = synth.csr_from_row_lengths(rng, 500, rng.integers(1, 5, 500))
        a.col_idx[a.row_offsets[:-1]] = np.arange(500, dtype=np.int32)  # first edge of each row: itself
        return a
    raise KeyError(name)


@pytest.mark.parametrize("name", ["powerlaw_4k", "sparse_random", "chain", "self_loops"])
@pytest.mark.parametrize("kind", ["integer", "unit", "real"])
def test_sssp_vs_oracle(lb, orc, name, kind):
    a = _graph(name)
    rng = np.random.default_rng(92)
    if kind == "integer":
        w = rng.integers(1, 100, a.nnz).astype(np.float32)
    elif kind == "real":
        w = rng.uniform(0.01, 1.0, a.nnz).astype(np.float32)
    else:
        w = None
    for src in (0, a.m // 2, a.m - 1):
        dist, iters = lb.sssp(dev(a.row_offsets), dev(a.col_idx), None if w is None else dev(w), src)
        torch.cuda.synchronize()
        ref = orc.sssp(a.row_offsets, a.col_idx, None if w is None else w.astype(np.float64), src)
        got = dist.cpu().numpy().astype(np.float64)
        assert np.array_equal(np.isinf(got), np.isinf(ref))
        fin = np.isfinite(ref)
        if kind == "real":
            # The minimum over paths of FP32 path sums: one rounding per edge of the path, so
            # within (hops + 1) * 2^-23 of the distance (hops from the BFS levels).
            hops = orc.sssp(a.row_offsets, a.col_idx, None, src)[fin]
            bound = (hops + 1) * 2.0**-23 * ref[fin] + 1e-12
            assert np.all(np.abs(got[fin] - ref[fin]) <= bound)
        else:
            assert np.array_equal(got[fin], ref[fin])
        assert iters >= 1
        if name == "chain" and src == 0:
            assert iters >= a.m - 1


def test_sssp_large_powerlaw(lb, orc):
    """The quarter-size power-law matrix as a graph (1M vertices, 16M edges), integer weights."""
    a = workload("powerlaw_4m", 0.25)
    w = np.random.default_rng(93).integers(1, 100, a.nnz).astype(np.float32)
    dist, iters = lb.sssp(dev(a.row_offsets), dev(a.col_idx), dev(w), 0)
    torch.cuda.synchronize()
    ref = orc.sssp(a.row_offsets, a.col_idx, w.astype(np.float64), 0)
    got = dist.cpu().numpy().astype(np.float64)
    assert np.array_equal(np.isinf(got), np.isinf(ref))
    fin = np.isfinite(ref)
    assert np.array_equal(got[fin], ref[fin])
    print(f"sssp powerlaw 1M: {iters} iterations, {int(fin.sum())} reachable")
