"""The seeded generators produce well-formed CSR with the stated shapes and laws."""
import numpy as np

from paper_2212_08964_gb300 import synth


def _check_csr(a: synth.CSR):
    ro = a.row_offsets.astype(np.int64)
    assert ro[0] == 0 and ro[-1] == a.nnz and np.all(np.diff(ro) >= 0)
    assert a.col_idx.dtype == np.int32 and a.values.dtype == np.float32
    if a.nnz:
        assert a.col_idx.min() >= 0 and a.col_idx.max() < a.n
    # Distinct and sorted within each row.
    d = np.diff(a.col_idx.astype(np.int64))
    starts = np.zeros(a.nnz, bool)
    starts[ro[:-1][np.diff(ro) > 0]] = True
    assert np.all(d[~starts[1:]] > 0)


def test_powerlaw_small_shape_and_determinism():
    a = synth.workload("powerlaw_4k")
    b = synth.workload("powerlaw_4k")
    _check_csr(a)
    assert a.m == a.n == 4096
    assert abs(a.nnz - 64_000) / 64_000 < 0.05
    assert a.row_lengths().max() <= 2048 and a.row_lengths().min() >= 1
    assert np.array_equal(a.col_idx, b.col_idx) and np.array_equal(a.values, b.values)


def test_values_exact_in_fp32_and_in_range():
    v = synth.uniform_pm1(np.random.default_rng(0), 100_000)
    assert v.min() >= -1 and v.max() <= 1
    k = v.astype(np.float64) * (1 << 23)
    assert np.array_equal(k, np.round(k))


def test_pareto_mean_solver():
    x_min = synth.solve_pareto_xmin(15.26, 1.3, 500_000)
    assert 3.6 < x_min < 3.85
    lengths = synth.pareto_row_lengths(np.random.default_rng(1), 400_000, x_min, 1.3, 500_000)
    # Heavy tail: the sample mean converges slowly, keep the check loose.
    assert 12 < lengths.mean() < 19


def test_stencil_counts():
    a = synth.stencil7_csr(6, seed=3, integer_values=True)
    _check_csr(a)
    assert a.nnz == 7 * 6**3 - 6 * 6**2
    # Integer variant: diagonal 6, off-diagonals -1, row sums 6 - (#neighbours).
    dense = np.zeros((a.m, a.n))
    rows = np.repeat(np.arange(a.m), a.row_lengths())
    dense[rows, a.col_idx] = a.values
    assert np.all(np.diag(dense) == 6)
    assert np.array_equal(dense, dense.T)


def test_batched_layout():
    b = synth.batched_powerlaw(10, 16, 512, 3000, 1.5, seed=5)
    assert len(b.row_offsets) == int(b.ms.sum() + b.count)
    assert len(b.col_idx) == int(b.nnzs.sum())
    for i in range(b.count):
        a = b.matrix(i)
        _check_csr(a)
        assert a.row_lengths().max() <= max(1, a.m // 4)


def test_lognormal_shape():
    a = synth.lognormal_csr(4096, 4096, 2.5, 1.2, seed=4)
    _check_csr(a)
    assert 15 < a.nnz / a.m < 35
