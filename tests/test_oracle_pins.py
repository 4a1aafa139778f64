"""Pins for the CPU oracle: checks against things other than the oracle itself.

* a hand-worked example (tests/golden/worked_example_4x4.txt);
* an explicit step-by-step merge of row ends and nonzeros, enumerated over every row-length
  vector with m <= 6 and nnz <= 8 and every tile size (the merge-path split, Alg.
  alg:work-oriented);
* library routines: numpy dense matvec and scipy.sparse (SpMV, transpose, A^T g);
* closed forms and special cases: identity, diagonal, permutation, integer-valued exact sums,
  the column-sum invariant sum(y) = (1^T A) x;
* central finite differences of the quadratic loss L = 1/2||Ax - t||^2, exact up to rounding;
* the tolerance scales |A| |x| and |A|^T |g| (and their batched form) against scipy;
* SpMM against dense and sparse products, SSSP against scipy's Dijkstra and a worked graph.
"""
import itertools

import numpy as np
import pytest
import scipy.sparse as sp

from golden.fixtures import load
from paper_2212_08964_gb300 import synth


def _scipy(a: synth.CSR):
    return sp.csr_matrix((a.values.astype(np.float64), a.col_idx, a.row_offsets), shape=(a.m, a.n))


# ------------------------------------------------------------------ worked example


def test_worked_example(orc):
    f = load("worked_example_4x4.txt")
    ro = f["row_offsets"].astype(np.int32)
    ci = f["col_idx"].astype(np.int32)
    v, x, g = f["values"], f["x"], f["g"]
    assert np.array_equal(orc.spmv(ro, ci, v, x), f["y"])
    for T in (3, 4):
        tr, tn = orc.partition(ro, T)
        assert np.array_equal(tr, f[f"tile_row_T{T}"])
        assert np.array_equal(tn, f[f"tile_nz_T{T}"])
    co, ri, perm = orc.transpose(ro, ci, f["n"])
    assert np.array_equal(co, f["col_offsets"])
    assert np.array_equal(ri, f["row_idx"])
    assert np.array_equal(perm, f["perm"])
    assert np.array_equal(orc.spmv_t(ro, ci, v, g, f["n"]), f["dx"])
    assert np.array_equal(orc.dvalues(ro, ci, g, x), f["dv"])


# ------------------------------------------------------------------ merge path


def _all_row_length_vectors(max_m=6, max_nnz=8):
    for m in range(1, max_m + 1):
        for lengths in itertools.product(range(max_nnz + 1), repeat=m):
            if sum(lengths) <= max_nnz:
                yield lengths


def _merge_prefix_counts(ro):
    """(rows, nonzeros) consumed before every position d = 0..W of the explicit merge."""
    import oracle

    seq = oracle.explicit_merge(ro)
    rows = np.concatenate([[0], np.cumsum([t == "R" for t, _ in seq])])
    nzs = np.concatenate([[0], np.cumsum([t == "N" for t, _ in seq])])
    return rows, nzs


def test_partition_matches_explicit_merge_bruteforce(orc):
    count = 0
    for lengths in _all_row_length_vectors():
        ro = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int32)
        m, nnz = len(lengths), int(ro[-1])
        W = m + nnz
        rows, nzs = _merge_prefix_counts(ro)
        # T = 1 cuts at every diagonal.
        tr, tn = orc.partition(ro, 1)
        assert np.array_equal(tr, rows) and np.array_equal(tn, nzs), lengths
        for T in range(2, W + 1):
            tr, tn = orc.partition(ro, T)
            d = np.minimum(np.arange(len(tr)) * T, W)
            assert len(tr) == -(-W // T) + 1
            assert np.array_equal(tr, rows[d]) and np.array_equal(tn, nzs[d]), (lengths, T)
        count += 1
    assert count == sum(1 for _ in _all_row_length_vectors())


def test_merge_split_counting_matches_explicit_merge(orc):
    rng = np.random.default_rng(7)
    for _ in range(200):
        m = int(rng.integers(1, 12))
        lengths = rng.integers(0, 6, size=m)
        ro = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int32)
        rows, nzs = _merge_prefix_counts(ro)
        for d in range(len(rows)):
            assert orc.merge_split(ro, d) == (rows[d], nzs[d])


def test_partition_invariants_powerlaw(orc):
    a = synth.workload("powerlaw_4k")
    W = a.m + a.nnz
    for T in (7, 128, 2048, 3001):
        tr, tn = orc.partition(a.row_offsets, T)
        G = len(tr) - 1
        assert G == -(-W // T)
        assert (tr[0], tn[0]) == (0, 0) and (tr[-1], tn[-1]) == (a.m, a.nnz)
        assert np.all(np.diff(tr) >= 0) and np.all(np.diff(tn) >= 0)
        d = tr.astype(np.int64) + tn
        assert np.array_equal(d, np.minimum(np.arange(G + 1) * T, W))
        # The split's nonzero index lies inside (or at the end of) the open row.
        inner = tr < a.m
        ro = a.row_offsets.astype(np.int64)
        assert np.all(ro[tr[inner]] <= tn[inner]) and np.all(tn[inner] <= ro[tr[inner] + 1])


def test_partition_empty_rows_and_no_nonzeros(orc):
    ro = np.zeros(6, np.int32)  # 5 empty rows
    tr, tn = orc.partition(ro, 2)
    assert np.array_equal(tr, [0, 2, 4, 5]) and np.array_equal(tn, [0, 0, 0, 0])


# ------------------------------------------------------------------ SpMV


def test_spmv_identity_diagonal_permutation(orc):
    rng = np.random.default_rng(1)
    n = 300
    x = synth.uniform_pm1(rng, n)
    eye = synth.from_dense(np.eye(n))
    assert np.array_equal(orc.spmv(eye.row_offsets, eye.col_idx, eye.values, x), x.astype(np.float64))
    d = synth.uniform_pm1(rng, n)
    d[d == 0] = 0.5
    dg = synth.from_dense(np.diag(d))
    assert np.array_equal(orc.spmv(dg.row_offsets, dg.col_idx, dg.values, x), d.astype(np.float64) * x)
    p = rng.permutation(n)
    pm = synth.from_dense(np.eye(n)[p])
    assert np.array_equal(orc.spmv(pm.row_offsets, pm.col_idx, pm.values, x), x[p].astype(np.float64))


def test_spmv_dense_as_csr_vs_dense_matvec(orc):
    rng = np.random.default_rng(2)
    a = rng.uniform(-1, 1, size=(57, 43))
    a[rng.random(a.shape) < 0.3] = 0.0
    a = a.astype(np.float32)
    x = rng.uniform(-1, 1, size=43).astype(np.float32)
    c = synth.from_dense(a)
    y = orc.spmv(c.row_offsets, c.col_idx, c.values, x)
    ref = a.astype(np.float64) @ x.astype(np.float64)
    np.testing.assert_allclose(y, ref, rtol=0, atol=1e-13)


def test_spmv_powerlaw_vs_scipy(orc):
    a = synth.workload("powerlaw_4k")
    rng = np.random.default_rng(3)
    x = synth.uniform_pm1(rng, a.n)
    y = orc.spmv(a.row_offsets, a.col_idx, a.values, x)
    ref = _scipy(a) @ x.astype(np.float64)
    scale = orc.row_absdot(a.row_offsets, a.col_idx, a.values, x)
    assert np.all(np.abs(y - ref) <= 1e-13 * np.maximum(scale, 1e-300))
    np.testing.assert_allclose(scale, abs(_scipy(a)) @ np.abs(x.astype(np.float64)), rtol=1e-13, atol=0)


def test_spmv_integer_values_exact(orc):
    rng = np.random.default_rng(4)
    a = synth.powerlaw_csr(1000, 800, 20_000, 1.4, 400, seed=11)
    a.values = rng.integers(-8, 9, size=a.nnz).astype(np.float32)
    x = rng.integers(-8, 9, size=a.n).astype(np.float32)
    y = orc.spmv(a.row_offsets, a.col_idx, a.values, x)
    ref = _scipy(a).astype(np.int64) @ x.astype(np.int64)
    assert np.array_equal(y, ref.astype(np.float64))


def test_spmv_column_sum_invariant(orc):
    a = synth.workload("powerlaw_4k")
    x = synth.uniform_pm1(np.random.default_rng(5), a.n)
    y = orc.spmv(a.row_offsets, a.col_idx, a.values, x)
    colsum = np.zeros(a.n)
    np.add.at(colsum, a.col_idx, a.values.astype(np.float64))
    bound = 1e-12 * float(orc.row_absdot(a.row_offsets, a.col_idx, a.values, x).sum())
    assert abs(y.sum() - colsum @ x.astype(np.float64)) <= bound


def test_spmv_empty_rows_zero_and_thread_independent(orc):
    a = synth.powerlaw_csr(3000, 3000, 30_000, 1.3, 3000, seed=12)
    # Empty every third row.
    lengths = a.row_lengths()
    keep = np.ones(a.nnz, bool)
    for r in range(0, a.m, 3):
        keep[a.row_offsets[r] : a.row_offsets[r + 1]] = False
    lengths[0::3] = 0
    ro = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int32)
    ci, v = a.col_idx[keep], a.values[keep]
    x = synth.uniform_pm1(np.random.default_rng(6), a.n)
    y1 = orc.spmv(ro, ci, v, x, threads=1)
    y8 = orc.spmv(ro, ci, v, x, threads=8)
    assert np.array_equal(y1, y8)
    assert np.all(y1[0::3] == 0.0)


# ------------------------------------------------------------------ transpose / backward


def test_transpose_vs_scipy(orc):
    a = synth.workload("powerlaw_4k")
    co, ri, perm = orc.transpose(a.row_offsets, a.col_idx, a.n)
    # Distinct tags make scipy's conversion reveal the permutation.
    tagged = sp.csr_matrix((np.arange(a.nnz, dtype=np.float64) + 1, a.col_idx, a.row_offsets), shape=(a.m, a.n)).tocsc()
    tagged.has_sorted_indices = False
    assert np.array_equal(co, tagged.indptr)
    assert np.array_equal(ri, tagged.indices)
    assert np.array_equal(perm, tagged.data.astype(np.int64) - 1)
    # Stability: inside a column the original index increases.
    for j in range(0, a.n, 97):
        assert np.all(np.diff(perm[co[j] : co[j + 1]]) > 0)


def test_spmv_t_vs_scipy_and_dense(orc):
    a = synth.workload("powerlaw_4k")
    g = synth.uniform_pm1(np.random.default_rng(8), a.m)
    dx = orc.spmv_t(a.row_offsets, a.col_idx, a.values, g, a.n)
    ref = _scipy(a).T @ g.astype(np.float64)
    scale = orc.col_absdot(a.row_offsets, a.col_idx, a.values, g, a.n)
    assert np.all(np.abs(dx - ref) <= 1e-13 * np.maximum(scale, 1e-300))
    small = synth.powerlaw_csr(60, 50, 600, 1.5, 50, seed=13)
    gs = synth.uniform_pm1(np.random.default_rng(9), 60)
    dense = _scipy(small).toarray()
    np.testing.assert_allclose(orc.spmv_t(small.row_offsets, small.col_idx, small.values, gs, 50), dense.T @ gs.astype(np.float64), atol=1e-13, rtol=0)


def _fd_matrix():
    """256x256 log-normal(2.5, 1.2) rows clipped to [1, 256]: the differentiable law at FD size."""
    return synth.lognormal_csr(256, 256, 2.5, 1.2, seed=4, l_max=256)


def test_finite_differences_pin_gradients(orc):
    a = _fd_matrix()
    rng = np.random.default_rng(10)
    x = rng.uniform(-1, 1, a.n)
    t = rng.uniform(-1, 1, a.m)
    v = a.values.astype(np.float64)
    ro, ci = a.row_offsets, a.col_idx
    g = orc.spmv(ro, ci, v, x) - t  # dL/dy
    dx = orc.spmv_t(ro, ci, v, g, a.n)
    dv = orc.dvalues(ro, ci, g, x)
    h = 1e-3

    def L(vv, xx):
        return orc.loss(ro, ci, vv, xx, t)

    # L is quadratic in x (and in v), so the central difference has no truncation term.
    for j in range(a.n):
        e = np.zeros(a.n)
        e[j] = h
        fd = (L(v, x + e) - L(v, x - e)) / (2 * h)
        assert abs(fd - dx[j]) <= 1e-9 * max(1.0, abs(dx[j])), j
    for k in rng.choice(a.nnz, size=300, replace=False):
        e = np.zeros(a.nnz)
        e[k] = h
        fd = (L(v + e, x) - L(v - e, x)) / (2 * h)
        assert abs(fd - dv[k]) <= 1e-9 * max(1.0, abs(dv[k])), k


def test_dense_gradient_identity(orc):
    """dx = A^T (A x - t) against a dense FP64 matmul."""
    a = _fd_matrix()
    rng = np.random.default_rng(11)
    x = rng.uniform(-1, 1, a.n)
    t = rng.uniform(-1, 1, a.m)
    dense = _scipy(a).toarray()
    g = orc.spmv(a.row_offsets, a.col_idx, a.values, x) - t
    np.testing.assert_allclose(orc.spmv_t(a.row_offsets, a.col_idx, a.values, g, a.n), dense.T @ (dense @ x - t), atol=1e-11, rtol=0)


# ------------------------------------------------------------------ batched


def test_block_diagonal_partition_equals_per_matrix_splits(orc):
    b = synth.batched_powerlaw(12, 4, 40, 300, 1.5, seed=21)
    ro_g = orc.block_diagonal_offsets(b.ms, b.nnzs, b.row_offsets)
    assert ro_g[-1] == b.nnzs.sum() and len(ro_g) == b.ms.sum() + 1
    T = 5
    tr, tn = orc.partition(ro_g, T)
    work = np.concatenate([[0], np.cumsum(b.ms + b.nnzs)])
    row_base = np.concatenate([[0], np.cumsum(b.ms)])
    nz_base = np.concatenate([[0], np.cumsum(b.nnzs)])
    for c in range(len(tr)):
        d = min(c * T, int(work[-1]))
        i = max(int(np.searchsorted(work, d, side="right")) - 1, 0)
        i = min(i, b.count - 1)
        li, lj = orc.merge_split(b.matrix(i).row_offsets, d - int(work[i]))
        assert (tr[c], tn[c]) == (row_base[i] + li, nz_base[i] + lj), c


def test_batched_spmv_vs_scipy_block_diag(orc):
    b = synth.batched_powerlaw(20, 8, 300, 4000, 1.5, seed=22)
    x = synth.uniform_pm1(np.random.default_rng(12), int(b.ns.sum()))
    mats = [_scipy(b.matrix(i)) for i in range(b.count)]
    ref = sp.block_diag(mats, format="csr") @ x.astype(np.float64)
    np.testing.assert_allclose(orc.batched_spmv(b, x), ref, atol=1e-12, rtol=0)


def test_tolerance_scales_vs_scipy(orc):
    """The scales every tolerance is measured in: sum_j |a_ij| |x_j| per row (|A| |x|),
    sum_i |a_ij| |g_i| per column (|A|^T |g|), their batched form over the block-diagonal
    matrix, and the tile count ceil((m + nnz) / T)."""
    rng = np.random.default_rng(31)
    a = synth.csr_from_row_lengths(rng, 120, rng.integers(0, 25, 150))
    x = rng.standard_normal(a.n)
    g = rng.standard_normal(a.m)
    A = abs(_scipy(a))
    np.testing.assert_allclose(orc.row_absdot(a.row_offsets, a.col_idx, a.values, x), A @ np.abs(x),
                               rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(orc.col_absdot(a.row_offsets, a.col_idx, a.values, g, a.n), A.T @ np.abs(g),
                               rtol=1e-13, atol=1e-13)
    b = synth.batched_powerlaw(12, 8, 200, 2500, 1.5, seed=23)
    xb = rng.standard_normal(int(b.ns.sum()))
    mats = [abs(_scipy(b.matrix(i))) for i in range(b.count)]
    np.testing.assert_allclose(orc.batched_row_absdot(b, xb), sp.block_diag(mats, format="csr") @ np.abs(xb),
                               rtol=1e-13, atol=1e-13)
    for m, nnz, T in ((0, 0, 5), (1, 0, 5), (7, 3, 5), (4096, 64080, 2040), (10, 10, 1)):
        assert orc.num_tiles(m, nnz, T) == -(-(m + nnz) // T)


@pytest.mark.parametrize("name", ["powerlaw_4k"])
def test_oracle_deterministic_across_threads(orc, name):
    a = synth.workload(name)
    x = synth.uniform_pm1(np.random.default_rng(13), a.n)
    g = synth.uniform_pm1(np.random.default_rng(14), a.m)
    for fn in (lambda th: orc.spmv(a.row_offsets, a.col_idx, a.values, x, th),
               lambda th: orc.spmv_t(a.row_offsets, a.col_idx, a.values, g, a.n, th),
               lambda th: orc.dvalues(a.row_offsets, a.col_idx, g, x, th)):
        assert np.array_equal(fn(1), fn(4))


def test_spmm_pins(orc):
    """SpMM against the dense product (numpy matmul of the dense A), against scipy's sparse
    product, and column by column against SpMV; identity A returns B; a single column is SpMV."""
    import scipy.sparse as sp

    rng = np.random.default_rng(41)
    a = synth.csr_from_row_lengths(rng, 90, rng.integers(0, 30, 70))
    for kc in (1, 3, 4, 17):
        B = rng.standard_normal((a.n, kc))
        C = orc.spmm(a.row_offsets, a.col_idx, a.values, B)
        A = sp.csr_matrix((a.values.astype(np.float64), a.col_idx, a.row_offsets), shape=(a.m, a.n))
        np.testing.assert_allclose(C, A.toarray() @ B, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(C, (A @ B), rtol=1e-12, atol=1e-12)
        for j in range(kc):
            assert np.array_equal(C[:, j], orc.spmv(a.row_offsets, a.col_idx, a.values, B[:, j]))
        S = orc.spmm_absdot(a.row_offsets, a.col_idx, a.values, B)
        assert np.allclose(S, np.abs(A.toarray()) @ np.abs(B))
        assert (np.abs(C) <= S + 1e-12).all()
    eye = synth.from_dense(np.eye(6))
    B = rng.standard_normal((6, 5))
    assert np.array_equal(orc.spmm(eye.row_offsets, eye.col_idx, eye.values, B), B)


def test_sssp_pins(orc):
    """Dijkstra against scipy's shortest paths (weighted and unweighted), and a hand-worked
    graph: 0 -> 1 (4), 0 -> 2 (1), 2 -> 1 (2), 1 -> 3 (1), 3 unreachable from 4."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import shortest_path

    ro = np.array([0, 2, 3, 4, 4, 4], np.int32)
    ci = np.array([1, 2, 3, 1], np.int32)
    w = np.array([4.0, 1.0, 1.0, 2.0])
    d = orc.sssp(ro, ci, w, 0)
    assert d[:4].tolist() == [0.0, 3.0, 1.0, 4.0] and np.isinf(d[4])
    assert orc.sssp(ro, ci, None, 0)[:4].tolist() == [0.0, 1.0, 1.0, 2.0]
    rng = np.random.default_rng(77)
    a = synth.csr_from_row_lengths(rng, 400, rng.integers(0, 6, 400))
    wts = rng.uniform(0.5, 3.0, a.nnz)
    G = sp.csr_matrix((wts, a.col_idx, a.row_offsets), shape=(400, 400))
    for src in (0, 7, 399):
        ref = shortest_path(G, method="D", directed=True, indices=src)
        got = orc.sssp(a.row_offsets, a.col_idx, wts, src)
        assert np.array_equal(np.isinf(ref), np.isinf(got))
        fin = np.isfinite(ref)
        np.testing.assert_allclose(got[fin], ref[fin], rtol=1e-12)
        ref_u = shortest_path(G, method="D", directed=True, unweighted=True, indices=src)
        assert np.array_equal(orc.sssp(a.row_offsets, a.col_idx, None, src), ref_u)
