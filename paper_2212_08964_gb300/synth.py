"""Seeded synthetic CSR inputs shaped like the workloads of the dissertation's SpMV study.

The evaluation of Ch.4 (Sec. "Evaluation") runs SpMV over the SuiteSparse collection,
which is not available here; these generators stand in for it with power-law,
log-normal, stencil and batched matrices.  This module only *constructs inputs*:
it holds none of the method's arithmetic (no SpMV, no partition, no transpose) and is
the one module shared by the CUDA path's tests/benchmark and the CPU oracle.

Every draw comes from ``numpy.random.Generator(PCG64(seed))`` so a (config, seed) pair
gives the same arrays on every machine with the same numpy.

Conventions (Sec. "Compressed Sparse Data Structures"): ``row_offsets`` is int32[m+1],
``col_idx`` int32[nnz] (distinct and sorted within each row), ``values`` float32[nnz].
Values, x and targets are uniform on [-1, 1] and built from 24-bit integers, so they are
exactly representable in FP32.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "CSR",
    "BatchedCSR",
    "uniform_pm1",
    "pareto_row_lengths",
    "solve_pareto_xmin",
    "lognormal_row_lengths",
    "csr_from_row_lengths",
    "powerlaw_csr",
    "lognormal_csr",
    "stencil7_csr",
    "batched_powerlaw",
    "from_dense",
    "workload",
    "WORKLOADS",
]


@dataclasses.dataclass
class CSR:
    """A CSR matrix held in host numpy arrays."""

    m: int
    n: int
    row_offsets: np.ndarray  # int32[m+1]
    col_idx: np.ndarray  # int32[nnz]
    values: np.ndarray  # float32[nnz]

    @property
    def nnz(self) -> int:
        return int(self.col_idx.shape[0])

    def row_lengths(self) -> np.ndarray:
        return np.diff(self.row_offsets.astype(np.int64))


@dataclasses.dataclass
class BatchedCSR:
    """K independent CSR matrices stored back to back.

    ``row_offsets`` concatenates each matrix's own offsets (m_i+1 entries, each starting
    at 0); ``col_idx`` holds local column indices in [0, n_i); ``values`` concatenates the
    values.  The i-th x (n_i entries) and y (m_i entries) are likewise concatenated.
    """

    ms: np.ndarray  # int64[K]
    ns: np.ndarray  # int64[K]
    nnzs: np.ndarray  # int64[K]
    row_offsets: np.ndarray  # int32[sum(m_i+1)]
    col_idx: np.ndarray  # int32[sum nnz_i]
    values: np.ndarray  # float32[sum nnz_i]

    @property
    def count(self) -> int:
        return int(self.ms.shape[0])

    def matrix(self, i: int) -> CSR:
        ro_start = int(self.ms[:i].sum() + i)
        nz_start = int(self.nnzs[:i].sum())
        m, n, nnz = int(self.ms[i]), int(self.ns[i]), int(self.nnzs[i])
        return CSR(
            m,
            n,
            self.row_offsets[ro_start : ro_start + m + 1],
            self.col_idx[nz_start : nz_start + nnz],
            self.values[nz_start : nz_start + nnz],
        )


def uniform_pm1(rng: np.random.Generator, size: int) -> np.ndarray:
    """Uniform values on [-1, 1] from 24-bit integers: (k - 2^23) / 2^23, exact in FP32."""
    k = rng.integers(0, (1 << 24) + 1, size=size, dtype=np.int64)
    return ((k - (1 << 23)).astype(np.float64) / float(1 << 23)).astype(np.float32)


def _pareto_mean(x_min: float, s: float, l_max: int) -> float:
    """Exact mean of clip(floor(x_min * U^(-1/s)), 1, l_max) with U ~ U(0, 1].

    P(L >= l) = 1 for l = 1 and min(1, (x_min / l)^s) for 2 <= l <= l_max, so the mean is
    1 + sum_{l=2}^{l_max} min(1, (x_min / l)^s).
    """
    ls = np.arange(2, l_max + 1, dtype=np.float64)
    return 1.0 + float(np.minimum(1.0, (x_min / ls) ** s).sum())


def solve_pareto_xmin(mean: float, s: float, l_max: int) -> float:
    """Bisection for the x_min whose clipped, floored Pareto tail has the requested mean."""
    if mean <= 1.0:
        return 0.0
    lo, hi = 0.0, float(l_max) + 1.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if _pareto_mean(mid, s, l_max) < mean:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def pareto_row_lengths(rng: np.random.Generator, m: int, x_min: float, s: float, l_max: int) -> np.ndarray:
    """Row lengths L = clip(floor(x_min * U^(-1/s)), 1, l_max), U ~ U(0, 1]."""
    u = 1.0 - rng.random(m)  # (0, 1]
    with np.errstate(over="ignore"):
        raw = np.floor(x_min * u ** (-1.0 / s))
    return np.clip(raw, 1, l_max).astype(np.int64)


def lognormal_row_lengths(rng: np.random.Generator, m: int, mu: float, sigma: float, l_max: int) -> np.ndarray:
    """Row lengths L = clip(floor(exp(mu + sigma Z)), 1, l_max), Z ~ N(0, 1)."""
    z = rng.standard_normal(m)
    with np.errstate(over="ignore"):
        raw = np.floor(np.exp(mu + sigma * z))
    return np.clip(raw, 1, l_max).astype(np.int64)


def csr_from_row_lengths(rng: np.random.Generator, n: int, lengths: np.ndarray, with_values: bool = True) -> CSR:
    """Distinct, sorted, uniformly placed columns for every row, without a sort.

    For a row of length L the sorted uniforms U_(1..L) are the normalised partial sums of
    L+1 exponential spacings; col_i = min(floor(U_(i) * (n - L + 1)), n - L) + (i - 1) is
    strictly increasing and stays in [0, n).
    """
    lengths = np.asarray(lengths, dtype=np.int64)
    m = int(lengths.shape[0])
    if m and int(lengths.max()) > n:
        raise ValueError("a row is longer than the number of columns")
    ro = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(lengths, out=ro[1:])
    nnz = int(ro[-1])
    if nnz >= 2**31:
        raise ValueError("nnz must fit int32")
    # L+1 spacings per row, laid out row after row.
    spacing_off = ro[:-1] + np.arange(m, dtype=np.int64)  # start of row r's spacings
    e = rng.standard_exponential(nnz + m)
    c = np.cumsum(e)
    before = np.where(spacing_off > 0, c[np.maximum(spacing_off - 1, 0)], 0.0)
    total = c[spacing_off + lengths] - before  # S_{L+1}
    row_of = np.repeat(np.arange(m, dtype=np.int64), lengths)
    within = np.arange(nnz, dtype=np.int64) - ro[:-1][row_of]  # i-1
    partial = c[spacing_off[row_of] + within] - before[row_of]  # S_i
    span = (n - lengths + 1)[row_of]
    base = np.minimum(np.floor(partial / total[row_of] * span).astype(np.int64), span - 1)
    cols = (base + within).astype(np.int32)
    vals = uniform_pm1(rng, nnz) if with_values else np.zeros(nnz, np.float32)
    return CSR(m, n, ro.astype(np.int32), cols, vals)


def powerlaw_csr(m: int, n: int, nnz_target: float, s: float, l_max: int, seed: int) -> CSR:
    """Power-law ("Zipf-tail") rows: Pareto lengths whose mean gives ~nnz_target nonzeros."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x_min = solve_pareto_xmin(nnz_target / m, s, l_max)
    lengths = pareto_row_lengths(rng, m, x_min, s, l_max)
    return csr_from_row_lengths(rng, n, lengths)


def lognormal_csr(m: int, n: int, mu: float, sigma: float, seed: int, l_max: int | None = None) -> CSR:
    """Log-normal row lengths (the differentiable workload's law)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lengths = lognormal_row_lengths(rng, m, mu, sigma, n if l_max is None else l_max)
    return csr_from_row_lengths(rng, n, lengths)


def stencil7_csr(nx: int, seed: int, integer_values: bool = False) -> CSR:
    """7-point 3-D Laplacian pattern on an nx^3 grid (natural ordering, sorted columns).

    With ``integer_values`` the diagonal is 6 and the off-diagonals -1; otherwise every
    stored entry is uniform on [-1, 1].
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    m = nx**3
    r = np.arange(m, dtype=np.int64)
    i, j, k = r // (nx * nx), (r // nx) % nx, r % nx
    # Neighbour offsets in increasing column order.
    offs = [(-nx * nx, i > 0), (-nx, j > 0), (-1, k > 0), (0, np.ones(m, bool)), (1, k < nx - 1), (nx, j < nx - 1), (nx * nx, i < nx - 1)]
    present = np.stack([p for _, p in offs], axis=1)  # [m, 7]
    cols = r[:, None] + np.array([o for o, _ in offs], dtype=np.int64)[None, :]
    lengths = present.sum(axis=1)
    ro = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(lengths, out=ro[1:])
    ci = cols[present].astype(np.int32)
    if integer_values:
        diag = np.broadcast_to(np.array([o == 0 for o, _ in offs]), present.shape)[present]
        vals = np.where(diag, 6.0, -1.0).astype(np.float32)
    else:
        vals = uniform_pm1(rng, int(ro[-1]))
    return CSR(m, m, ro.astype(np.int32), ci, vals)


def batched_powerlaw(count: int, m_lo: int, m_hi: int, nnz_target: float, s: float, seed: int) -> BatchedCSR:
    """``count`` square matrices with m_i log-uniform in [m_lo, m_hi] and power-law rows.

    Row lengths follow clip(floor(x_min U^(-1/s)), 1, max(1, m_i // 4)); one x_min is
    solved so that the expected total nonzero count is ``nnz_target``.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    logm = rng.uniform(math.log(m_lo), math.log(m_hi), size=count)
    ms = np.clip(np.floor(np.exp(logm)), m_lo, m_hi).astype(np.int64)
    lmax = np.maximum(1, ms // 4)
    # Expected total nnz for a given x_min, from prefix sums of l^-s.
    top = int(lmax.max())
    ls = np.arange(0, top + 1, dtype=np.float64)
    pw = np.zeros(top + 1)
    pw[2:] = ls[2:] ** (-s)
    cpw = np.cumsum(pw)  # cpw[L] = sum_{l=2}^{L} l^-s

    def expected_total(x_min: float) -> float:
        f = int(min(math.floor(x_min), top))  # lengths l <= x_min have P = 1
        cut = np.minimum(lmax, max(f, 1))
        ones = np.maximum(cut - 1, 0)  # l in [2, cut]
        tail = cpw[lmax] - cpw[cut]
        return float((ms * (1.0 + ones + (x_min**s) * tail)).sum())

    lo, hi = 0.0, float(top) + 1.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if expected_total(mid) < nnz_target:
            lo = mid
        else:
            hi = mid
    x_min = 0.5 * (lo + hi)
    lengths = pareto_row_lengths(rng, int(ms.sum()), x_min, s, top)
    # Clip each matrix's rows to its own maximum.
    owner = np.repeat(np.arange(count), ms)
    lengths = np.minimum(lengths, lmax[owner])
    ros, cis, vas, nnzs = [], [], [], []
    start = 0
    for i in range(count):
        li = lengths[start : start + ms[i]]
        start += int(ms[i])
        a = csr_from_row_lengths(rng, int(ms[i]), li)
        ros.append(a.row_offsets)
        cis.append(a.col_idx)
        vas.append(a.values)
        nnzs.append(a.nnz)
    return BatchedCSR(
        ms,
        ms.copy(),
        np.asarray(nnzs, dtype=np.int64),
        np.concatenate(ros),
        np.concatenate(cis),
        np.concatenate(vas),
    )


def stencil5_csr(k: int, rng: np.random.Generator) -> CSR:
    """5-point 2-D Laplacian pattern on a k x k grid (natural ordering, sorted columns),
    every stored entry uniform on [-1, 1]."""
    m = k * k
    r = np.arange(m, dtype=np.int64)
    i, j = r // k, r % k
    offs = [(-k, i > 0), (-1, j > 0), (0, np.ones(m, bool)), (1, j < k - 1), (k, i < k - 1)]
    present = np.stack([p for _, p in offs], axis=1)
    cols = r[:, None] + np.array([o for o, _ in offs], dtype=np.int64)[None, :]
    ro = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(present.sum(axis=1), out=ro[1:])
    return CSR(m, m, ro.astype(np.int32), cols[present].astype(np.int32), uniform_pm1(rng, int(ro[-1])))


def batched_grid(count: int, k_lo: int, k_hi: int, seed: int) -> BatchedCSR:
    """``count`` 5-point Laplacians on k x k grids, k log-uniform in [k_lo, k_hi]: a batch of
    regular matrices of uneven size (a batch of small PDE problems)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ks = np.clip(np.floor(np.exp(rng.uniform(math.log(k_lo), math.log(k_hi + 1), size=count))), k_lo, k_hi)
    mats = [stencil5_csr(int(k), rng) for k in ks.astype(np.int64)]
    ms = np.array([a.m for a in mats], dtype=np.int64)
    return BatchedCSR(ms, ms.copy(), np.array([a.nnz for a in mats], dtype=np.int64),
                      np.concatenate([a.row_offsets for a in mats]), np.concatenate([a.col_idx for a in mats]),
                      np.concatenate([a.values for a in mats]))


def from_dense(a: np.ndarray) -> CSR:
    """CSR of the nonzero pattern of a small dense matrix (row-major scan)."""
    a = np.asarray(a, dtype=np.float32)
    m, n = a.shape
    rows, cols = np.nonzero(a)
    ro = np.zeros(m + 1, dtype=np.int64)
    np.add.at(ro, rows + 1, 1)
    ro = np.cumsum(ro)
    return CSR(m, n, ro.astype(np.int32), cols.astype(np.int32), a[rows, cols].astype(np.float32))


# Named workloads: the paper-shaped configurations, with their seeds.
WORKLOADS = {
    "powerlaw_4k": dict(kind="powerlaw", m=4096, n=4096, nnz=64_000, s=1.5, l_max=2048, seed=1),
    "powerlaw_4m": dict(kind="powerlaw", m=4_194_304, n=4_194_304, nnz=64_000_000, s=1.3, l_max=500_000, seed=2),
    "stencil7_160": dict(kind="stencil", nx=160, seed=3),
    "lognormal_1m": dict(kind="lognormal", m=1_048_576, n=1_048_576, mu=2.5, sigma=1.2, seed=4),
    "batched_4096": dict(kind="batched", count=4096, m_lo=64, m_hi=65536, nnz=50_000_000, s=1.5, seed=5),
    "powerlaw_8m": dict(kind="powerlaw", m=8_388_608, n=8_388_608, nnz=128_000_000, s=1.3, l_max=500_000, seed=6),
    # A second batch class: 1024 2-D Laplacians of uneven size (m_i = k^2, k log-uniform in
    # [8, 256], so m_i spans [64, 65536] as in batched_4096), about 48M nonzeros.
    "batched_grid_1024": dict(kind="batched_grid", count=1024, k_lo=8, k_hi=256, seed=7),
}


def workload(name: str, scale: float = 1.0):
    """Build a named workload; ``scale`` < 1 shrinks m, n and nnz together (tests)."""
    w = dict(WORKLOADS[name])
    kind = w.pop("kind")
    if kind == "powerlaw":
        m = max(1, int(w["m"] * scale))
        n = max(1, int(w["n"] * scale))
        return powerlaw_csr(m, n, w["nnz"] * scale, w["s"], min(w["l_max"], n), w["seed"])
    if kind == "lognormal":
        m = max(1, int(w["m"] * scale))
        n = max(1, int(w["n"] * scale))
        return lognormal_csr(m, n, w["mu"], w["sigma"], w["seed"])
    if kind == "stencil":
        nx = max(2, int(round(w["nx"] * scale ** (1.0 / 3.0))))
        return stencil7_csr(nx, w["seed"])
    if kind == "batched_grid":
        count = max(1, int(w["count"] * scale))
        return batched_grid(count, w["k_lo"], w["k_hi"], w["seed"])
    if kind == "batched":
        count = max(1, int(w["count"] * scale))
        return batched_powerlaw(count, w["m_lo"], w["m_hi"], w["nnz"] * count / w["count"], w["s"], w["seed"])
    raise KeyError(name)
