"""Helpers shared by the GPU parity tests: device transfer, tolerance checks, cached inputs."""
import numpy as np
import torch

from paper_2212_08964_gb300 import synth

_cache = {}


def workload(name: str, scale: float = 1.0):
    key = (name, scale)
    if key not in _cache:
        _cache[key] = synth.workload(name, scale)
    return _cache[key]


def dev(a: np.ndarray, dtype=None) -> torch.Tensor:
    t = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return t if dtype is None else t.to(dtype)


def to_dev(a: synth.CSR, dtype=torch.float32):
    return dev(a.row_offsets), dev(a.col_idx), dev(a.values, dtype)


def vec(n: int, seed: int) -> np.ndarray:
    return synth.uniform_pm1(np.random.default_rng(seed), n)


def rounded(values: np.ndarray, dtype) -> np.ndarray:
    """FP32 values rounded to `dtype` (round-to-nearest-even) and widened back, exactly."""
    return torch.from_numpy(values).to(dtype).to(torch.float32).numpy()


def check_bound(got, ref, scale, tol, what="rows"):
    """|got - ref| <= tol * scale element-wise (scale 0 demands an exact 0).

    Returns (max, median) of |got - ref| / scale over the entries with scale > 0.
    """
    got = np.asarray(got, np.float64)
    err = np.abs(got - ref)
    bound = tol * scale
    bad = np.nonzero(err > bound)[0]
    assert bad.size == 0, (
        f"{bad.size} {what} exceed {tol} * sum|a||x|; first {bad[:5].tolist()}, "
        f"err {err[bad[:5]].tolist()}, bound {bound[bad[:5]].tolist()}"
    )
    pos = scale > 0
    rel = err[pos] / scale[pos] if pos.any() else np.zeros(1)
    return float(rel.max()), float(np.median(rel))
