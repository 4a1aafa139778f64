"""lb_spmv_static (the allocation-free one-shot SpMV) against lb_spmv, through the C ABI.

The file name sorts last so pytest collects it after every other test: it must pass both
alone in a fresh process (where its first call does the per-device set-up) and after the
rest of the suite has run other kernels on the device.
"""
import ctypes

import numpy as np
import pytest
import torch

from gpu_helpers import check_bound, dev, to_dev, vec, workload
from paper_2212_08964_gb300 import synth

from paper_2212_08964_gb300 import lbspmv as _lbspmv

TOL32 = 1e-5
MAX_WORK = _lbspmv.STATIC_MAX_TILES * _lbspmv.STATIC_TILE_ITEMS  # LB_SPMV_STATIC_MAX_TILES * ..._TILE_ITEMS


def _raw_lib():
    from paper_2212_08964_gb300 import _build

    lib = ctypes.CDLL(_build.build())
    lib.lb_status_string.restype = ctypes.c_char_p
    P = ctypes.c_void_p
    I = ctypes.c_int
    lib.lb_spmv_static.argtypes = [I, I, I, P, P, P, I, P, P, P]
    lib.lb_spmv_static.restype = I
    lib.lb_spmv.argtypes = [I, I, I, P, P, P, I, P, P, P]
    lib.lb_spmv.restype = I
    return lib


def test_static_limits_rejected_on_host():
    """Sizes past the static workspace, and bad arguments, are refused before any GPU work."""
    lib = _raw_lib()
    fake = 256  # never dereferenced: every case below returns before touching the device
    assert lib.lb_status_string(-7).startswith(b"LB_ERR_TOO_LARGE")
    m = 1 << 20
    assert lib.lb_spmv_static(m, m, MAX_WORK - m + 1, fake, fake, fake, 0, fake, fake, None) == -7
    assert lib.lb_spmv_static(2**31 - 1, 8, 2**31 - 1, fake, fake, fake, 0, fake, fake, None) == -7
    assert lib.lb_spmv_static(-1, 4, 0, None, None, None, 0, None, None, None) == -1
    assert lib.lb_spmv_static(4, 4, 4, fake, fake, fake, 9, fake, fake, None) == -1
    assert lib.lb_spmv_static(4, 4, 4, None, fake, fake, 0, fake, fake, None) == -1
    assert lib.lb_spmv_static(0, 0, 0, None, None, None, 0, None, None, None) == 0


def _both(lib, m, n, nnz, ro, ci, v, vdt, x, stream):
    """y from lb_spmv, then two lb_spmv_static calls in a row into NaN-poisoned outputs."""
    y_ref = torch.empty(m, device="cuda")
    ys = [torch.full((m,), float("nan"), device="cuda") for _ in range(2)]
    p = lambda t: t.data_ptr()
    assert lib.lb_spmv(m, n, nnz, p(ro), p(ci), p(v), vdt, p(x), p(y_ref), stream) == 0
    for y in ys:
        assert lib.lb_spmv_static(m, n, nnz, p(ro), p(ci), p(v), vdt, p(x), p(y), stream) == 0
    torch.cuda.synchronize()
    return y_ref, ys


def _device_error_clear(lb):
    assert lb.device_error(clear=True) == 0


@pytest.mark.gpu
@pytest.mark.parametrize("name,scale,dtype", [("powerlaw_4k", 1.0, torch.float32),
                                              ("lognormal_1m", 0.3, torch.float32),
                                              ("powerlaw_4k", 1.0, torch.bfloat16)])
def test_static_matches_lb_spmv_twice(lb, orc, name, scale, dtype):
    lib = _raw_lib()
    a = workload(name, scale)
    ro, ci, v = to_dev(a, dtype)
    x = vec(a.n, 77)
    xd = dev(x)
    stream = torch.cuda.current_stream().cuda_stream
    vdt = {torch.float32: 0, torch.bfloat16: 1}[dtype]
    y_ref, ys = _both(lib, a.m, a.n, a.nnz, ro, ci, v, vdt, xd, stream)
    vals = a.values if dtype == torch.float32 else v.float().cpu().numpy()
    scale_rows = orc.row_absdot(a.row_offsets, a.col_idx, vals, x)
    ref = y_ref.cpu().numpy().astype(np.float64)
    for y in ys:
        check_bound(y.cpu().numpy(), ref, 2 * scale_rows, TOL32)
    assert torch.equal(ys[0], ys[1])
    _device_error_clear(lb)


@pytest.mark.gpu
def test_static_workspace_reused_across_sizes(lb, orc):
    """A many-tile call, then a one-tile call, then the many-tile call again: nothing stale
    from the earlier call leaks into the later ones."""
    lib = _raw_lib()
    stream = torch.cuda.current_stream().cuda_stream
    big = workload("lognormal_1m", 0.3)
    rng = np.random.default_rng(78)
    small = synth.csr_from_row_lengths(rng, 900, rng.integers(0, 5, 300))
    for a in (big, small, big):
        ro, ci, v = to_dev(a)
        x = vec(a.n, 79)
        y_ref, ys = _both(lib, a.m, a.n, a.nnz, ro, ci, v, 0, dev(x), stream)
        scale_rows = orc.row_absdot(a.row_offsets, a.col_idx, a.values, x)
        for y in ys:
            check_bound(y.cpu().numpy(), orc.spmv(a.row_offsets, a.col_idx, a.values, x), scale_rows, TOL32)
            check_bound(y.cpu().numpy(), y_ref.cpu().numpy().astype(np.float64), 2 * scale_rows, TOL32)
    _device_error_clear(lb)


@pytest.mark.gpu
def test_static_at_the_maximum_size(lb, orc):
    """m + nnz exactly at the static limit (every workspace tile in use), against lb_spmv."""
    lib = _raw_lib()
    stream = torch.cuda.current_stream().cuda_stream
    L = 127
    m = MAX_WORK // (L + 1)
    n = 1 << 22
    nnz = m * L
    assert m + nnz == MAX_WORK
    g = torch.Generator(device="cuda").manual_seed(80)
    ro = (torch.arange(m + 1, device="cuda", dtype=torch.int64) * L).to(torch.int32)
    ci = torch.randint(0, n, (nnz,), device="cuda", dtype=torch.int32, generator=g)
    v = torch.rand(nnz, device="cuda", generator=g) * 2 - 1
    x = torch.rand(n, device="cuda", generator=g) * 2 - 1
    y_ref, ys = _both(lib, m, n, nnz, ro, ci, v, 0, x, stream)
    scale_rows = (v.abs() * x[ci.long()].abs()).view(m, L).double().sum(1)
    bound = 2 * TOL32 * scale_rows
    for y in ys:
        err = (y.double() - y_ref.double()).abs()
        assert bool((err <= bound).all()), float((err / bound.clamp_min(1e-300)).max())
    assert torch.equal(ys[0], ys[1])
    # Sampled rows against the oracle itself, one row at a time (first, last and random rows).
    rows = np.unique(np.concatenate([[0, 1, m - 2, m - 1], np.random.default_rng(81).integers(0, m, 60)]))
    sel = torch.from_numpy(rows).cuda()
    cols = ci.view(m, L)[sel].cpu().numpy()
    vals = v.view(m, L)[sel].cpu().numpy()
    ro_s = (np.arange(len(rows) + 1) * L).astype(np.int32)
    xs = x.cpu().numpy()
    ref = orc.spmv(ro_s, cols.reshape(-1).astype(np.int32), vals.reshape(-1), xs)
    sc = orc.row_absdot(ro_s, cols.reshape(-1).astype(np.int32), vals.reshape(-1), xs)
    check_bound(ys[1][sel].cpu().numpy(), ref, sc, TOL32)
    del ci, v
    _device_error_clear(lb)


def _cudart():
    """The CUDA runtime the library is linked against (already loaded in this process)."""
    return ctypes.CDLL("libcudart.so.13")


# cudaMemPoolAttr values from the CUDA runtime API.
_POOL_USED_CURRENT = 7
_POOL_USED_HIGH = 8


def _pool_attr(rt, pool, attr):
    v = ctypes.c_uint64()
    assert rt.cudaMemPoolGetAttribute(pool, attr, ctypes.byref(v)) == 0
    return v.value


@pytest.mark.gpu
def test_static_allocates_nothing(lb):
    """Two calls after the set-up call leave the device's free memory and the default
    stream-ordered pool's high-water mark where they were: no cudaMalloc and no
    cudaMallocAsync (lb_spmv itself takes its workspace from that pool)."""
    lib = _raw_lib()
    stream = torch.cuda.current_stream().cuda_stream
    a = workload("lognormal_1m", 0.3)
    ro, ci, v = to_dev(a)
    x = dev(vec(a.n, 82))
    ys = [torch.empty(a.m, device="cuda") for _ in range(2)]
    p = lambda t: t.data_ptr()
    assert lib.lb_spmv_static(a.m, a.n, a.nnz, p(ro), p(ci), p(v), 0, p(x), p(ys[0]), stream) == 0  # set-up
    torch.cuda.synchronize()
    rt = _cudart()
    pool = ctypes.c_void_p()
    assert rt.cudaDeviceGetDefaultMemPool(ctypes.byref(pool), torch.cuda.current_device()) == 0
    zero = ctypes.c_uint64(0)
    assert rt.cudaMemPoolSetAttribute(pool, _POOL_USED_HIGH, ctypes.byref(zero)) == 0  # reset to current use
    used0 = _pool_attr(rt, pool, _POOL_USED_CURRENT)
    free0 = torch.cuda.mem_get_info()[0]
    live0 = lb.live_allocations()
    lb.fail_allocations_after(0)  # any allocation through the library's own allocator would now fail
    try:
        for y in ys:
            assert lib.lb_spmv_static(a.m, a.n, a.nnz, p(ro), p(ci), p(v), 0, p(x), p(y), stream) == 0
        torch.cuda.synchronize()
    finally:
        lb.fail_allocations_after(-1)
    assert _pool_attr(rt, pool, _POOL_USED_HIGH) == used0
    assert torch.cuda.mem_get_info()[0] == free0
    assert lb.live_allocations() == live0
    assert torch.equal(ys[0], ys[1])
    _device_error_clear(lb)
