"""The C-ABI library builds, loads, exports every symbol include/lbspmv.h declares, and
rejects bad arguments on the host before touching the GPU (runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbspmv.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lb_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2212_08964_gb300 import _build

    path = _build.build()
    lib = ctypes.CDLL(path)
    lib.lb_status_string.restype = ctypes.c_char_p
    return lib


def test_header_declares_the_boundary():
    names = _declared()
    for required in ["lb_spmv", "lb_partition", "lb_plan_create", "lb_spmv_planned", "lb_plan_build_transpose",
                     "lb_spmv_t", "lb_spmv_dvalues", "lb_batched_plan_create", "lb_spmv_batched", "lb_validate_csr"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_and_version(lib):
    for code in (0, -1, -2, -3, -4, -5, -6):
        assert lib.lb_status_string(code).startswith(b"LB_")
    assert lib.lb_version() >= 10000


def test_num_tiles_arithmetic(lib):
    assert lib.lb_num_tiles(4, 6, 3) == 4
    assert lib.lb_num_tiles(4, 6, 4) == 3
    assert lib.lb_num_tiles(0, 0, 8) == 0
    assert lib.lb_num_tiles(-1, 0, 8) == -1


def test_host_side_argument_rejection(lib):
    P = ctypes.c_void_p
    # Negative sizes, nnz without rows, unknown dtype: rejected before any CUDA call.
    assert lib.lb_spmv(-1, 4, 0, None, None, None, 0, None, None, None) == -1
    assert lib.lb_spmv(0, 4, 5, None, None, None, 0, None, None, None) == -1
    assert lib.lb_spmv(4, 4, 4, None, None, None, 7, None, None, None) == -1
    assert lib.lb_spmv(0, 0, 0, None, None, None, 0, None, None, None) == 0  # m == 0: no-op
    assert lib.lb_partition(4, 6, None, 0, None, None, None) == -1
    # Tiles of one item over 2^31 work items: a tile count beyond 32 bits, refused on the host
    # (the pointers are never dereferenced).
    fake = ctypes.c_void_p(256)
    assert lib.lb_partition(1 << 30, (1 << 31) - 1, fake, 1, fake, fake, None) == -1
    out = P()
    assert lib.lb_plan_create(4, 4, 4, None, 0, None, None, ctypes.byref(out)) == -1  # null offsets
    assert lib.lb_plan_create(4, 4, 4, ctypes.c_void_p(16), 99, None, None, ctypes.byref(out)) == -1  # bad schedule

    class Tuning(ctypes.Structure):
        _fields_ = [("threads", ctypes.c_int), ("items_per_thread", ctypes.c_int), ("group_size", ctypes.c_int)]

    bad = Tuning(256, 7, 0)  # shape not compiled
    assert lib.lb_plan_create(4, 4, 4, ctypes.c_void_p(16), 5, ctypes.byref(bad), None, ctypes.byref(out)) == -1
    bad_group = Tuning(0, 0, 3)
    assert lib.lb_plan_create(4, 4, 4, ctypes.c_void_p(16), 4, ctypes.byref(bad_group), None, ctypes.byref(out)) == -1
    assert lib.lb_batched_plan_create(1, None, None, None, None, 1, None, None, ctypes.byref(out)) == -1
    one = (ctypes.c_int * 1)(4)
    assert lib.lb_batched_plan_create(1, one, one, one, ctypes.c_void_p(16), 2, None, None, ctypes.byref(out)) == -3
    assert lib.lb_spmv_planned(None, None, None, 0, None, None, None) == -1
    assert lib.lb_spmv_t(None, None, 0, None, None, None) == -1
    assert lib.lb_spmv_dvalues(None, None, None, None, None, 0, None) == -1
    # dvalues types: FP32 or the values' 16-bit type only (a fake plan pointer, never read:
    # the type check comes first).
    fake = ctypes.c_void_p(256)
    assert lib.lb_spmv_dvalues(fake, None, None, None, None, 7, None) == -1
    assert lib.lb_spmv_dvalues_gathered(fake, None, None, None, 7, None) == -1
    assert lib.lb_spmv_batched(None, None, None, 0, None, None, None) == -1
    assert lib.lb_validate_csr(-1, 0, 0, None, None, 0, None, None) == -1
    assert lib.lb_device_error(None, 0) == -1


def test_allocation_failure_injection_on_host(lib):
    """A plan whose first device allocation fails reports LB_ERR_NO_MEMORY, returns no plan
    and holds nothing; the failure is injected on the host, before any device memory."""
    lib.lb_debug_live_allocations.restype = ctypes.c_longlong
    out = ctypes.c_void_p()
    live = lib.lb_debug_live_allocations()
    lib.lb_debug_fail_allocations_after(0)
    try:
        assert lib.lb_plan_create(4, 4, 4, ctypes.c_void_p(16), 5, None, None, ctypes.byref(out)) == -4
        assert out.value is None
        assert lib.lb_debug_live_allocations() == live
    finally:
        lib.lb_debug_fail_allocations_after(-1)
