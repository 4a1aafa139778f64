"""Merge-path partition on the GPU vs the oracle's counting definition: bit-exact."""
import itertools

import numpy as np
import pytest
import torch

from golden.fixtures import load
from gpu_helpers import dev, to_dev, workload

pytestmark = pytest.mark.gpu


def _gpu_partition(lb, ro_np, T):
    ro = dev(np.asarray(ro_np, np.int32))
    nnz = int(ro_np[-1]) if len(ro_np) > 1 else 0
    tr, tn = lb.partition(ro, nnz, T)
    torch.cuda.synchronize()
    return tr.cpu().numpy(), tn.cpu().numpy()


def test_worked_example(lb):
    f = load("worked_example_4x4.txt")
    for T in (3, 4):
        tr, tn = _gpu_partition(lb, f["row_offsets"].astype(np.int32), T)
        assert np.array_equal(tr, f[f"tile_row_T{T}"]) and np.array_equal(tn, f[f"tile_nz_T{T}"])


def test_bruteforce_small_matrices(lb, orc):
    count = 0
    for m in range(1, 5):
        for lengths in itertools.product(range(5), repeat=m):
            if sum(lengths) > 6:
                continue
            ro = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int32)
            W = m + int(ro[-1])
            for T in sorted({1, 2, 3, 5, W}):
                tr, tn = _gpu_partition(lb, ro, T)
                otr, otn = orc.partition(ro, T)
                assert np.array_equal(tr, otr) and np.array_equal(tn, otn), (lengths, T)
                count += 1
    assert count > 500


@pytest.mark.parametrize("T", [1, 7, 512, 2048, 4096, 99991])
def test_powerlaw_4k(lb, orc, T):
    a = workload("powerlaw_4k")
    tr, tn = _gpu_partition(lb, a.row_offsets, T)
    otr, otn = orc.partition(a.row_offsets, T)
    assert np.array_equal(tr, otr) and np.array_equal(tn, otn)


def test_degenerate_structures(lb, orc):
    rng = np.random.default_rng(3)
    cases = {
        "all_empty": np.zeros(1001, np.int32),
        "one_row_long": np.array([0, 1_000_003], np.int32),
        "huge_row_in_middle": np.concatenate([[0], np.cumsum([3, 0, 0, 250_000, 1, 0, 2])]).astype(np.int32),
        "mostly_empty": np.concatenate([[0], np.cumsum(np.where(rng.random(50_000) < 0.9, 0, rng.integers(1, 40, 50_000)))]).astype(np.int32),
        "single_empty_row": np.zeros(2, np.int32),
    }
    for name, ro in cases.items():
        for T in (1, 2, 64, 2048, 3072):
            tr, tn = _gpu_partition(lb, ro, T)
            otr, otn = orc.partition(ro, T)
            assert np.array_equal(tr, otr) and np.array_equal(tn, otn), (name, T)


@pytest.mark.parametrize("name", ["powerlaw_4m", "stencil7_160"])
def test_full_size_plan_partition(lb, orc, name):
    a = workload(name)
    ro, _, _ = to_dev(a)
    plan = lb.Plan(ro, a.n, a.nnz, schedule="merge_path")
    info = plan.info()
    tr, tn = plan.partition()
    otr, otn = orc.partition(a.row_offsets, info["tile_items"])
    assert len(tr) == info["num_tiles"] + 1
    assert np.array_equal(tr, otr) and np.array_equal(tn, otn)
    # The merge-path forward's warp tiles: the same split at its own tile size.
    G, T = plan.tiles("merge")
    assert T == 32 * info["items_per_thread"] - 8
    wtr, wtn = plan.partition(which="merge")
    assert len(wtr) == G + 1
    owtr, owtn = orc.partition(a.row_offsets, T)
    assert np.array_equal(wtr, owtr) and np.array_equal(wtn, owtn)
