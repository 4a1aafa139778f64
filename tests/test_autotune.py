"""Autotuner host logic (CPU): shape classes, the table and its JSON round trip, the fallback
to the size rule; on the GPU: the measured candidates and the tuned plan's results."""
import json

import numpy as np
import pytest

from paper_2212_08964_gb300 import autotune, synth


def _ro(lengths):
    ro = np.zeros(len(lengths) + 1, np.int64)
    np.cumsum(lengths, out=ro[1:])
    return ro.astype(np.int32)


def test_shape_class_fields():
    # 1000 rows of 8: work 9000 -> size 13; mean 8 -> 2*log2(8) = 6; skew 1 -> bucket 0.
    assert autotune.shape_class(_ro([8] * 1000)) == "size13-mean6-skew0-lrb3-f32"
    # One long row among short ones: skew = max / mean.
    lengths = [1] * 999 + [1001]
    mean = sum(lengths) / 1000  # 2.0
    assert 1001 / mean >= 256
    assert autotune.shape_class(_ro(lengths), "bf16").endswith("skew4-lrb9-bf16")
    # Empty matrix and all-empty rows do not fail.
    assert autotune.shape_class(np.zeros(1, np.int32)).startswith("size0-")
    assert "mean-99" in autotune.shape_class(_ro([0] * 10))


def test_shape_class_separates_the_workload_families():
    a = synth.workload("powerlaw_4k")
    b = synth.stencil7_csr(12, seed=3)
    assert autotune.shape_class(a.row_offsets) != autotune.shape_class(b.row_offsets)
    # Same law at the same size: same class.
    c = synth.powerlaw_csr(4096, 4096, 64_000, 1.5, 2048, seed=99)
    assert autotune.shape_class(a.row_offsets) == autotune.shape_class(c.row_offsets)


def test_batch_class_uses_the_largest_member():
    ms = np.array([10, 500, 20])
    lengths = [[1] * 10, [4] * 500, [2] * 20]
    nnzs = np.array([sum(x) for x in lengths])
    ro = np.concatenate([_ro(x) for x in lengths])
    key = autotune.batch_class(ms, nnzs, ro)
    assert key.startswith("batch1-") and autotune.shape_class(_ro([4] * 500)) in key


def test_table_record_lookup_and_json_round_trip(tmp_path):
    t = autotune.Table()
    res = [{"schedule": "merge_path", "threads": 256, "items_per_thread": 8, "group_size": 0, "ms": 0.5},
           {"schedule": "thread_mapped", "threads": 0, "items_per_thread": 0, "group_size": 0, "ms": 0.2}]
    t.record("k", res)
    assert t.lookup("k")["schedule"] == "thread_mapped"
    assert t.lookup("missing") is None
    path = str(tmp_path / "table.json")
    t.save(path)
    assert json.load(open(path))["k"]["ms"] == 0.2
    t2 = autotune.Table.load(path)
    assert t2.lookup("k") == t.lookup("k")
    with pytest.raises(ValueError):
        t.record("empty", [])


def test_choose_falls_back_to_the_size_rule():
    ro = _ro([3] * 100)
    assert autotune.choose(ro, None)["schedule"] == "auto"
    t = autotune.Table()
    assert autotune.choose(ro, t)["schedule"] == "auto"
    t.record(autotune.shape_class(ro), [{"schedule": "group_mapped", "threads": 0, "items_per_thread": 0,
                                         "group_size": 8, "ms": 0.1}])
    assert autotune.choose(ro, t) == {"schedule": "group_mapped", "threads": 0, "items_per_thread": 0, "group_size": 8}
    assert autotune.choose(ro, t, "bf16")["schedule"] == "auto"  # the class includes the value type


@pytest.mark.gpu
def test_tune_measures_every_candidate_and_the_tuned_plan_is_correct(lb, orc):
    import torch

    from gpu_helpers import check_bound, dev, to_dev, vec

    for a in (synth.workload("powerlaw_4k"), synth.stencil7_csr(24, seed=3)):
        ro, ci, v = to_dev(a)
        x = vec(a.n, 401)
        t = autotune.Table()
        res = autotune.tune(ro, ci, v, dev(x), a.n, reps=5, table=t)
        assert len(res) == lb.ensure_loaded().lb_tune_candidates()
        assert all(r["ms"] > 0 for r in res)
        assert [r["ms"] for r in res] == sorted(r["ms"] for r in res)
        assert {r["schedule"] for r in res} == {"merge_path", "thread_mapped", "warp_mapped", "group_mapped",
                                                 "block_mapped", "nonzero_split"}
        plan = autotune.plan_for(ro, a.n, t)
        assert plan.info()["schedule"] == res[0]["schedule"]
        y = plan.spmv(ci, v, dev(x))
        torch.cuda.synchronize()
        check_bound(y.cpu().numpy(), orc.spmv(a.row_offsets, a.col_idx, a.values, x),
                    orc.row_absdot(a.row_offsets, a.col_idx, a.values, x), 1e-5)


@pytest.mark.gpu
def test_tune_batched(lb, orc):
    import torch

    from gpu_helpers import check_bound, dev, vec

    b = synth.workload("batched_4096", 0.02)
    x = vec(int(b.ns.sum()), 402)
    t = autotune.Table()
    res = autotune.tune_batched(b.ms, b.ns, b.nnzs, dev(b.row_offsets), dev(b.col_idx), dev(b.values), dev(x),
                                reps=3, table=t)
    assert len(res) == 6
    assert sorted({r["schedule"] for r in res}) == ["merge_path", "thread_mapped"]
    best = res[0]
    plan = autotune.batched_plan_for(b.ms, b.ns, b.nnzs, dev(b.row_offsets), t)
    assert plan.info()["schedule"] == best["schedule"]
    y = plan.spmv(dev(b.col_idx), dev(b.values), dev(x))
    torch.cuda.synchronize()
    check_bound(y.cpu().numpy(), orc.batched_spmv(b, x), orc.batched_row_absdot(b, x), 1e-5)
    assert len(t.entries) == 1


def test_lrb_bins():
    b = autotune.lrb_bins(_ro([1, 1, 2, 3, 4, 0, 1000]))
    # nonzeros: lengths 1,1 -> bin 0 (2); 2,3 -> bin 1 (5); 4 -> bin 2 (4); 1000 -> bin 9 (1000)
    assert np.allclose(b[[0, 1, 2, 9]], np.array([2, 5, 4, 1000]) / 1011)
    assert abs(b.sum() - 1) < 1e-12
    assert not autotune.lrb_bins(_ro([0, 0])).any()


def test_roofline_selector():
    calib = {"gathers_per_s": 3e11, "read_GBps": 7000.0, "copy_GBps": 6500.0}
    skewed = _ro([2] * 100000 + [500000])
    uniform = _ro([7] * 400000)
    t = autotune.predict(skewed, 1000, calib)
    assert t["thread_mapped"] > 10 * t["merge_path"]  # one 500k row on one thread
    assert autotune.choose_by_roofline(skewed, 1000, calib) == "merge_path"
    tu = autotune.predict(uniform, 1000, calib)
    assert tu["thread_mapped"] == tu["merge_path"]  # short rows: both at the same ceiling
    assert autotune.choose_by_roofline(uniform, 1000, calib) == "merge_path"  # ties go to merge path
    assert tu["nonzero_split"] > tu["merge_path"]


def test_shipped_gb300_table():
    """The table measured on a GB300 loads, names only schedules and launch shapes the library
    has, and covers the standard workloads' classes (the stencil's winner is thread-mapped,
    the power-law matrices' merge path)."""
    from paper_2212_08964_gb300 import lbspmv

    t = autotune.default_table()
    assert t is not None and t.entries
    for key, e in t.entries.items():
        b = e["best"]
        assert b["schedule"] in lbspmv.SCHEDULES
        if b["schedule"] == "merge_path":
            assert (b["threads"], b["items_per_thread"]) in lbspmv.MERGE_SHAPES
        assert e["ms"] == min(c["ms"] for c in e["candidates"])
    stencil = synth.workload("stencil7_160", 0.05)
    full_stencil_class = "size24-mean5-skew0-lrb2-f32"
    assert full_stencil_class in t.entries
    assert t.lookup(full_stencil_class)["schedule"] == "thread_mapped"
    assert autotune.shape_class(stencil.row_offsets).endswith("-f32")
    assert t.lookup("size26-mean7-skew4-lrb2-f32")["schedule"] == "merge_path"
