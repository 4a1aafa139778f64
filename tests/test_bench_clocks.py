"""bench.py's clock record on CPU: a fake nvidia-smi log with timestamps is split into the
samples inside the timed region and those of the loaded window around it, and the throttle
reasons of either are reported."""
import datetime
import os
import sys
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


class _Proc:
    def poll(self):
        return 0


def _sampler(rows, t_start, t_end, t_hold):
    c = bench.ClockSampler(0)
    fd, c.path = tempfile.mkstemp(suffix=".csv")
    with os.fdopen(fd, "w") as f:
        for r in rows:
            f.write(", ".join(r) + "\n")
    c.proc = _Proc()
    c.t_start, c.t_end, c.t_hold = t_start, t_end, t_hold
    return c


def _row(t, sm, reasons=()):
    stamp = datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    flags = ["Active" if n in reasons else "Not Active"
             for n in ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")]
    return [stamp, "0", str(sm), "2070", "900.0", "0x0"] + flags


def test_short_region_falls_back_to_the_loaded_window():
    t0 = 1_800_000_000.0
    rows = [_row(t0 - 1.0, 345)]                                   # idle, before the region
    rows += [_row(t0 + 0.005, 2070)]                               # the only sample inside
    rows += [_row(t0 + 0.03 + 0.02 * i, 2055 if i % 2 else 2070, ("sw_power_cap",) if i == 3 else ())
             for i in range(10)]                                  # the untimed hold
    rows += [_row(t0 + 5.0, 345, ("hw_slowdown",))]                # after the window: ignored
    s = _sampler(rows, t0, t0 + 0.016, t0 + 0.22).summary()
    assert s["samples"] == 1
    assert s["window_samples"] == 11
    assert s["basis"].startswith("timed region + untimed hold")
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]


def test_long_region_uses_its_own_samples():
    t0 = 1_800_000_000.0
    rows = [_row(t0 + 0.02 * i, 1900 if i < 5 else 2070, ("hw_thermal_slowdown",) if i == 2 else ())
            for i in range(8)]
    s = _sampler(rows, t0, t0 + 0.15, None).summary()
    assert s["basis"] == "timed region"
    assert s["samples"] == 8
    assert s["sm_mhz"] == 1900.0
    assert "hw_thermal_slowdown" in s["reasons"]
