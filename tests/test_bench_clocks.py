"""bench.py's clock record: only nvidia-smi samples taken inside the timed region count (CPU)."""
import datetime
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402


def row(t, mhz, reasons=("Not Active",) * 4):
    stamp = datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    return ", ".join([stamp, "0", str(mhz), "2070", "900.5", "0x0000000000000000"] + list(reasons))


def test_only_samples_inside_the_timed_region_count():
    t0 = 1.8e9
    lines = [row(t0 - 0.4, 900), row(t0 - 0.2, 1200)]  # idle samples before the region
    lines += [row(t0 + 0.1 * i, 2070) for i in range(5)]
    lines += [row(t0 + 0.7, 600, ("Not Active", "Active", "Not Active", "Not Active"))]  # after it
    out = bench.summarize_clocks(lines, t0, t0 + 0.45)
    assert out["samples"] == 5 and out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == []


def test_throttle_reasons_inside_the_region_are_reported():
    t0 = 1.8e9
    lines = [row(t0 + 0.1, 1900, ("Not Active", "Not Active", "Not Active", "Active")),
             row(t0 + 0.2, 1800, ("Active", "Not Active", "Not Active", "Not Active")),
             "garbage line", ""]
    out = bench.summarize_clocks(lines, t0, t0 + 0.3)
    assert out["samples"] == 2 and out["sm_mhz"] == 1850.0
    assert out["reasons"] == ["hw_slowdown", "sw_power_cap"]


def test_a_region_without_samples_says_so():
    t0 = 1.8e9
    out = bench.summarize_clocks([row(t0 - 5.0, 2070)], t0, t0 + 0.1)
    assert out["samples"] == 0 and out["sm_mhz"] is None
    assert out["reasons"] == ["no samples in the timed region"] and out["samples_total"] == 1
