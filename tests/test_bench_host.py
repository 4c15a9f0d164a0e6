"""Host-side logic of bench.py, on the CPU: the clock record is summarised
over the timed region only (samples before or after it, and their throttle
reasons, are ignored), an empty record reads "unsampled", the issue-rate
roofline is the instruction count per cell-update times the rate against
152 SMs x 4 schedulers x 32 lanes at the sampled clock, and non-finite
numbers become JSON nulls."""
import datetime
import json
import math
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def stamp(t):
    return datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]


def line(t, sm, mx, power_cap=False, thermal=False):
    act = "Active" if power_cap else "Not Active"
    th = "Active" if thermal else "Not Active"
    return (f"{stamp(t)}, 0, {sm}, {mx}, 900.00 W, 0x0000000000000000, Not Active, {th}, "
            f"Not Active, {act}\n")


def sampler_with(tmp_path, lines, t0, t1):
    cs = bench.ClockSampler(0)
    cs.path = str(tmp_path / "clocks.csv")
    with open(cs.path, "w") as f:
        f.writelines(lines)
    cs.t0, cs.t1 = t0, t1
    return cs


def test_clock_summary_keeps_the_timed_region_only(tmp_path):
    t0 = 1_800_000_000.0
    lines = [line(t0 - 1.0, 1000, 2070, thermal=True)]                 # before: ignored
    lines += [line(t0 + 0.1 * i, sm, 2070, power_cap=(i == 2))
              for i, sm in enumerate((2070, 2055, 2040, 2070, 2070))]
    lines += [line(t0 + 2.0, 900, 2070, thermal=True)]                  # after: ignored
    lines += ["garbage line\n", "a, b, c\n"]
    cs = sampler_with(tmp_path, lines, t0, t0 + 0.45)
    s = cs.summary()
    assert s["samples"] == 5
    assert s["sm_mhz"] == 2070 and s["sm_max_mhz"] == 2070
    assert s["reasons"] == ["sw_power_cap"]
    assert s["timed_region_s"] == pytest.approx(0.45)
    assert cs.summary() is s                     # cached: the record is read once
    assert not os.path.exists(cs.path)


def test_clock_summary_unsampled(tmp_path):
    t0 = 1_800_000_000.0
    cs = sampler_with(tmp_path, [line(t0 - 5.0, 2070, 2070)], t0, t0 + 1.0)
    s = cs.summary()
    assert s["reasons"] == ["unsampled"] and s["sm_mhz"] is None
    assert s["samples_outside_region"] == 1


class FakeClock:
    def __init__(self, mhz):
        self.mhz = mhz

    def summary(self):
        return {"sm_mhz": self.mhz}


def test_issue_roofline_arithmetic():
    per = bench.THREAD_INST_PER_CELL_UPDATE[("mixed", True)]
    ncell, step_s = 4096 * 4096, 5e-3
    r = bench.issue_roofline("mixed", True, ncell, step_s, FakeClock(2000.0))
    peak = 152 * 4 * 32 * 2000e6 / 1e12
    assert r["peak"] == pytest.approx(peak)
    assert r["achieved"] == pytest.approx(per * ncell / step_s / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / peak)
    assert r["bound"] == "alu"
    assert bench.issue_roofline("fp64", True, ncell, step_s, FakeClock(2000.0)) is None


def test_finite_json_nulls_non_finite():
    x = {"a": math.inf, "b": [1.0, math.nan, {"c": -math.inf}], "d": 2, "e": "s"}
    y = bench.finite_json(x)
    assert y == {"a": None, "b": [1.0, None, {"c": None}], "d": 2, "e": "s"}
    json.dumps(y, allow_nan=False)


def test_peaks_reads_the_measured_copy_bandwidth():
    gbs, src = bench.peaks()
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        assert src == "measured" and gbs == float(json.load(open(path))["hbm_gbs"])
    else:
        assert src == "fallback" and gbs == 6800.0
