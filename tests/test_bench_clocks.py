"""Host logic of the benchmark's clock record: nvidia-smi samples are kept only inside the timed
region's window, throttle reasons are collected from those samples, and a region shorter than the
sampling interval falls back to the nearest sample (checked on canned nvidia-smi output)."""
import datetime

import bench


def _canned(t0, n, sm=lambda k: 2070, reason=lambda k: "Not Active"):
    lines = []
    for k in range(n):
        ts = (t0 + datetime.timedelta(milliseconds=50 * k)).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
        lines.append("%s, 0, %d, 2070, 512.5, 0x0, Not Active, Not Active, Not Active, %s" % (ts, sm(k), reason(k)))
    return "\n".join(lines)


def test_samples_outside_the_timed_window_are_dropped():
    t0 = datetime.datetime(2026, 1, 1, 12, 0, 0)
    c = bench.ClockSampler(0)
    # warm-up at low clocks (k < 4), timed region at 2070 MHz, a power-cap event after it
    c.out = _canned(t0, 20, sm=lambda k: 1200 if k < 4 else 2070,
                    reason=lambda k: "Active" if k >= 17 else "Not Active")
    c.t0 = t0 + datetime.timedelta(milliseconds=300)
    c.t1 = t0 + datetime.timedelta(milliseconds=700)
    s = c.summary()
    assert s["sm_mhz"] == 2070 and s["sm_max_mhz"] == 2070 and s["reasons"] == []
    assert s["window"] == "timed region" and 8 <= s["samples"] <= 12


def test_throttle_reason_inside_the_window_is_reported():
    t0 = datetime.datetime(2026, 1, 1, 12, 0, 0)
    c = bench.ClockSampler(0)
    c.out = _canned(t0, 10, reason=lambda k: "Active" if k == 5 else "Not Active")
    c.t0, c.t1 = t0, t0 + datetime.timedelta(milliseconds=450)
    assert c.summary()["reasons"] == ["sw_power_cap"]


def test_short_region_takes_the_nearest_sample():
    t0 = datetime.datetime(2026, 1, 1, 12, 0, 0)
    c = bench.ClockSampler(0)
    c.out = _canned(t0, 4, sm=lambda k: 2000 + k)
    c.t0 = t0 + datetime.timedelta(milliseconds=1000)
    c.t1 = t0 + datetime.timedelta(milliseconds=1001)
    s = c.summary()
    assert s["samples"] == 1 and s["sm_mhz"] == 2003 and s["window"].startswith("nearest")


def test_no_output_is_unsampled():
    c = bench.ClockSampler(0)
    c.out = ""
    assert c.summary()["reasons"] == ["unsampled"]
