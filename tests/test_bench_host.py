"""Host-side logic of bench.py that decides what a measurement reports (no GPU).

The clock summary keeps only the samples of the timed region, reports the median
SM clock and every throttle reason seen active there; the cell count of a stream
is the number of admissible window pairs.
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _row(sm, mx, hw="Not Active", hwt="Not Active", swt="Not Active", pcap="Not Active"):
    # index, clocks.sm, clocks.max.sm, power.draw, reasons.active, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap
    return ["0", str(sm), str(mx), "900.0", "0x0", hw, hwt, swt, pcap]


def _sampler(rows, window=None):
    s = bench.ClockSampler(0)
    s.rows = rows
    s.window = window
    return s


def test_clock_summary_keeps_the_timed_region_and_its_reasons():
    rows = [(0.0, _row(1200, 2070, hw="Active")),        # before the region: ignored
            (1.0, _row(2070, 2070)),
            (1.1, _row(2070, 2070, pcap="Active")),
            (1.2, _row(1980, 2070)),
            (3.0, _row(600, 2070, hwt="Active"))]        # after the region: ignored
    out = _sampler(rows, (0.95, 1.25)).summary()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"] and out["samples"] == 3


def test_a_region_shorter_than_the_sampling_interval_takes_the_nearest_samples():
    rows = [(0.0, _row(2070, 2070)), (0.5, _row(2050, 2070, hwt="Active")), (5.0, _row(100, 2070))]
    out = _sampler(rows, (0.51, 0.52)).summary()
    assert out["samples"] == 2 and "hw_thermal_slowdown" in out["reasons"]
    assert out["sm_mhz"] == 2060.0


def test_no_samples_is_reported_as_unsampled():
    out = _sampler([], (0.0, 1.0)).summary()
    assert out == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}


def test_cells_per_stream_counts_the_admissible_pairs():
    for n, m, excl in [(10, 3, 2), (50, 7, 2), (64, 16, 4), (20, 20, 1), (30, 5, 30)]:
        l = n - m + 1
        brute = sum(1 for i in range(l) for j in range(i, l) if j - i >= excl)
        assert bench.cells_per_stream(n, m, excl) == brute, (n, m, excl)
