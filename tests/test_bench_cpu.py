"""Host logic of bench.py that needs no GPU: the clock record keeps the
nvidia-smi samples stamped inside the timed region."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _row(mhz, active=("Not Active",) * 4, mx=2070):
    return [str(mhz), str(mx), "900.0", "0x0", *active]


def test_clock_record_keeps_the_samples_of_the_timed_region():
    rows = [(0.9, _row(1000)), (1.0, _row(2070)), (1.1, _row(2055)), (1.2, _row(2070)),
            (1.6, _row(900, ("Active", "Not Active", "Not Active", "Not Active")))]
    c = bench.summarize_clocks(rows, 1.0, 1.25)
    assert c["samples"] == 3 and c["samples_in_region"] == 3
    assert c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == []  # the slowdown sample came after the region


def test_clock_record_reports_throttle_reasons_inside():
    rows = [(1.0, _row(1980, ("Not Active", "Not Active", "Not Active", "Active"))),
            (1.1, _row(2070))]
    c = bench.summarize_clocks(rows, 0.95, 1.2)
    assert c["reasons"] == ["sw_power_cap"] and c["samples"] == 2


def test_clock_record_of_a_short_region_takes_the_neighbours():
    rows = [(0.5, _row(1500)), (0.9, _row(2070)), (1.3, _row(2040)), (1.7, _row(1200))]
    c = bench.summarize_clocks(rows, 1.0, 1.1)
    assert c["samples_in_region"] == 0 and c["samples"] == 2
    assert c["sm_mhz"] == statistics_median([2070.0, 2040.0])


def test_clock_record_without_samples_is_none():
    assert bench.summarize_clocks([], 0.0, 1.0) is None
    assert bench.summarize_clocks([(0.5, ["N/A"] * 8)], 0.0, 1.0) is None


def statistics_median(xs):
    xs = sorted(xs)
    k = len(xs) // 2
    return xs[k] if len(xs) % 2 else (xs[k - 1] + xs[k]) / 2
