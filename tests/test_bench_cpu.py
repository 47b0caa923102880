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


def test_cpu_baseline_child_times_one_full_oracle_realization():
    # The oracle runs in a child process on a host core beside the GPU legs;
    # its rate is voxels per second of one whole realization.
    p = dict(bench.rank_workload(0, 24))
    c = bench.finish_cpu_baseline(bench.start_cpu_baseline(p), p)
    assert c["kind"] == "oracle" and c["cores"] == 1
    assert c["host_cores"] >= 1
    assert c["value"] is not None and c["value"] > 0
    assert "24^3" in c["sample"]


def test_step_byte_model_matches_its_definition():
    # 4 B read + 36 B gather + 36 B prune test per front voxel, 4 B per voxel
    # of the next front, 4 B atomicOr + 36 B prune test per claim.
    assert bench.BYTES_PER_FRONT_VOXEL + bench.BYTES_PER_NEXT_FRONT_VOXEL == 80
    assert bench.BYTES_PER_CLAIM == 40
    # The derived multiply-rate ceiling on 152 SMs at 2070 MHz.
    peak = 152 * bench.INT_MULS_PER_SM_CLOCK * 2070e6 / bench.PHILOX_BLOCK_MULS
    assert abs(peak - 503.4e9) < 0.1e9
