"""Host logic of bench.py that decides what a JSON line reports: which clock samples
count as taken during the timed region, and the algorithmic byte model of the stages."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _line(mhz, hw="Not Active", cap="Not Active"):
    # index, clocks.sm, clocks.max.sm, power, active, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap
    return f"0, {mhz}, 2070, 900.0, 0x0, {hw}, Not Active, Not Active, {cap}\n"


def test_clock_samples_inside_the_region_and_the_first_after():
    c = bench.ClockSampler(0)
    c.t0, c.t1 = 10.0, 11.0
    c.lines = [(9.5, _line(1000, hw="Active")),      # before: ignored
               (10.2, _line(2070)), (10.7, _line(2060)),
               (11.05, _line(2050, cap="Active")),    # first after the region: kept
               (11.2, _line(800, hw="Active"))]       # later: ignored
    s = c.summary()
    assert s["samples"] == 3
    assert s["sm_mhz"] == 2060.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]


def test_no_samples_reads_unsampled():
    c = bench.ClockSampler(0)
    c.t0, c.t1 = 10.0, 11.0
    c.lines = [(9.0, _line(2070)), (20.0, "garbage\n")]
    s = c.summary()
    assert s["samples"] == 0 and s["reasons"] == ["unsampled"]


def test_stage_bytes_counts_each_buffer_once():
    # one triangle at SH degree 3 (236 B of parameters), one visible item, 3 pairs, 10 pixels
    b = bench.stage_bytes(n=1, views=1, n_vis=1, pairs=3, pixels=10)
    assert b["preprocess"] == 236 + 8 + 88
    assert b["bin_sort"] == 16 + 3 * 20
    assert b["render_fwd"] == 3 * 76 + 10 * 44
    assert b["render_bwd"] == 3 * 72 + 64 + 10 * 20
    assert b["preprocess_bwd"] == 2 * 236 + 8 + 80
    assert bench.stage_bytes(1, 1, 1, 3, 10, loss=False)["render_fwd"] == 3 * 76 + 10 * 20
