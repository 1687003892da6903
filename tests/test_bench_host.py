"""Host logic of the benchmark, without a GPU: the algorithmic work units of
a frame's stages (the roofline numerators), the roofline arithmetic, the
parsing of the sampled clocks and their throttle reasons, and the job rate
of the replicas."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_frame_units_follow_the_per_unit_figures():
    R, n_vis, K, ne, nc, tiles, kp, pixels = 1000, 900, 5000, 70_000, 30_000, 64, 2, 16_384
    u = bench.frame_units(R, n_vis, K, ne, nc, tiles, kp, sh_bytes=192, pixels=pixels)
    par = 32 + 192
    assert u["project"] == ("hbm", 12 * R + (par + 68) * n_vis)
    assert u["blend_fwd"] == ("alu", 7 * ne + 11 * nc)
    assert u["blend_bwd"] == ("alu", 7 * ne + 40 * nc)
    assert u["project_bwd"] == ("hbm", (2 * (12 + par) + 48 + 4) * R)
    assert u["g2d_clear"] == ("hbm", 48 * R)
    assert u["tile_order"] == ("hbm", 4 * pixels + 12 * tiles)
    dup = u["duplicate_sort"]
    assert dup[0] == "hbm"
    # the sort part grows by 16 bytes per key and pass
    u3 = bench.frame_units(R, n_vis, K, ne, nc, tiles, kp + 1, sh_bytes=192, pixels=pixels)
    assert u3["duplicate_sort"][1] - dup[1] == 16 * K


class _FakePeaks(bench.Peaks):
    def __init__(self):  # no device: the denominators are set by hand
        self.hbm, self.hbm_src = 6000.0, "test"
        self.alu, self.alu_src = 40.0, "test"


def test_roofline_entries_and_the_lower_bound():
    p = _FakePeaks()
    e = p.entry("hbm", 6e9, 2.0)  # 6 GB in 2 ms = 3000 GB/s
    assert e["unit"] == "GB/s" and e["achieved"] == pytest.approx(3000.0) and e["frac"] == pytest.approx(0.5)
    a = p.entry("alu", 8e9, 1.0)  # 8 G lane-ops in 1 ms = 8 T/s
    assert a["unit"] == "Tops/s" and a["frac"] == pytest.approx(0.2)
    # 6 GB at 6000 GB/s (1 ms) + 40 G ops at 40 T/s (1 ms)
    assert p.lower_bound_ms([("hbm", 6e9), ("alu", 40e9)]) == pytest.approx(2.0)


def test_clock_rows_are_parsed_with_their_throttle_reasons():
    c = bench.ClockSampler(0)
    c.rows = [["0", "2070", "2070", "900.1", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"],
              ["0", "2055", "2070", "1390.0", "0x4", "Not Active", "Not Active", "Not Active", "Active"],
              ["0", "[N/A]", "2070", "1000.0", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"],
              ["0", "2070", "2070"]]  # a short row is skipped
    s = c.summary()
    assert s["samples"] == 2 and s["sm_mhz"] == pytest.approx(2062.5) and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]
    c.rows = [["0", "1500", "2070", "700", "0x8", "Active", "Not Active", "Active", "Not Active"]]
    assert c.summary()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_job_rate_counts_every_rank():
    assert bench.job_rate(1, 2.0) == pytest.approx(500.0)
    assert bench.job_rate(4, 2.0) == pytest.approx(2000.0)
