"""Host logic of bench.py: the clock record taken during the timed region and the
traffic record that belongs to one kernel source and launch variant."""
import hashlib
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_clock_record_median_and_reasons():
    import bench
    lines = [
        "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n",
        "0, 1980, 2070, 1399.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active\n",
        "0, 2070, 2070, 1010.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n",
        "garbage line\n",
        "0, [N/A], 2070, 1010.0, 0x0, Not Active, Not Active, Not Active, Not Active\n",
    ]
    out = bench.Clocks.parse(lines)
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0 and out["samples"] == 3
    assert out["reasons"] == ["sw_power_cap"]
    hot = bench.Clocks.parse(["0, 1500, 2070, 1400, 0x8, Active, Not Active, Active, Not Active\n"])
    assert hot["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    assert bench.Clocks.parse(["no samples\n"]) is None


def _record(tmp_path, source_text, digest=None):
    (tmp_path / "profiles").mkdir()
    src = tmp_path / "kernel.cu"
    src.write_text(source_text)
    rec = {"source": "kernel.cu",
           "source_sha256": digest or hashlib.sha256(source_text.encode()).hexdigest(),
           "captures": {"31": {"dram_bytes_read_per_launch": 1000, "dram_bytes_write_per_launch": 24}}}
    (tmp_path / "profiles" / "rec.json").write_text(json.dumps(rec))
    return src


def test_traffic_record_per_variant_and_source(tmp_path):
    import bench
    src = _record(tmp_path, "kernel v1\n")
    assert bench.recorded_traffic(31, "rec.json", root=str(tmp_path)) == 1024
    assert bench.recorded_traffic(30, "rec.json", root=str(tmp_path)) is None      # not captured
    assert bench.recorded_traffic(31, "missing.json", root=str(tmp_path)) is None
    src.write_text("kernel v2\n")                                                   # source changed
    assert bench.recorded_traffic(31, "rec.json", root=str(tmp_path)) is None


def test_whole_job_rate_is_units_over_slowest_rank():
    import bench
    assert bench.whole_job_rate(1e9, 10, 4, 2000.0) == pytest.approx(4 * 1e9 * 10 / 2.0)
