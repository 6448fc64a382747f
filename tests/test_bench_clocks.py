"""bench.py's summary of the nvidia-smi clock samples taken during the timed
region: median SM clock, maximum clock and the throttle reasons seen active
(a run with a hardware or thermal slowdown is to be rejected)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

NA, A = "Not Active", "Active"


def _line(sm, mx, hw=NA, hwt=NA, swt=NA, pcap=NA):
    return ", ".join(["0", str(sm), str(mx), "1100.5", "0x0000000000000000", hw, hwt, swt, pcap])


def test_median_max_and_no_reasons():
    s = bench.Clocks.summarise([_line(1980, 2070), _line(2070, 2070), _line(1900, 2070)])
    assert s == {"sm_mhz": 1980.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 3}


def test_reasons_are_collected():
    s = bench.Clocks.summarise([_line(1400, 2070, pcap=A), _line(1300, 2070, hwt=A), _line(2000, 2070)])
    assert s["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"] and s["sm_mhz"] == 1400.0


def test_malformed_lines_are_skipped():
    s = bench.Clocks.summarise(["", "garbage", "0, [N/A], 2070, 1, 0x0, Active, x, y, z", _line(1800, 2070)])
    assert s["samples"] == 1 and s["sm_mhz"] == 1800.0 and s["reasons"] == []
    assert bench.Clocks.summarise([]) == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
