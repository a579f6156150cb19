"""Host logic of the benchmark, on CPU: the clock record that decides
whether a timed run stands (median SM clock, highest max clock, throttle
reasons seen), the peak it divides by, and the whole-job rate."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

# index, clocks.sm, clocks.max.sm, power.draw, reasons.active, hw_slowdown,
# hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap
ROW = "0, {sm}, 2070, 900.5, 0x0000000000000000, {hw}, {hwt}, {swt}, {cap}\n"


def _row(sm, hw="Not Active", hwt="Not Active", swt="Not Active", cap="Not Active"):
    return ROW.format(sm=sm, hw=hw, hwt=hwt, swt=swt, cap=cap)


def test_clean_run():
    got = bench.parse_clocks([_row(2070), _row(2055), _row(2070)])
    assert got == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 3}


def test_reasons_seen_in_any_sample():
    rows = [_row(2070), _row(1900, cap="Active"), _row(1500, hwt="Active"), _row(2070)]
    got = bench.parse_clocks(rows)
    assert got["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert got["sm_mhz"] == 1985.0 and got["samples"] == 4


def test_rows_that_do_not_parse_are_skipped():
    rows = ["", "garbage\n", "0, [N/A], 2070, 1, 0x0, Not Active, Not Active, Not Active, Not Active\n",
            _row(2000, hw="Active")]
    got = bench.parse_clocks(rows)
    assert got == {"sm_mhz": 2000.0, "sm_max_mhz": 2070.0, "reasons": ["hw_slowdown"], "samples": 1}


def test_no_samples():
    assert bench.parse_clocks([]) == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_peak_and_rate():
    peak, kind = bench.peaks()
    assert peak > 0 and kind in ("measured", "fallback")
    assert bench.whole_job_rate(100, 4, 2.0) == 200.0


def test_sampler_stop_reads_and_removes_its_file(tmp_path):
    """stop() on a sampler whose nvidia-smi has written two rows: the record
    is parsed and the temporary file removed."""
    class FakeProc:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    path = tmp_path / "clocks.csv"
    path.write_text(_row(2070) + _row(2040, cap="Active"))
    s = bench.ClockSampler(0)
    s.proc, s.path = FakeProc(), str(path)
    got = s.stop()
    assert got == {"sm_mhz": 2055.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 2}
    assert not path.exists()


def test_sampler_without_nvidia_smi():
    assert bench.ClockSampler(0).stop()["reasons"] == ["unavailable"]
