"""Host helpers of bench.py that need no GPU: the clock record of the timed
region (parsed from nvidia-smi's CSV), the peak lookup and the line contract's
derived figures."""
import importlib.util
import json
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_record_median_max_and_reasons():
    b = _bench()
    cs = b.ClockSampler(0)
    cs.proc = _FakeProc()
    # index, clocks.sm, clocks.max.sm, power.draw, active mask, hw_slowdown,
    # hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap
    cs.lines = [
        "0, 2070, 2070, 905.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1965, 2070, 1398.7, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2040, 2070, 1201.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "",
        "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "truncated, line",
    ]
    r = cs.stop()
    assert r["sm_mhz"] == 2040.0 and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == ["sw_power_cap"] and r["samples"] == 3


def test_clock_record_flags_thermal_and_hw_slowdown():
    b = _bench()
    cs = b.ClockSampler(0)
    cs.proc = _FakeProc()
    cs.lines = ["0, 1500, 2070, 1400, 0x48, Active, Not Active, Active, Not Active"]
    r = cs.stop()
    assert r["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_clock_record_without_nvidia_smi():
    b = _bench()
    r = b.ClockSampler(0).stop()
    assert r["sm_mhz"] is None and r["reasons"] == ["nvidia-smi unavailable"]


def test_peaks_read_the_measured_file_else_the_fallback(tmp_path, monkeypatch):
    b = _bench()
    hbm, kind, j = b.peaks()
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        assert kind == "measured" and hbm == json.load(open(path)).get("hbm_gbs", 6800.0)
    else:
        assert (hbm, kind) == (6800.0, "fallback")
    monkeypatch.setattr(b, "ROOT", str(tmp_path))
    assert b.peaks()[:2] == (6800.0, "fallback")
