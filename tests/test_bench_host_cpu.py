"""Host logic of bench.py that decides what a bench line says about its own
validity: the clock record taken during the timed region (median SM clock,
throttle reasons seen), the median and spread of the repeated timings, and the
bandwidth peak the roofline fraction divides by."""
import json
import math

import bench

ROW = "0, {sm}, 2070, {pw}, 0x0, {hw}, {hwt}, {swt}, {cap}\n"


def _sampler(tmp_path, rows):
    p = tmp_path / "clocks.csv"
    p.write_text("".join(rows))
    s = bench.ClockSampler(0)
    s.path = str(p)
    return s


def test_clock_summary_median_max_and_reasons(tmp_path):
    rows = [ROW.format(sm=2070, pw=400, hw="Not Active", hwt="Not Active", swt="Not Active", cap="Not Active"),
            ROW.format(sm=2055, pw=455, hw="Not Active", hwt="Not Active", swt="Not Active", cap="Active"),
            ROW.format(sm=2070, pw=430, hw="Not Active", hwt="Not Active", swt="Not Active", cap="Not Active")]
    out = _sampler(tmp_path, rows).summary()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["samples"] == 3 and out["power_w_max"] == 455.0
    assert out["reasons"] == ["sw_power_cap"]  # kept and noted, not a rejection reason


def test_clock_summary_names_every_slowdown_seen(tmp_path):
    rows = [ROW.format(sm=1400, pw=300, hw="Active", hwt="Not Active", swt="Not Active", cap="Not Active"),
            ROW.format(sm=1500, pw=310, hw="Not Active", hwt="Active", swt="Active", cap="Not Active")]
    out = _sampler(tmp_path, rows).summary()
    assert out["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert out["sm_mhz"] == 1450.0  # (median of two samples: their mean)


def test_clock_summary_tolerates_missing_values_and_no_samples(tmp_path):
    rows = [ROW.format(sm="[N/A]", pw="[N/A]", hw="Not Active", hwt="Not Active", swt="Not Active",
                       cap="Not Active"),
            ROW.format(sm=2070, pw=420, hw="Not Active", hwt="Not Active", swt="Not Active", cap="Not Active"),
            "garbled line\n"]
    out = _sampler(tmp_path, rows).summary()
    assert out["samples"] == 2 and out["sm_mhz"] == 2070.0 and out["reasons"] == []
    empty = _sampler(tmp_path, []).summary()
    assert empty["samples"] == 0 and empty["sm_mhz"] is None and empty["reasons"] == ["no nvidia-smi samples"]


def test_spread_is_median_and_relative_range():
    s = bench.spread([0.0021, 0.0019, 0.0020, 0.0030, 0.0020])
    assert math.isclose(s["median_ms"], 2.0) and math.isclose(s["min_ms"], 1.9) and math.isclose(s["max_ms"], 3.0)
    assert math.isclose(s["spread"], (0.0030 - 0.0019) / 0.0020) and s["reps"] == 5


def test_measured_peak_and_its_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6793.4, "bf16_tflops": 1900}))
    assert bench.measured_peaks() == (6793.4, "measured")
