"""Host logic of bench.py (CPU): the event-count arithmetic behind the roofline, the
co-bounds and their binding resource, the capture-to-source matching of the traffic
figure, and the clock summary.  No GPU and no library call."""
import json
import os

import numpy as np
import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WALK = os.path.join(ROOT, "paper_1711_03244_gb300", "csrc", "walk.cu")

STATS = {"scatter": 1000, "face": 200, "fresnel": 10, "flush": 150, "photons": 2}


def test_algorithmic_ops_follow_the_per_event_table():
    # segments = scatter + face + photon launches, hops = scatter + launches (by hand)
    want = (35 * 1202 + 17 * 1002 + 65 * 1000 + 15 * 200 + 25 * 10 + 3 * 150 + 60 * 2)
    assert bench.algorithmic_ops(STATS, None) == want
    assert bench.xu_ops(STATS) == 1 * 1202 + 1 * 1002 + 8 * 1000 + 4 * 10


def _rates(**over):
    r = {"ffma": 4e13, "lg2": 5e12, "ex2": 1e13, "rsqrt": 5e12, "sin": 5e12,
         "red_f64_c2": 2e11, "red_f64_c3": 2e10}
    r.update(over)
    return r


def test_co_bounds_name_the_slowest_measured_resource():
    n, ms = 2, 1e-3                                     # 2 photons in 1 us: 2000 photons/ms
    cb = bench.co_bounds(STATS, n, ms, _rates(sin=1e9), "c2", 40.0)
    b = cb["bounds"]
    assert cb["achieved_photons_per_ms"] == pytest.approx(2000.0)
    for k, v in b.items():
        assert v["bound_photons_per_ms"] == pytest.approx(v["rate"] / v["per_photon"] / 1e3)
        assert v["frac"] == pytest.approx(2000.0 / v["bound_photons_per_ms"])
    # the special-function rate is the slowest of lg2 / ex2 / rsqrt / sin
    assert b["xu"]["rate"] == 1e9 and cb["binding"] == "xu"
    assert "hbm" not in b and "atomics_spread_over_map" not in cb
    assert cb["walk_atomics_per_s"] == pytest.approx(150 / 1e-6)


def test_co_bounds_nominal_issue_never_binds_and_hbm_joins_with_traffic():
    # a nominal peak far below every measured rate still does not become the binding one
    cb = bench.co_bounds(STATS, 2, 1.0, _rates(), "c3", 1e-9, traffic=2e6, hbm_gbs=1e-3)
    assert cb["binding"] == "hbm"
    assert cb["bounds"]["hbm"]["per_photon"] == pytest.approx(1e6)
    spread = cb["atomics_spread_over_map"]
    assert spread["rate"] == 2e10
    assert spread["bound_photons_per_ms"] == pytest.approx(2e10 / 75 / 1e3)


def test_code_hash_ignores_comments_and_blank_lines_only(tmp_path):
    a = tmp_path / "a.cu"
    a.write_text("int f(int x)\n{\n    return x + 1;\n}\n")
    b = tmp_path / "b.cu"
    b.write_text("// a comment\nint f(int x)   \n{\n\n    return x + 1;  // trailing note\n}\n\n")
    c = tmp_path / "c.cu"
    c.write_text("int f(int x)\n{\n    return x + 2;\n}\n")
    assert bench.walk_code_hash(str(a)) == bench.walk_code_hash(str(b))
    assert bench.walk_code_hash(str(a)) != bench.walk_code_hash(str(c))


def test_traffic_is_read_only_from_a_capture_of_the_current_code(tmp_path):
    h = bench.walk_code_hash(WALK)
    full = tmp_path / "full.md"
    full.write_text(f"walk.cu code sha256[:16] at capture (note): {h}\ndram bytes per full launch: 1.5e+08\n")
    assert bench.walk_traffic(str(full)) == 1.5e8
    per = tmp_path / "per.md"
    per.write_text(f"walk.cu code sha256[:16] at capture: {h}\ndram bytes per photon: 9000.5\n")
    assert bench.walk_traffic(str(per), photons=10 ** 9) == pytest.approx(9000.5e9)
    assert bench.walk_traffic(str(per)) is None                 # per-photon form needs a count
    stale = tmp_path / "stale.md"
    stale.write_text("walk.cu code sha256[:16] at capture: 0123456789abcdef\ndram bytes per full launch: 1e8\n")
    assert bench.walk_traffic(str(stale)) is None
    assert bench.walk_traffic(str(tmp_path / "missing.md")) is None


def test_clock_summary_reports_median_maximum_and_reasons():
    s = bench.ClockSampler(0)
    s.lines = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
               "0, 2000, 2070, 1350.0, 0x4, Not Active, Not Active, Not Active, Active",
               "0, 1990, 2070, 1360.0, 0x4, Not Active, Not Active, Not Active, Active",
               "garbage line", "0, N/A, 2070, 0, 0x0, a, b, c, d"]
    out = s.summary()
    assert out["sm_mhz"] == float(np.median([2070, 2000, 1990]))
    assert out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"] and out["samples"] == 3
    assert bench.ClockSampler(0).summary()["reasons"] == ["unavailable"]


def test_peaks_take_the_measured_file():
    p = bench.peaks()
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        assert p["source"] == "measured"
        assert p["hbm_gbs"] == float(d["hbm_gbs"]) and p["bf16_tflops"] == float(d["bf16_tflops"])
    else:
        assert p["source"] == "fallback" and p["hbm_gbs"] == 6800.0
