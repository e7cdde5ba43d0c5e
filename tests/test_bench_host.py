"""Host-side logic of the benchmark: the clock record kept beside each number."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _line(ts, sm, reasons=("Not Active",) * 4):
    return ", ".join([ts, str(sm), "2070", "812.40", *reasons])


def test_clock_line_parses_timestamp_and_fields():
    ts, f = bench.ClockSampler.parse_line(_line("2026/12/03 01:52:33.125", 2070))
    import datetime
    assert ts == datetime.datetime(2026, 12, 3, 1, 52, 33, 125000).timestamp()
    assert f[0] == "2070" and f[1] == "2070" and len(f) == 7
    assert bench.ClockSampler.parse_line("garbage") is None


def test_clock_summary_keeps_only_samples_inside_the_region():
    c = bench.ClockSampler(0)
    c.t0, c.t1 = 100.0, 101.0
    act = ("Not Active", "Not Active", "Not Active", "Active")
    hot = ("Active", "Not Active", "Not Active", "Not Active")
    c.samples = [
        (99.5, ["1200", "2070", "500", *hot]),      # before the region: ignored
        (100.2, ["2070", "2070", "900", *act]),
        (100.5, ["2055", "2070", "950", *act]),
        (100.9, ["2040", "2070", "990", "Not Active", "Not Active", "Not Active", "Not Active"]),
        (101.5, ["900", "2070", "400", *hot]),      # after: ignored
    ]
    s = c.summary()
    assert s["samples"] == 3 and s["window"] == "timed region"
    assert s["sm_mhz"] == 2055.0 and s["sm_mhz_min"] == 2040.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]


def test_clock_summary_short_region_takes_nearest_samples():
    c = bench.ClockSampler(0)
    c.t0, c.t1 = 100.00, 100.01
    c.samples = [(99.0, ["1000", "2070", "1", "Not Active", "Not Active", "Not Active", "Not Active"]),
                 (100.02, ["2070", "2070", "1", "Not Active", "Not Active", "Not Active", "Not Active"]),
                 (99.98, ["2060", "2070", "1", "Not Active", "Not Active", "Not Active", "Not Active"])]
    s = c.summary()
    assert s["window"] == "nearest to the timed region" and s["samples"] == 2
    assert s["sm_mhz"] == 2065.0


def test_clock_summary_without_samples():
    c = bench.ClockSampler(0)
    c.t0, c.t1 = 1.0, 2.0
    assert c.summary()["reasons"] == ["unsampled"]


def test_reference_arm_line(tmp_path):
    """The reference arm (the oracle on the host) prints one JSON line with the
    contract's keys, on the default workload's name, after its warm-up."""
    import json
    import subprocess
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "1"], capture_output=True, text=True, timeout=600,
                         cwd=str(tmp_path))
    assert out.returncode == 0, out.stderr
    lines = out.stdout.splitlines()
    assert len(lines) == 1 and lines[0].startswith("{"), out.stdout   # stdout holds the JSON line only
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "attempts/s"
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 1 and d["higher_is_better"] is True
    assert d["config"]["workload"] == bench.WORKLOAD
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "attempts/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_timed_window_holds_the_most_control_events():
    """The K-step window starts at or after step 40, ends within the
    schedule, and holds as many cluster-move and reheat iterations of the
    runs as any window can (earliest on ties)."""
    ev = [{"ncm": [121, 160, 233], "reheat": [120, 159, 232], "restart": [399]},
          {"ncm": [301], "reheat": [300], "restart": [399]}]
    for K in (5, 20, 60):
        a = bench.choose_window(ev, K)
        assert 40 <= a <= bench.STEPS_SCHEDULE - K
        marks = [t for e in ev for t in e["ncm"] + e["reheat"]]
        got = sum(1 for t in marks if a <= t < a + K)
        for b in range(40, bench.STEPS_SCHEDULE - K + 1):
            assert sum(1 for t in marks if b <= t < b + K) <= got
    assert bench.choose_window(ev, 20) == 102        # the earliest window holding steps 120 and 121
    # no events at all: the window starts at step 40
    assert bench.choose_window([{"ncm": [], "reheat": [], "restart": []}], 20) == 40
    s = bench.window_summary(ev, 115, 20, [{"ncm_flipped": 5}, {"ncm_flipped": 0}],
                             [{"ncm_flipped": 17}, {"ncm_flipped": 0}])
    assert s["first"] == 115 and s["last"] == 134
    assert s["ncm_steps"] == [[121], []] and s["reheat_steps"] == [[120], []]
    assert s["ncm_spins_flipped"] == [12, 0]


def test_sweep_roofline_counts():
    """The ALU roofline of a sweep window: the method's count (18 operations
    per attempt, 1 + 2 x degree per counted flip) and the pull sweep's count
    (18 + 2 x degree per attempt, no flip term) over the summed launch time,
    against 152 SMs x 128 lanes x the clock."""
    import workloads as W
    inst = W.torus(10, 10, signed=True, seed=1)        # degree 4
    att = bench.R * inst.n * bench.SWEEPS * 3
    flips = att // 20
    r = bench.sweep_roofline(inst, 3, {"flips": 0}, {"flips": flips, "ms": 2.0, "launches": 3}, 2000.0)
    peak = 152 * 128 * 2000e6 / 1e12
    assert abs(r["peak"] - peak) < 1e-9
    assert abs(r["achieved"] - (att * 18 + flips * 9) / 2e-3 / 1e12) < 1e-9
    assert abs(r["frac"] - r["achieved"] / peak) < 1e-12
    assert r["pull_count"]["ops_per_attempt"] == 26.0
    assert abs(r["pull_count"]["frac"] - att * 26 / 2e-3 / 1e12 / peak) < 1e-12
    assert r["launches"] == 3 and abs(r["avg_launch_ms"] - 2.0 / 3) < 1e-12
    assert abs(r["flip_fraction"] - flips / att) < 1e-12
