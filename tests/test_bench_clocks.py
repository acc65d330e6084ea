"""Host logic of bench.py's clock record: nvidia-smi samples are kept when their own
timestamps fall inside the timed window; throttle reasons are collected from those samples;
with no sample inside (a window shorter than the sampling interval, or unparsable stamps)
the whole run's samples are reported and the record says so."""
import datetime
import os
import time

import bench


def _line(t, sm, reasons=()):
    stamp = datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    flags = ["Active" if nm in reasons else "Not Active" for nm in bench.ClockSampler.NAMES]
    return ", ".join([stamp, "0", str(sm), "2070", "800.0", "0x0", *flags])


def test_samples_inside_the_window_only():
    t = time.time()
    lines = [_line(t - 1.0, 1200.0, ("hw_slowdown",)), _line(t + 0.02, 2070.0, ("sw_power_cap",)),
             _line(t + 0.07, 2055.0), _line(t + 3.0, 900.0, ("sw_thermal_slowdown",)), "not a sample"]
    out = bench.ClockSampler.parse(lines, t, t + 0.08)
    assert out["window"] == "timed region" and out["samples"] == 2
    assert out["sm_mhz"] == (2070.0 + 2055.0) / 2 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]


def test_whole_run_when_the_window_holds_no_sample():
    t = time.time()
    lines = [_line(t - 1.0, 2070.0), _line(t + 1.0, 2070.0, ("hw_thermal_slowdown",))]
    out = bench.ClockSampler.parse(lines, t, t + 0.01)
    assert out["window"] == "run" and out["samples"] == 2
    assert out["reasons"] == ["hw_thermal_slowdown"]
    bad = [ln.replace("/", "-") for ln in lines]           # unparsable stamps: no window
    assert bench.ClockSampler.parse(bad, t, t + 0.01)["window"] == "run"
    assert bench.ClockSampler.parse([], t, t + 1.0)["sm_mhz"] is None


def test_unstamped_layout():
    lines = ["0, 2070, 2070, 700.0, 0x0, Not Active, Not Active, Not Active, Active"]
    out = bench.ClockSampler.parse(lines, 0.0, 1.0, stamped=False)
    assert out["samples"] == 1 and out["window"] == "run" and out["reasons"] == ["sw_power_cap"]


def _fake_smi(tmp_path, takes_timestamp: bool):
    # a stand-in nvidia-smi on PATH: prints one sample line every 20 ms until terminated,
    # or refuses the timestamp field the way an unknown field is refused
    script = tmp_path / "nvidia-smi"
    script.write_text(
        "#!/usr/bin/env python3\n"
        "import sys, time, datetime\n"
        "q = [a for a in sys.argv if a.startswith('--query-gpu=')][0]\n"
        f"if 'timestamp' in q and not {takes_timestamp}:\n"
        "    sys.exit(2)\n"
        "while True:\n"
        "    row = '0, 2070, 2070, 800.0, 0x0, Not Active, Not Active, Not Active, Not Active'\n"
        "    if 'timestamp' in q:\n"
        "        row = datetime.datetime.now().strftime('%Y/%m/%d %H:%M:%S.%f')[:-3] + ', ' + row\n"
        "    print(row, flush=True)\n"
        "    time.sleep(0.02)\n")
    script.chmod(0o755)


def test_sampler_windows_and_falls_back(tmp_path, monkeypatch):
    for takes in (True, False):
        d = tmp_path / str(takes)
        d.mkdir()
        _fake_smi(d, takes)
        monkeypatch.setenv("PATH", f"{d}{os.pathsep}{os.environ['PATH']}")
        c = bench.ClockSampler(0)
        c.start()
        time.sleep(0.1)
        c.begin()
        time.sleep(0.2)
        c.end()
        time.sleep(0.1)
        out = c.stop()
        assert c.stamped == takes
        assert out["sm_mhz"] == 2070.0 and out["reasons"] == []
        assert out["window"] == ("timed region" if takes else "run")
        if takes:
            assert 3 <= out["samples"] <= 20
