"""Host-side logic of bench.py that needs no GPU: the clock sampler (run
against a stand-in nvidia-smi that prints fixed samples) and the lookup of
the measured peak bandwidth."""
import json
import os
import stat
import time

import bench

SAMPLE = "0, {sm}, 2070, 500.0, {act}, {hw}, Not Active, Not Active, {pc}\n"


def _fake_smi(tmp_path, delay: float, lines: list[str]) -> str:
    """A directory holding an executable `nvidia-smi` that waits `delay`
    seconds, then prints `lines` over and over every 20 ms."""
    d = tmp_path / "bin"
    d.mkdir()
    body = "".join(f"printf '%s'\n" % ln.replace("\n", "\\n") for ln in lines)
    script = f"#!/bin/sh\nsleep {delay}\nwhile true; do\n{body}sleep 0.02\ndone\n"
    exe = d / "nvidia-smi"
    exe.write_text(script)
    exe.chmod(exe.stat().st_mode | stat.S_IXUSR | stat.S_IXGRP | stat.S_IXOTH)
    return str(d)


def test_clock_sampler_waits_for_the_first_sample(tmp_path, monkeypatch):
    d = _fake_smi(tmp_path, 0.4, [SAMPLE.format(sm=2070, act="Not Active", hw="Not Active",
                                                pc="Not Active")])
    monkeypatch.setenv("PATH", d + os.pathsep + os.environ["PATH"])
    t0 = time.perf_counter()
    with bench.ClockSampler(0) as c:
        entered = time.perf_counter() - t0
        time.sleep(0.1)
    assert entered >= 0.35                  # the start-up stayed outside the region
    s = c.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == [] and s["samples"] >= 1


def test_clock_sampler_reports_throttle_reasons(tmp_path, monkeypatch):
    lines = [SAMPLE.format(sm=1800, act="Active", hw="Active", pc="Not Active"),
             SAMPLE.format(sm=1900, act="Active", hw="Not Active", pc="Active")]
    d = _fake_smi(tmp_path, 0.0, lines)
    monkeypatch.setenv("PATH", d + os.pathsep + os.environ["PATH"])
    with bench.ClockSampler(0) as c:
        time.sleep(0.15)
    s = c.summary()
    assert set(s["reasons"]) == {"hw_slowdown", "sw_power_cap"}
    assert 1800.0 <= s["sm_mhz"] <= 1900.0


def test_clock_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    t0 = time.perf_counter()
    with bench.ClockSampler(0) as c:
        pass
    assert time.perf_counter() - t0 < 1.0
    assert c.summary() is None


def test_peaks_measured_file_and_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.peaks() == (bench.PEAK_FALLBACK_GBS, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6693.8}))
    assert bench.peaks() == (6693.8, "measured")
