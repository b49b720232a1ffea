"""Host logic of the benchmark, on CPU: the clock sampler's parsing of
nvidia-smi lines and its timed-region mark, against a stand-in nvidia-smi that
prints prepared lines (no GPU and no real nvidia-smi involved)."""
import os
import stat
import time

import bench

LINE = "0, {sm}, 2070, 900.00, {active}, {hw}, Not Active, {swt}, {cap}\n"


def fake_smi(tmp_path, lines_before, lines_after, gap_s):
    """A script named nvidia-smi printing lines_before at once, then, after
    gap_s seconds, lines_after, then waiting to be terminated."""
    before = "".join(lines_before).replace("'", "")
    after = "".join(lines_after).replace("'", "")
    script = tmp_path / "nvidia-smi"
    script.write_text("#!/bin/sh\n"
                      f"printf '%s' '{before}'\n"
                      f"sleep {gap_s}\n"
                      f"printf '%s' '{after}'\n"
                      "exec sleep 30\n")
    script.chmod(script.stat().st_mode | stat.S_IEXEC)
    return str(tmp_path)


def run_sampler(monkeypatch, path_dir, wait_s):
    monkeypatch.setenv("PATH", path_dir + os.pathsep + os.environ.get("PATH", ""))
    c = bench.ClockSampler(0)
    c.start()
    c.begin()
    time.sleep(wait_s)
    return c.stop()


def test_samples_after_the_mark_only(tmp_path, monkeypatch):
    # an idle line before the timed region, three loaded lines inside it
    before = [LINE.format(sm=1200, active="Active", hw="Not Active", swt="Not Active", cap="Not Active")]
    after = [LINE.format(sm=s, active="Not Active", hw="Not Active", swt="Not Active", cap="Not Active")
             for s in (2070, 2055, 2070)]
    r = run_sampler(monkeypatch, fake_smi(tmp_path, before, after, 0.3), 1.0)
    assert r["samples"] == 3
    assert r["sm_mhz"] == 2070 and r["sm_max_mhz"] == 2070
    assert r["reasons"] == []


def test_throttle_reasons_are_reported(tmp_path, monkeypatch):
    before = [LINE.format(sm=2070, active="Not Active", hw="Not Active", swt="Not Active", cap="Not Active")]
    after = [LINE.format(sm=1900, active="Active", hw="Active", swt="Not Active", cap="Active"),
             LINE.format(sm=1950, active="Active", hw="Not Active", swt="Active", cap="Not Active")]
    r = run_sampler(monkeypatch, fake_smi(tmp_path, before, after, 0.3), 1.0)
    assert r["samples"] == 2
    assert r["sm_mhz"] == 1925
    assert r["reasons"] == ["hw_slowdown", "sw_power_cap", "sw_thermal_slowdown"]


def test_short_region_keeps_the_earlier_samples(tmp_path, monkeypatch):
    # nothing arrives after the mark: the sampler falls back to what it has
    before = [LINE.format(sm=2070, active="Not Active", hw="Not Active", swt="Not Active", cap="Not Active")]
    r = run_sampler(monkeypatch, fake_smi(tmp_path, before, [], 5), 0.2)
    assert r["samples"] == 1 and r["sm_mhz"] == 2070


def test_missing_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    c = bench.ClockSampler(0)
    c.start()
    c.begin()
    assert c.stop()["reasons"] == ["nvidia-smi unavailable"]


def test_serving_window_rates():
    """The steady-state test of the serving sweep: a server that completes every
    request 50 ms after it arrives keeps up (ratio 1); one that completes them
    at half the arrival rate falls behind (ratio 0.5), whatever the tail."""
    import numpy as np
    sub = np.arange(1000) * 1e-3                      # 1,000 requests/s for 1 s
    off, ach = bench.serving_window_rates(sub, np.full(1000, 50.0))
    assert abs(off - 1000) < 1e-6 and abs(ach / off - 1) < 1e-9
    done = np.arange(1000) * 2e-3                     # completions every 2 ms
    off, ach = bench.serving_window_rates(sub, (done - sub) * 1e3 + 10.0)
    assert abs(ach / off - 0.5) < 1e-9
