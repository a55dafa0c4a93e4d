"""bench.py's clock record (no GPU): samples are stamped on arrival, so the
summary of a time window takes only that window's samples and counts those
of the timed region; a fake nvidia-smi on PATH stands in for the real one."""
import os
import stat
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

FAKE = """#!{py}
import sys, time
i = 0
while True:
    # index, sm, max sm, power, active, hw, hw thermal, sw thermal, sw power cap
    mhz = 2070 if i < 3 else 1500
    cap = "Active" if i >= 3 else "Not Active"
    print(f"0, {{mhz}}, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, {{cap}}", flush=True)
    i += 1
    time.sleep(0.05)
"""


def test_clock_sampler_windows(tmp_path, monkeypatch):
    fake = tmp_path / "nvidia-smi"
    fake.write_text(FAKE.format(py=sys.executable))
    fake.chmod(fake.stat().st_mode | stat.S_IEXEC)
    monkeypatch.setenv("PATH", f"{tmp_path}{os.pathsep}{os.environ['PATH']}")
    import bench
    with bench.ClockSampler(0) as c:
        c.wait_first()
        t0 = time.monotonic()
        time.sleep(0.12)  # samples 0-2 or so: 2070 MHz, no reason
        t1 = time.monotonic()
        time.sleep(0.4)   # later samples: 1500 MHz, power cap active
        t2 = time.monotonic()
    assert c.samples, "no sample read"
    early = c.summary((0.0, t1))
    assert early["sm_mhz"] == 2070.0 and early["reasons"] == [] and early["samples"] >= 1
    whole = c.summary((t0, t2), (t0, t1))
    assert whole["sm_max_mhz"] == 2070.0
    assert "sw_power_cap" in whole["reasons"]
    assert 1 <= whole["samples_in_timed_region"] <= whole["samples"]
    assert c.summary((t2 + 10, t2 + 20))["samples"] == 0  # an empty window


def test_clock_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))  # nothing to run
    import bench
    with bench.ClockSampler(0) as c:
        c.wait_first(timeout_s=0.1)
    s = c.summary((0.0, time.monotonic()), (0.0, 1.0))
    assert s["samples"] == 0 and s["sm_mhz"] is None and s["samples_in_timed_region"] == 0
