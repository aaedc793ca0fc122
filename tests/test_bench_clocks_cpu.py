"""bench.py's clock sampler on the CPU, with a stand-in for nvidia-smi that
prints rows in its CSV query format at the requested interval: the sampler
is running before the timed region opens, counts the rows inside the
region, and reads throttle reasons from the rows around it."""
import os
import stat
import sys
import time

import bench

FAKE = r'''#!{py}
import sys, time
ms = int(sys.argv[sys.argv.index("-lms") + 1])
time.sleep({startup})
k = 0
while True:
    cap = "Active" if {cap_from} <= k else "Not Active"
    print(f"0, {{2070 - k % 2}}, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, {{cap}}", flush=True)
    k += 1
    time.sleep(ms / 1000.0)
'''


def _fake(tmp_path, startup=0.2, cap_from=10 ** 9):
    p = tmp_path / "fake-nvidia-smi"
    p.write_text(FAKE.format(py=sys.executable, startup=startup, cap_from=cap_from))
    p.chmod(p.stat().st_mode | stat.S_IEXEC)
    return str(p)


def test_samples_inside_the_region(tmp_path):
    c = bench.ClockSampler(0, exe=_fake(tmp_path))
    t = time.perf_counter()
    c.start()
    assert c.rows, "start returns once the sampler has produced a row"
    assert time.perf_counter() - t >= 0.2
    c.region(True)
    time.sleep(0.4)
    c.region(False)
    c.stop()
    s = c.summary()
    assert s["samples"] >= 4
    assert s["sm_mhz"] in (2069.0, 2070.0) and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == []


def test_throttle_reason_in_the_region_is_reported(tmp_path):
    c = bench.ClockSampler(0, exe=_fake(tmp_path, startup=0.0, cap_from=3))
    c.start()
    c.region(True)
    time.sleep(0.4)
    c.region(False)
    c.stop()
    assert "sw_power_cap" in c.summary()["reasons"]


def test_region_shorter_than_the_interval_uses_the_next_row(tmp_path):
    c = bench.ClockSampler(0, exe=_fake(tmp_path, startup=0.0))
    c.start()
    time.sleep(0.02)
    c.region(True)
    c.region(False)
    c.stop()
    s = c.summary()
    assert s["samples"] == 0
    assert s["sm_mhz"] in (2069.0, 2070.0)


def test_missing_tool_is_reported_unsampled(tmp_path):
    c = bench.ClockSampler(0, exe=os.path.join(str(tmp_path), "no-such-tool"))
    c.start()
    c.region(True)
    c.region(False)
    c.stop()
    assert c.summary()["reasons"] == ["unsampled"]
