"""bench.py's clock sampler on CPU, against a stand-in nvidia-smi on PATH.

The stand-in prints one timestamped CSV sample per period, as
``nvidia-smi --query-gpu=... -lms P`` does; the SM clock it reports is low
before the timed region and while a thermal slowdown is flagged after it, so
the summary must keep exactly the samples stamped between ``begin()`` and
``end()``.
"""
import os
import stat
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

FAKE = r'''#!/usr/bin/env python3
import sys, time
from datetime import datetime
period = 0.025
for i, a in enumerate(sys.argv):
    if a == "-lms":
        period = float(sys.argv[i + 1]) / 1e3
mark = float(open(sys.argv[0] + ".mark").read())  # wall time the region opens
while True:
    now = time.time()
    busy = now >= mark
    late = now >= mark + 0.4
    sm = 2070 if busy and not late else 1100
    thermal = "Active" if late else "Not Active"
    stamp = datetime.fromtimestamp(now).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    print("%s, 0, %d, 2070, 900.0, 0x0, Not Active, %s, Not Active, Not Active" % (stamp, sm, thermal),
          flush=True)
    time.sleep(period)
'''


def test_clock_samples_are_the_timed_region_only(tmp_path, monkeypatch):
    smi = tmp_path / "nvidia-smi"
    smi.write_text(FAKE)
    smi.chmod(smi.stat().st_mode | stat.S_IEXEC)
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep + os.environ.get("PATH", ""))
    sys.path.insert(0, ROOT)
    import bench

    mark = time.time() + 0.3
    (tmp_path / "nvidia-smi.mark").write_text(repr(mark))
    ck = bench.Clocks(0)
    ck.start()
    time.sleep(max(0.0, mark - time.time()) + 0.05)
    ck.begin()
    time.sleep(0.25)  # the "timed region": fast clocks, no reason active
    ck.end()
    time.sleep(0.35)  # afterwards the stand-in reports a thermal slowdown at low clocks
    out = ck.stop()
    assert out is not None
    assert out["samples"] >= 3, out
    assert out["sm_mhz"] == 2070.0, out
    assert out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == [], out
    assert 0.2 < out["region_s"] < 0.4


def test_clock_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    sys.path.insert(0, ROOT)
    import bench

    ck = bench.Clocks(0)
    ck.start()
    ck.begin()
    ck.end()
    assert ck.stop() is None
