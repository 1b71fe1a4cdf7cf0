"""bench.py on the CPU: the reference arm's JSON line (the oracle on the host cores) keeps
the contract's keys and the measured arm's workload config, and the clock sampler's
summary (run against a stand-in nvidia-smi that prints fixed rows)."""
from __future__ import annotations

import json
import os
import stat
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "1"], capture_output=True, text=True,
                         timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    lines = [ln for ln in out.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 1
    sys.path.insert(0, ROOT)
    import bench
    assert d["config"]["workload"] == bench.VOIGT_WORKLOAD
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1


def test_clock_sampler_summary(tmp_path, monkeypatch):
    fake = tmp_path / "nvidia-smi"
    fake.write_text("#!/bin/sh\n"
                    "echo '0, 1200 MHz, 2070 MHz, 90.00 W, 0x0, Not Active, Not Active, Not Active, Not Active'\n"
                    "while true; do\n"
                    "echo '0, 2070 MHz, 2070 MHz, 900.00 W, 0x4, Not Active, Not Active, Not Active, Active'\n"
                    "sleep 0.05; done\n")
    fake.chmod(fake.stat().st_mode | stat.S_IEXEC)
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep + os.environ["PATH"])
    sys.path.insert(0, ROOT)
    import bench
    c = bench.Clocks(0)
    assert c.n0 >= 1  # the sampler ran before the region began
    time.sleep(0.4)
    r = c.stop()
    # the idle line written before the region is left out of the median
    assert r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == ["sw_power_cap"] and r["samples"] >= 2
