"""Host logic of bench.py that needs no GPU: the reference arm (the CPU
oracle timed on the host cores) prints one JSON line with the contract's
keys, and the clock-sample summary reads nvidia-smi's CSV rows (median SM
clock, maximum clock, throttle reasons that were active)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference"
    assert d["steps"] == 1 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_clock_summary_parses_samples(tmp_path):
    sys.path.insert(0, ROOT)
    import bench
    cs = bench.ClockSampler(0)
    rows = [
        "0, 2070, 2070, 850.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2010, 2070, 1200.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
    ]
    with open(cs.f.name, "w") as fh:
        fh.write("\n".join(rows) + "\n")
    s = cs.summary()
    assert s["sm_mhz"] == pytest.approx(2010.0)
    assert s["sm_max_mhz"] == pytest.approx(2070.0)
    assert s["reasons"] == ["sw_power_cap"]
    assert s["samples"] == 3
    assert not os.path.exists(cs.f.name)
    empty = bench.ClockSampler(0)
    assert empty.summary()["reasons"] == ["unsampled"]
