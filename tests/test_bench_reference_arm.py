"""The reference arm of bench.py (the FP64 CPU oracle timed on the host
cores) prints one JSON line with the benchmark's metric, unit and workload,
a cpu_baseline describing the sample, and an e2e block without transfers."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.slow
def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3",
                          "--oracle-budget", "2"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["unit"] == "GDoF/s" and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["ms_per_step"] > 0
    # the mesh the oracle ran (a sample of the channel workload), measured
    # there: no extrapolation to the benchmark's size
    assert d["config"]["workload"].startswith("channel") and "sample" in d["config"]["workload"]
    assert d["ms_per_step"] == pytest.approx(d["cpu_baseline"]["ms_per_step"])
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    # the assembled momentum apply at the full 32^3 Taylor-Green size
    assert cb["apply"]["value"] > 0 and "32x32x32" in cb["apply"]["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
