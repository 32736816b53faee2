"""The reference arm of bench.py (the FP64 oracle on the host cores) keeps the JSON contract:
one line with the metric, the oracle's rate, a cpu_baseline object describing the sample it
timed, and an e2e object with no host-device copies. It needs no GPU, so it runs here."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _line(*args):
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", *args], cwd=ROOT,
                         capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    return json.loads(lines[0])


@pytest.mark.parametrize("workload", ["heat1d", "schrodinger1d"])
def test_reference_arm_json_contract(workload):
    d = _line("--workload", workload, "--steps", "1", "--warmup", "3")
    assert d["impl"] == "reference" and d["metric"] == "LEM dof-steps/s" and d["unit"] == d["metric"]
    assert d["value"] > 0 and d["higher_is_better"] is True and d["n_gpus"] == 1
    assert d["steps"] == 1 and d["warmup"] == 3 and d["data"] == "synthetic"
    assert d["config"]["workload"].startswith(workload)
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
