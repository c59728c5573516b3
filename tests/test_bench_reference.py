"""The benchmark's reference arm (the oracle timed on the host) keeps the
one-line JSON contract, on CPU: small workloads, a few steps."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_reference(workload, steps=2, warmup=3):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", workload, "--steps", str(steps), "--warmup", str(warmup)],
                         capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1, out.stdout
    return json.loads(lines[0])


@pytest.mark.parametrize("workload,dtype", [("srd-10c-rho5-fp64", "f64"),
                                            ("srd-batch64-mixed", "f32+i64")])
def test_reference_line(workload, dtype):
    line = run_reference(workload)
    assert line["impl"] == "reference"
    assert line["metric"] == "MPCD particle-steps/s"
    assert line["unit"] == "particle-steps/s"
    assert line["value"] > 0.0 and line["ms_per_step"] > 0.0
    assert line["n_gpus"] == 1 and line["steps"] == 2 and line["warmup"] == 3
    assert line["higher_is_better"] is True
    assert line["vs_baseline"] is None
    assert line["dtype"] == dtype and line["data"] == "synthetic"
    assert line["config"]["workload"] == workload
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    assert cb["unit"] == line["unit"] and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_warmup_is_at_least_three():
    line = run_reference("srd-10c-rho5-fp64", steps=1, warmup=0)
    assert line["warmup"] == 3
