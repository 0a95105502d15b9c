"""The reference arm of bench.py (the FP64 oracle timed on the host cores) prints one JSON
line with the fields of the benchmark contract.  CPU only: a 2 s sample instead of the
default minute."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    env = dict(os.environ, PCF_REFERENCE_SECONDS="2")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "3"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == "gradient evals/s" and d["unit"] == "gradient evals/s"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["vs_baseline"] is None
    assert (d["n_gpus"], d["steps"], d["warmup"]) == (1, 2, 3)
    assert d["scaling"] == "weak" and d["dtype"] == "f64" and d["data"] == "synthetic"
    assert d["config"]["grid"] == [32, 33, 32] and d["config"]["batch"] == 8 and d["config"]["workload"]
    # one step of the workload is 8 gradient evaluations
    assert abs(d["ms_per_step"] - 8e3 / d["value"]) <= 1e-9 * d["ms_per_step"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
