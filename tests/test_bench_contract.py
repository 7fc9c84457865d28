"""bench.py's reference arm (the oracle on the host cores) keeps the JSON
contract: one line with the required keys, the same metric, unit and config
as the GPU arm, a cpu_baseline describing the run, and an e2e object."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KEYS = {"impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
        "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
        "cpu_baseline", "e2e"}


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--waters", "2",
                          "--steps", "1", "--warmup", "0"], cwd=ROOT, capture_output=True,
                         text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert KEYS <= set(d)
    assert d["impl"] == "reference" and d["higher_is_better"] is True
    assert d["unit"] == "Fock builds/s" and d["value"] > 0
    assert d["config"]["workload"].startswith("(H2O)_2 ") and "N=50" in d["config"]["workload"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0


def test_whole_job_rate_and_config_helpers():
    sys.path.insert(0, ROOT)
    import bench
    import workload
    c = bench.config(workload.water_cluster(64), "mixed_tf32x3")
    assert "N=1600, Naux=4800, nocc=320" in c["workload"]
    assert "98.3 GB" in c["l2"] and "49.2 GB" in c["l2"]
    assert bench.whole_job_rate(4, 10, 2.0) == 20.0
