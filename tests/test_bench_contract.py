"""The benchmark's reference arm (the oracle on the host cores) runs without a GPU: one JSON line
with the contract's keys, the same metric as the GPU arm, a positive throughput, and the
cpu_baseline / e2e objects describing this run (no host-device copies)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    out = json.loads(lines[0])
    sys.path.insert(0, ROOT)
    import bench
    assert out["impl"] == "reference" and out["metric"] == bench.METRIC
    for k in ("value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in out, k
    assert out["value"] > 0 and out["unit"] == "cell-updates/s" and out["higher_is_better"] is True
    assert out["n_gpus"] == 1 and out["steps"] == 1 and out["warmup"] >= 3 and out["dtype"] == "f64"
    assert out["config"]["workload"]
    cb = out["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == out["value"]
    e = out["e2e"]
    assert e["value"] == out["value"] and e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
