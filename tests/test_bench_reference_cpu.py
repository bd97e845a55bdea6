"""bench.py's reference arm (the oracle on the host cores) keeps the JSON
contract: one line with the metric, the rate and its unit, the CPU baseline
it measured and an e2e object without transfers.  The rate is measured on a
bounded sample graph, and the line names that graph (scale, n, m) beside
the workload it stands in for."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "dtype", "config"):
        assert k in d, k
    assert d["value"] > 0 and d["unit"] == "edges/s" and d["higher_is_better"] is True
    assert d["config"]["workload"] == "rmat22_ef16_plm"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["sample"]
    assert cb["cores"] == os.cpu_count()            # the OpenMP build on every host core
    sample = d["config"]["cpu_sample"]
    assert sample["n"] == 1 << 20 and sample["m"] == cb["sample_graph"]["m"] > 0
    assert "R-MAT scale 20" in sample["graph"] and f"m={sample['m']}" in cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
