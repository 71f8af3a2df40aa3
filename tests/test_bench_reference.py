"""bench.py's reference arm on CPU: `--impl reference` times the oracle on
the host threads and prints the bench's one JSON line with the keys the
contract names (impl, metric, value, unit, steps, warmup, ms_per_step,
higher_is_better, scaling, dtype, data, config.workload, cpu_baseline, e2e
with zero copy bytes).  A small lattice keeps it to a few seconds."""
import json
import os
import subprocess
import sys

from test_fixed_point import ROOT


def test_reference_arm_prints_one_contract_line():
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--L", "6",
                        "--M", "64", "--steps", "2", "--warmup", "3"],
                       capture_output=True, text=True, timeout=300, cwd=ROOT, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "spin updates/s" and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 3 and d["value"] > 0 and d["ms_per_step"] > 0
    assert d["metric"].startswith("spin updates/s") and d["dtype"] == "f64" and d["data"] == "synthetic"
    assert "workload" in d["config"] and d["config"]["L"] == 6
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
