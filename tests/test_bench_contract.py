"""The benchmark's reference arm (the oracle on the host cores) prints one JSON
line with the keys the benchmark contract names; run on the small workload."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                          "maxcut_d6_kron_cap16", "--steps", "2", "--warmup", "0"], capture_output=True, text=True,
                         timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference"
    assert line["higher_is_better"] is False and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["config"]["workload"] == "maxcut_d6_kron_cap16"


def test_batch_partition_covers_every_order_of_the_batch():
    sys.path.insert(0, ROOT)
    import bench
    from paper_2509_11890_gb300 import inputs
    insts = inputs.batch_maxcut(64, 0)
    assert {i["d"] for i in insts} == set(range(6, 12))
    shards = bench.partition_batch([i["d"] for i in insts], 4, 64)
    assert all(len(sh) > 0 for sh in shards)
