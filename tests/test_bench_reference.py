"""The benchmark's reference arm (the FP64 oracle on the host cores) keeps the
JSON-line contract: the same metric, unit and workload config as the GPU arm,
a bounded CPU sample described in cpu_baseline, an e2e entry with no host
transfers, and under torchrun only rank 0 prints."""
import json
import os
import subprocess
import sys
from pathlib import Path

ROOT = Path(__file__).resolve().parents[1]


def run(env_extra):
    env = dict(os.environ, **env_extra)
    r = subprocess.run([sys.executable, str(ROOT / "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "3"], capture_output=True, text=True,
                       env=env, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    return r.stdout.strip()


def test_reference_arm_json_line():
    sys.path.insert(0, str(ROOT))
    import bench
    out = run({"WORLD_SIZE": "1", "RANK": "0"})
    line = json.loads(out.splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["higher_is_better"] is True
    assert line["config"] == bench.workload_config(16384, 16384, 1)
    assert line["value"] > 0 and line["cpu_baseline"]["value"] == line["value"]
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert "sample" in line["cpu_baseline"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"],
                           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_print_nothing():
    assert run({"WORLD_SIZE": "2", "RANK": "1"}) == ""
