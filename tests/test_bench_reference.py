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


def test_oracle_pool_runs_every_route():
    """oracle.pool's worker processes run the unmodified oracle on their shares:
    the items of one step add up to the sample, for each route."""
    import tempfile
    import numpy as np
    sys.path.insert(0, str(ROOT))
    from oracle.pool import OraclePool
    from paper_1807_08084_gb300 import synth as S
    with tempfile.TemporaryDirectory() as d:
        z = S.WORKLOADS["plain_256"].packed_z(np.arange(1000, dtype=np.uint64))
        np.save(f"{d}/z.npy", z)
        for route in ("ge", "adj"):
            with OraclePool(route, f"{d}/z.npy", workers=3) as pool:
                items, wall, slowest = pool.step()
            assert items == 1000 and wall > 0 and 0 < slowest <= wall
        w = S.scaled(S.WORKLOADS["wishart_pair_4k"], 12, 20)
        np.save(f"{d}/a.npy", w.image(0))
        np.save(f"{d}/b.npy", w.image(1))
        with OraclePool("wishart", (f"{d}/a.npy", f"{d}/b.npy"), workers=2) as pool:
            items, _, _ = pool.step()
        assert items == 12 * 20
