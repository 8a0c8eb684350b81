"""The benchmark's reference arm (the oracle on the host cores) keeps the line format on CPU:
same metric and config as the GPU arm of the workload, `impl: "reference"`, an e2e object with no
host-device bytes, and only rank 0 printing under a multi-rank launch."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_ref(workload, env_extra=None):
    env = dict(os.environ)
    env.update(env_extra or {})
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        workload, "--steps", "1", "--warmup", "0"], capture_output=True, text=True, env=env,
                       cwd=ROOT, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    return [ln for ln in r.stdout.splitlines() if ln.strip()]


@pytest.mark.parametrize("workload,metric_name", [("cfd128_b16_f4_fp64", "METRIC"),
                                                  ("advect128_b32_x2_f4_fp64", "ADVECT_METRIC")])
def test_reference_line(workload, metric_name):
    sys.path.insert(0, ROOT)
    import bench
    lines = run_ref(workload)
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == getattr(bench, metric_name)
    assert d["unit"] == "Gpoint-ops/s" and d["higher_is_better"] is True
    assert d["config"]["workload"] == workload
    assert d["steps"] == 1 and d["warmup"] == 0
    assert d["value"] > 0 and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_other_ranks_print_nothing():
    assert run_ref("cfd128_b16_f4_fp64", {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}) == []
