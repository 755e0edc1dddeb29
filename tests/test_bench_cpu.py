"""bench.py's reference arm (the oracle on the host cores) runs without a GPU and prints the
JSON line the measurement contract asks for, with the same metric as the GPU arm; under a
multi-rank launch only rank 0 works and prints."""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                           "--warmup", "3", "--ref-step-s", "0.3"], cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_one_contract_line():
    sys.path.insert(0, ROOT)
    import bench

    p = _run({"RANK": "0", "WORLD_SIZE": "1", "LOCAL_RANK": "0"})
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    j = json.loads(lines[0])
    assert j["impl"] == "reference" and j["metric"] == bench.METRIC
    assert j["unit"] == "stencils/s" and j["higher_is_better"] is True
    assert (j["steps"], j["warmup"], j["n_gpus"]) == (1, 3, 1)
    assert j["value"] > 0 and j["ms_per_step"] > 0
    assert j["config"]["workload"] == "helm2d_n1024"
    cb = j["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == j["value"]
    assert cb["sample"]
    e = j["e2e"]
    assert (e["value"], e["unit"]) == (j["value"], j["unit"])
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_quietly():
    p = _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert p.returncode == 0, p.stderr[-2000:]
    assert not [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
