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


def _fake_result(bench):
    """A result object shaped like the GPU arm's, with made-up timings and long strings."""
    peaks = {"hbm_gbs": 6683.8, "bf16_tflops": 1963.0}
    roof = bench.roofline("stage1", 2.07, (1.76e9, "flop"), "fp64", peaks,
                          ("stage1", "helm2d_n1024", "fp64"))
    rows = bench.roofline("rows", 0.0629, (224 * 1048576, "byte"), "fp64", peaks)
    forms = [{"workload": wl, "mode": m, "mode_used": m, "value": 1.234567e9, "ms": 0.5612345,
              "kernel": "stage2", "bound": "alu", "frac": 0.412345, "dalpha_p50": 6.1e-4,
              "dalpha_p99": 6.8e-3, "dalpha_max": 0.13, "resid_p50": 1.2, "resid_p99": 3.4,
              "fallback_frac": 0.0123, "gmres": 9, "gmres_fp64": 8}
             for wl, m in bench.FORMS]
    return {"metric": bench.METRIC, "value": 2.9234567e8, "unit": "stencils/s", "n_gpus": 1,
            "steps": 50, "warmup": 5, "ms_per_step": 3.58765432, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "helm2d_n1024", "policy": "local", "mode": "fp64",
                       "mode_used": "fp64", "d": 2, "n": 1024, "points": 1048576,
                       "shifts": 93491, "l2": "flushed before every timed step (256 MiB "
                       "write), outside the step events", "parallelism": "replicas x1"},
            "roofline": roof, "rows_roofline": rows, "gpu_launches": 450,
            "clocks": {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "samples": 40, "reasons": []},
            "e2e": {"value": 2.68e8, "unit": "stencils/s", "h2d_bytes_per_step": 8388608,
                    "d2h_bytes_per_step": 226492416, "ms_per_step": 3.91, "loop": "x" * 400,
                    "one_step_at_a_time": {"value": 2.16e8, "ms_per_step": 4.85}},
            "cpu_baseline": {"value": 5123.4, "unit": "stencils/s", "cores": 16, "kind": "oracle",
                             "sample": "y" * 500, "seconds": 15.0,
                             "single_core": {"value": 385.1, "cores": 1, "sample": "z" * 300}},
            "forms": forms, "detail": "bench_detail.json"}


def test_result_line_is_compact_and_complete():
    sys.path.insert(0, ROOT)
    import bench

    line = bench.contract_line(_fake_result(bench))
    assert len(line.encode()) <= bench.LINE_LIMIT
    j = json.loads(line)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "roofline", "e2e", "cpu_baseline", "clocks", "gpu_launches"):
        assert k in j, k
    assert j["config"]["workload"] == "helm2d_n1024"
    r = j["roofline"]
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    # 1.76e9 flop in 2.07 ms against 4 flop/SM/clk x 152 SMs x 2070 MHz
    assert abs(r["achieved"] - 1.76e9 / 2.07e-3 / 1e12) < 1e-3
    assert abs(r["peak"] - 4 * 152 * 2070e6 / 1e12) < 1e-3
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-3
    e = j["e2e"]
    assert e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] > 0
    assert j["cpu_baseline"]["cores"] == 16 and j["cpu_baseline"]["single_core"]["cores"] == 1
    assert len(j["forms"]) == len(bench.FORMS)


def test_result_line_drops_optional_parts_before_the_contract_keys():
    sys.path.insert(0, ROOT)
    import bench

    res = _fake_result(bench)
    res["forms"] = res["forms"] * 8  # far too long: the optional summaries go first
    line = bench.contract_line(res)
    assert len(line.encode()) <= bench.LINE_LIMIT
    j = json.loads(line)
    assert "forms" not in j and j["value"] > 0 and "roofline" in j and "cpu_baseline" in j


def test_cpu_oracle_sample_reports_the_processes_it_used():
    p = subprocess.run([sys.executable, "bench.py", "--cpu-only", "--workload", "helm2d_n32",
                        "--cpu-procs", "2", "--cpu-budget", "0.5"], cwd=ROOT,
                       capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stderr[-2000:]
    j = json.loads([ln for ln in p.stdout.splitlines() if ln.startswith("{")][-1])
    assert j["cores"] == 2 and j["kind"] == "oracle" and j["value"] > 0
    assert "2 process(es)" in j["sample"]
