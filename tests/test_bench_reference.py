"""The reference arm of bench.py (the FP64 oracle timed on the host cores):
one JSON line with the contract's keys on rank 0, nothing on other ranks
(CPU, no GPU needed)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra, workload="duct64x32_n8", extra=()):
    env = dict(os.environ, **env_extra)
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload",
                          workload, "--steps", "1", "--warmup", "0"] + list(extra),
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    return [l for l in out.stdout.splitlines() if l.strip()]


def test_reference_arm_prints_one_contract_line():
    lines = _run({"WORLD_SIZE": "1", "RANK": "0"})
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "impl",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_do_no_work():
    assert _run({"WORLD_SIZE": "2", "RANK": "1"}) == []


def test_reference_arm_describes_the_measured_workload():
    """The reference line's config is the measured arm's workload config
    (same workload text, runs, steps, cells, partner choice); the mixed
    workload is sampled on its median grid."""
    sys.path.insert(0, ROOT)
    import argparse
    import bench
    from paper_cs_9902024_gb300 import workloads as W
    env = {"WORLD_SIZE": "1", "RANK": "0"}
    d = json.loads(_run(env, extra=["--partner", "subcell", "--n-sub", "3"])[0])
    a = argparse.Namespace(workload="duct64x32_n8", partner="subcell", n_sub=3)
    ref = bench.workload_config(bench.workload(None, "duct64x32_n8", "subcell", 3), a)
    for k, v in ref.items():
        assert d["config"][k] == v, k
    assert d["config"]["partner"] == "subcell (3 subcells per axis)"
    m = json.loads(_run(env, workload="mixed_n1024")[0])
    assert m["value"] > 0 and m["config"]["grids"] == len(W.mixed_n1024()["groups"])
    assert "median" not in m["config"]["workload"] and "duct_mixed" in m["cpu_baseline"]["sample"]
