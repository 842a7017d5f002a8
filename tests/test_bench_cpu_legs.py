"""The bench's CPU legs run without a GPU: the oracle sample behind `cpu_baseline`, and the
reference arm (`--impl reference`), whose JSON line must carry the contract's keys."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_oracle_sample_is_bounded_and_described():
    import bench
    from paper_2202_02264_gb300 import workloads as W
    out = bench.oracle_sample(W.workload("lgssm_1d"), target_s=0.3)
    assert out["kind"] == "oracle" and out["value"] > 0 and out["cores"] >= 1
    assert "first" in out["sample"] and out["unit"] == bench.UNIT


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "lgssm_1d", "--steps", "1", "--warmup", "3"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["config"]["workload"] == "lgssm_1d"
