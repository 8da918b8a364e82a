"""The benchmark's JSON line on the CPU: the reference arm (the oracle on host cores) at N = 1 carries
every key of the contract, with its own metric and unit and no host-device traffic; its CPU baseline
states the host threads it was given, the CPU time it actually used and the CPU model."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="", OPENBLAS_NUM_THREADS="1")
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "square512", "--steps", "2",
                          "--warmup", "0", "--cpu-seconds", "1", "--tree", "flatts"],
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.strip().splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "e2e", "cpu_baseline", "impl"):
        assert k in d, k
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 2 and d["higher_is_better"] is True
    assert d["unit"] == "TFLOP/s" and d["value"] > 0 and d["ms_per_step"] > 0
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["unit"] == d["unit"]
    assert isinstance(cb["sample"], str) and cb["sample"]
    assert cb["cores"] == len(os.sched_getaffinity(0))
    assert cb["cores_effective"] > 0 and isinstance(cb["cpu_model"], str) and cb["cpu_model"]
    assert "whole task list" in cb["sample"]       # the 512 x 512 reduction is timed in full
    e = d["e2e"]
    assert e["unit"] == d["unit"] and e["value"] == d["value"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
