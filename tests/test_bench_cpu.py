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


def test_trace_report_on_a_synthetic_trace():
    """The per-sub-task summary of a traced launch: classes, busy share and the critical chain, on a
    hand-made three-sub-task program (PF -> PU -> UNMQR strip, a fourth independent strip)."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench

    class FakeHandle:
        def trace(self):
            # start, end (ns), SM, op word (type | strip << 8 | block << 16 | kind << 24)
            return np.array([[0, 100, 0, 7], [110, 150, 1, 8 | (1 << 8)], [170, 300, 2, 1],
                             [0, 50, 3, 1 | (1 << 8)]], dtype=np.int64)

        def trace_program(self):
            prog = np.zeros((4, 8), dtype=np.int32)
            prog[:, 0] = [7, 8 | (1 << 8), 1, 1 | (1 << 8)]
            prog[1, 5:7] = [0, 1]       # PU waits for PF
            prog[2, 5:7] = [1, 2]       # the strip waits for PU
            return prog, np.array([0, 1], dtype=np.int32)

    txt = bench.trace_report(FakeHandle(), 64, 16, 8, 4, "synthetic")
    assert "4 sub-tasks" in txt
    assert "critical chain: 3 sub-tasks, 0.00 ms" in txt
    # chain: PF 100 + PU 40 + strip 130 = 270 ns of sub-task time, gaps 10 + 20 = 30 ns
    assert "| UNMQR strip | 2 |" in txt and "| PF GE | 1 |" in txt and "| PU GE | 1 |" in txt
    assert "waiting gaps" in txt
    b, f = bench.subtask_bytes_flops(1, 64, 16, 32, 8)
    assert f == 6 * 64 * 64 * 32 / 3.0 and b > 2 * 64 * 32 * 8
