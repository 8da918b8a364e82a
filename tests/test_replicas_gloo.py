"""The N > 1 path of bench.py on the CPU: two ranks over gloo (127.0.0.1).

A single reduction does not shard, so N GPUs run independent replicas: no collective on the data
path, a barrier around the timed region, the step time taken as the maximum over ranks, and the
whole-job value = total work of all ranks / that time.  These tests run the bench's own helpers in two
processes, and the reference arm under two ranks (rank 0 alone runs the oracle and prints; the other
rank exits 0 without work)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


HELPER = r"""
import json, os, sys
sys.path.insert(0, {root!r})
import bench
import torch
world, rank, local = bench.dist_setup()
# each rank's own step time; the job time is the maximum
t = bench.max_over_ranks(10.0 + 5.0 * rank, world, "cpu")
bench.barrier(world)
# replicas use different matrices (seed offset per rank) and no collective on the data
w = dict(bench.WORKLOADS["square512"], name="square512")
A = bench.make_input(w, rank, "cpu")
s = float(A[:4, :4].sum())
g = torch.tensor([s], dtype=torch.float64)
import torch.distributed as dist
gathered = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
dist.all_gather(gathered, g)
flops = bench.metric_flops(512, 512)
value = world * flops / (t * 1e-3) / 1e12
print(json.dumps({{"rank": rank, "world": world, "t": t, "sums": [float(x) for x in gathered], "value": value}}))
dist.destroy_process_group()
"""


def run_ranks(args, world=2, timeout=600):
    port = free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, WORLD_SIZE=str(world), RANK=str(r), LOCAL_RANK=str(r), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="", OPENBLAS_NUM_THREADS="1")
        procs.append(subprocess.Popen(args, env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True,
                                      cwd=ROOT))
    outs = []
    for p in procs:
        try:
            o, e = p.communicate(timeout=timeout)
        except subprocess.TimeoutExpired:
            p.kill()
            o, e = p.communicate()
        outs.append((p.returncode, o, e))
    return outs


def test_replica_helpers_two_ranks():
    outs = run_ranks([sys.executable, "-c", HELPER.format(root=ROOT)])
    lines = []
    for rc, o, e in outs:
        assert rc == 0, e[-2000:]
        lines.append(json.loads(o.strip().splitlines()[-1]))
    for d in lines:
        assert d["world"] == 2
        assert d["t"] == 15.0                      # max over ranks of 10 and 15
        assert d["sums"][0] != d["sums"][1]        # different seeds per replica
        assert abs(d["value"] - 2 * (4 * 512 ** 3 - 4 * 512 ** 3 / 3) / 15e-3 / 1e12) < 1e-9


def test_reference_arm_two_ranks():
    """bench.py --impl reference under two ranks: rank 0 prints one JSON line, rank 1 exits 0 silently."""
    outs = run_ranks([sys.executable, "bench.py", "--impl", "reference", "--workload", "square512", "--gpus", "2",
                      "--steps", "1", "--warmup", "0", "--cpu-seconds", "1", "--tree", "flatts"])
    (rc0, o0, e0), (rc1, o1, e1) = outs
    assert rc0 == 0, e0[-2000:]
    assert rc1 == 0, e1[-2000:]
    assert o1.strip() == ""
    line = json.loads(o0.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["value"] > 0 and line["e2e"]["h2d_bytes_per_step"] == 0
