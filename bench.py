#!/usr/bin/env python
"""Benchmark of the tiled band bidiagonalization (GE2BND) on GB300.

One step = one full reduction B = Q^T A P (pack, the whole task DAG of QR/LQ panel and update kernels,
band extraction) of one synthetic matrix already resident in HBM.  Throughput is counted with the
paper's operation count for BiDiag, 4 m n^2 - 4 n^3 / 3 flops (Sec. 6.2 credits R-BiDiag with the same
count), reported in TFLOP/s.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--tree T] [--impl ours|reference]

N > 1 (torchrun, one process per GPU): independent replicas, one matrix per rank, no collective on the
data path; value = total flops of all ranks / max-over-ranks time ("scaling": "weak").
--impl reference times the plain CPU oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    "square8192": dict(m=8192, n=8192, nb=256, ib=32, variant="bidiag", kind="sv", seeds=(2, 3),
                       desc="square FP64 8192x8192, A = U diag(s) V^T (Haar U, V; s geometric 1..1e-8), "
                            "nb=256 ib=32, BiDiag"),
    "square4096": dict(m=4096, n=4096, nb=256, ib=32, variant="bidiag", kind="sv", seeds=(2, 3),
                       desc="square FP64 4096x4096, A = U diag(s) V^T (Haar U, V; s geometric 1..1e-8), "
                            "nb=256 ib=32, BiDiag"),
    "square512": dict(m=512, n=512, nb=64, ib=16, variant="bidiag", kind="gauss", seeds=(1,),
                      desc="square FP64 512x512 N(0,1), nb=64 ib=16, BiDiag"),
    "tall65536x1024": dict(m=65536, n=1024, nb=256, ib=32, variant="rbidiag", kind="gauss", seeds=(4,),
                           desc="tall-skinny FP64 65536x1024 N(0,1), nb=256 ib=32, R-BiDiag"),
    "batched512": dict(m=1024, n=1024, nb=0, ib=0, variant="auto", kind="batch", seeds=(6,),
                       desc="batch of 512 matrices, m ~ U[64, 1024], n ~ U[32, m], N(0,1), one persistent launch, "
                            "autotuned nb / ib / tree / variant per matrix"),
    "tall65536x2048": dict(m=65536, n=2048, nb=256, ib=32, variant="rbidiag", kind="gauss", seeds=(5,),
                           desc="tall-skinny FP64 65536x2048 N(0,1), nb=256 ib=32, R-BiDiag"),
    "grad8192": dict(m=8192, n=8192, nb=256, ib=32, variant="bidiag", kind="grad", seeds=(12, 13), tree="auto",
                     desc="differentiation FP64 8192x8192 N(0,1), nb=256 ib=32, BiDiag: forward reduction + adjoint "
                          "(dL/dA from a N(0,1) band gradient W, L = <W, B>)"),
    "grad4096x1024": dict(m=4096, n=1024, nb=256, ib=32, variant="bidiag", kind="grad", seeds=(7, 8),
                          desc="differentiation FP64 4096x1024 N(0,1), nb=256 ib=32, BiDiag: forward reduction "
                               "+ adjoint (dL/dA from a N(0,1) band gradient W, L = <W, B>)"),
}
# FP64 peak of the GB300 from its unit counts and clock: 152 SMs x 2 FP64 FMA/clock/SM (4 flops) x
# 2070 MHz = 1258.6 GFLOP/s.  Reported beside the measured peaks; the roofline divides by the measured
# DFMA-loop rate (bidiag_measure_fp64_peaks), the FP64 unit the reduction's contractions run on.
FP64_DERIVED_GFLOPS = 152 * 4 * 2.070
# DRAM bytes (read + write) of one executor launch on the 8192^2 Auto workload, from the ncu capture
# summarised under profiles/exec_kernel_square8192_launches.md (set to None when the kernel changes).
EXEC_TRAFFIC_BYTES = 11638296576 + 11605000704
CPU_SAMPLE_SECONDS = 12.0


def measure_peaks(G, torch, local, f32):
    """Measured denominators, taken on this GPU before the timed region: the FP64 DFMA and FP64 MMA
    loops of the library's probe, cuBLAS DGEMM (torch.matmul, FP64, 4096^3) and, for the split-precision
    form, cuBLAS TF32 (torch.matmul, FP32 with TF32 allowed, 8192^3); best of several runs each."""
    out = {}
    fma, mma = G.bidiag_measure_fp64_peaks(local, None)
    out["fp64_dfma_loop_gflops"] = fma
    out["fp64_mma_loop_gflops"] = mma
    out["fp64_derived_gflops"] = FP64_DERIVED_GFLOPS

    def best_rate(dtype, nsz, reps):
        a = torch.randn(nsz, nsz, dtype=dtype, device=f"cuda:{local}")
        b = torch.randn(nsz, nsz, dtype=dtype, device=f"cuda:{local}")
        best = 0.0
        for r in range(reps + 1):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b)
            e1.record()
            torch.cuda.synchronize()
            if r:
                best = max(best, 2.0 * nsz ** 3 / (e0.elapsed_time(e1) * 1e-3) / 1e9)
        del a, b
        return best

    out["fp64_dgemm_gflops"] = best_rate(torch.float64, 4096, 3)
    if f32:
        prev = torch.backends.cuda.matmul.allow_tf32
        torch.backends.cuda.matmul.allow_tf32 = True
        try:
            out["tf32_gemm_gflops"] = best_rate(torch.float32, 8192, 10)
        finally:
            torch.backends.cuda.matmul.allow_tf32 = prev
    torch.cuda.empty_cache()
    return out


def roofline_peak(peaks, f32):
    """(peak GFLOP/s, bound, source) of the reduction's executor: FP64 storage against the measured
    DFMA loop; FP32 storage against the measured TF32 GEMM rate over the three TF32 products that
    make one useful product."""
    if f32:
        return (peaks["tf32_gemm_gflops"] / 3.0, "tensor",
                "measured: cuBLAS TF32 GEMM 8192^3 (torch.matmul) / 3 products per useful flop")
    return (peaks["fp64_dfma_loop_gflops"], "alu",
            "measured: FP64 DFMA loop (bidiag_measure_fp64_peaks), all SMs")


def cpu_info():
    """Host threads the oracle may use (this process's CPU affinity) and the CPU model name."""
    threads = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() == "Model name":
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as fh:
                for line in fh:
                    if line.lower().startswith("model name"):
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    import platform
    return {"threads": threads, "model": model or platform.processor() or platform.machine()}


def cpu_env(threads):
    """Environment of an oracle subprocess: its BLAS may use `threads` threads."""
    t = str(threads)
    return dict(os.environ, OPENBLAS_NUM_THREADS=t, OMP_NUM_THREADS=t, MKL_NUM_THREADS=t)


def cpu_baseline_entry(value, info, r, sample):
    """cpu_baseline object: BLAS threads allowed, the CPU time / wall time the oracle actually used,
    the CPU model and the sample it ran on."""
    eff = r.get("cpu_seconds", 0.0) / r["seconds"] if r.get("seconds") else None
    return {"value": value, "unit": "TFLOP/s", "cores": info["threads"],
            "cores_effective": round(eff, 2) if eff is not None else None, "cpu_model": info["model"],
            "kind": "oracle", "sample": sample}


TABLE1_WEIGHTS = (4, 6, 6, 12, 2, 6, 0)   # GEQRT, UNMQR, TSQRT, TSMQR, TTQRT, TTMQR, COPY in nb^3/3 flops


def table1_flops(G, m, n, nb, tree, variant, resources):
    """Algorithmic flops of the executed task list (Table 1 weights x nb^3 / 3), the roofline's work:
    it counts what the kernels do (R-BiDiag and three-step do fewer flops than 4mn^2 - 4n^3/3)."""
    import numpy as np
    p, q = -(-m // nb), -(-n // nb)
    tk, _, _ = G.bidiag_plan_tasks(p, q, tree, variant, resources)
    return float(np.asarray(TABLE1_WEIGHTS)[tk[:, 0]].sum()) * nb ** 3 / 3.0


SUBTASK_NAMES = {1: "UNMQR strip", 3: "TSMQR strip", 5: "TTMQR strip", 6: "COPY", 7: "PF", 8: "PU",
                 9: "adjoint PF", 10: "adjoint PU", 11: "adjoint strip", 12: "adjoint COPY", 13: "adjoint reduce"}
PANEL_KINDS = {0: "GE", 1: "TS", 2: "TT"}
UPDATE_UNITS = {1: 6, 3: 12, 5: 6}        # Table 1 units (nb^3/3 flops) of a whole tile update


def subtask_class(op):
    typ, kind, blk = op & 15, (op >> 24) & 3, (op >> 16) & 0xff
    if typ in (7, 8, 9, 10):
        return f"{SUBTASK_NAMES[typ]} {PANEL_KINDS.get(kind, '?')}"
    return SUBTASK_NAMES.get(typ, f"type {typ}")


def subtask_bytes_flops(op, nb, ib, w, esize):
    """Algorithmic global-memory bytes (loads + stores of the tiles it stages) and flops of one
    sub-task of the executor, from its op word (the blocks each sub-task moves: see kernels.cu)."""
    typ, kind, strip, blk = op & 15, (op >> 24) & 3, (op >> 8) & 0xff, (op >> 16) & 0xff
    c0 = blk * ib
    if typ == 7:                          # PF(b): the block's columns of the panel (and pivot triangle)
        rows = nb - c0 if kind == 0 else (nb if kind == 1 else c0 + ib)
        elems = 2 * rows * ib + ib * ib + (0 if kind == 0 else ib * (ib + 1))
        return elems * esize, None
    if typ == 8:                          # PU(b, s): block b applied to column block s of the panel
        rows = nb - c0 if kind == 0 else (nb if kind == 1 else c0 + ib)
        elems = 2 * rows * ib + rows * ib + ib * ib + (0 if kind == 0 else 2 * ib * ib)
        return elems * esize, None
    if typ in (1, 3, 5):                  # update strip: all blocks of the tile on ncols columns
        ncols = min(w, nb - strip * w)
        nblk = nb // ib
        vrows = sum((nb - b * ib) if typ == 1 else (nb if typ == 3 else (b + 1) * ib) for b in range(nblk))
        elems = 2 * nb * ncols + vrows * ib + nblk * ib * ib + (0 if typ == 1 else 2 * nblk * ib * ncols)
        return elems * esize, UPDATE_UNITS[typ] * nb * nb * ncols / 3.0
    if typ == 6:
        return 2 * nb * nb * esize, None
    return 0, None


def trace_report(h, nb, ib, esize, nsm, title, w=32):
    """Markdown summary of the last traced launch: per sub-task class its count, time, share of the
    busy time, algorithmic bytes and GB/s (flops and GFLOP/s for the update strips); SM occupancy;
    and the critical chain (walking back from the last sub-task through the dependency that finished
    last), split into sub-task time by class and waiting gaps."""
    import numpy as np
    tr = h.trace()
    prog, deps = h.trace_program()
    n = len(tr)
    start, end, op = tr[:, 0].astype(np.float64), tr[:, 1].astype(np.float64), tr[:, 3].astype(np.int64)
    dur = end - start
    t0, t1 = start.min(), end.max()
    cls = [subtask_class(int(o)) for o in op]
    stats = {}
    for y in range(n):
        b, f = subtask_bytes_flops(int(op[y]), nb, ib, w, esize)
        s = stats.setdefault(cls[y], [0, 0.0, 0.0, 0.0, 0.0])
        s[0] += 1
        s[1] += dur[y]
        s[2] += b
        s[3] += f or 0.0
    busy = dur.sum()
    tc5 = int(((op >> 32) & 1).sum())
    nupd = int(sum(1 for o in op if (int(o) & 15) in (1, 3, 5, 8)))
    lines = [f"### {title}", "",
             f"launch span {1e-6 * (t1 - t0):.2f} ms, {n} sub-tasks, SMs busy {busy / (nsm * (t1 - t0)):.1%} "
             f"of the span ({nsm} SMs)" + (f"; {tc5} of {nupd} update sub-tasks ran C -= V W on tcgen05"
                                           if tc5 else ""), "",
             "| sub-task | count | total ms | share of busy | mean us | alg. bytes | GB/s | GFLOP/s |",
             "|---|---|---|---|---|---|---|---|"]
    for k in sorted(stats, key=lambda c: -stats[c][1]):
        c, tot, by, fl, _ = stats[k]
        lines.append(f"| {k} | {c} | {1e-6 * tot:.2f} | {tot / busy:.1%} | {1e-3 * tot / c:.1f} | "
                     f"{by / c / 1e3:.0f} KB | {by / tot:.1f} | " + (f"{fl / tot:.1f} |" if fl else "- |"))
    # critical chain
    y = int(np.argmax(end))
    chain_t, gaps, steps = {}, 0.0, 0
    while True:
        chain_t[cls[y]] = chain_t.get(cls[y], 0.0) + dur[y]
        steps += 1
        d0, d1 = int(prog[y, 5]), int(prog[y, 6])
        ds = [int(d) for d in deps[d0:d1] if 0 <= int(d) < n]
        if not ds:
            gaps += start[y] - t0
            break
        p = max(ds, key=lambda d: end[d])
        gaps += max(0.0, start[y] - end[p])
        y = p
    lines += ["", f"critical chain: {steps} sub-tasks, {1e-6 * (sum(chain_t.values()) + gaps):.2f} ms "
                  f"= sub-task time {1e-6 * sum(chain_t.values()):.2f} ms + waiting gaps {1e-6 * gaps:.2f} ms", "",
              "| on the chain | ms | share of span |", "|---|---|---|"]
    for k in sorted(chain_t, key=lambda c: -chain_t[c]):
        lines.append(f"| {k} | {1e-6 * chain_t[k]:.2f} | {chain_t[k] / (t1 - t0):.1%} |")
    lines.append(f"| waiting gaps | {1e-6 * gaps:.2f} | {gaps / (t1 - t0):.1%} |")
    return "\n".join(lines) + "\n"


def metric_flops(m, n):
    return 4.0 * m * n * n - 4.0 * n ** 3 / 3.0


def batch_shapes(seed, count=512):
    import numpy as np
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        m = int(rng.integers(64, 1025))
        out.append((m, int(rng.integers(32, m + 1))))
    return out


def make_input(w, rank, device):
    from paper_1611_06892_gb300 import inputs
    m, n = w["m"], w["n"]
    if w["kind"] == "sv":
        s = inputs.geometric_sv(n)
        su, sv = w["seeds"]
        return inputs.torch_prescribed_singular_values(m, n, s, su + 1000 * rank, sv + 1000 * rank, device)
    return inputs.torch_gaussian(m, n, w["seeds"][0] + 1000 * rank, device)


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.lines = []
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(gpu_index)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        # NCCL between GPUs; gloo when there is no GPU (the multi-process CPU tests)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return world, rank, local


def max_over_ranks(x, world, device):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def variant_code(v):
    """bidiag | rbidiag | auto | threestep | threestep:S | an integer code -> the library's variant code."""
    if isinstance(v, int):
        return v
    v = str(v)
    if v.startswith("threestep:"):
        return 4 + int(v.split(":", 1)[1])
    if v.lstrip("-").isdigit():
        return int(v)
    return {"bidiag": 0, "rbidiag": 1, "auto": 2, "threestep": 3}[v]


def cpu_sample(path, w, tree, seconds, max_tasks=None):
    """Times the oracle on the first tasks of the workload's task list (wall and process CPU time)."""
    import numpy as np

    from oracle import bidiag as OB
    from oracle import trees as T

    A = np.load(path, mmap_mode="r")
    variant = variant_code(w["variant"])
    treec = {"flatts": T.FLATTS, "flattt": T.FLATTT, "greedy": T.GREEDY, "auto": T.AUTO}[tree]
    p, q = -(-A.shape[0] // w["nb"]), -(-A.shape[1] // w["nb"])
    if variant == 2:      # the shorter critical path of the two variants (Sec. 4.3.3)
        cb = T.critical_path(p, q, treec, T.BIDIAG, w["resources"])
        cr = T.critical_path(p, q, treec, T.RBIDIAG, w["resources"])
        variant = T.RBIDIAG if cr < cb else T.BIDIAG
    elif variant == 3:    # the best three-step split (Sec. 4.5)
        variant = T.THREESTEP + T.best_split(p, q, treec, w["resources"])[0]
    st = OB.new_state(np.asarray(A), w["nb"], w["ib"], treec, variant, resources=w["resources"])
    units = 0
    done = 0
    t0, c0 = time.perf_counter(), time.process_time()
    for idx, t in enumerate(st["tasks"]):
        OB.run_tasks(st, [(idx, t)])
        units += T.WEIGHT[t[0]]
        done += 1
        if time.perf_counter() - t0 > seconds or (max_tasks and done >= max_tasks):
            break
    el, cpu = time.perf_counter() - t0, time.process_time() - c0
    flops = units * w["nb"] ** 3 / 3.0
    return {"tasks": done, "total_tasks": len(st["tasks"]), "flops": flops, "seconds": el, "cpu_seconds": cpu}


def run_cpu_sample_subprocess(A_host_np, w, tree, seconds, max_tasks=None, threads=None):
    import numpy as np
    with tempfile.TemporaryDirectory() as td:
        path = os.path.join(td, "A.npy")
        np.save(path, A_host_np)
        env = cpu_env(threads or cpu_info()["threads"])
        cmd = [sys.executable, os.path.abspath(__file__), "--cpu-sample", path, "--workload", w["name"],
               "--tree", tree, "--cpu-seconds", str(seconds), "--auto-resources", str(w["resources"]),
               "--variant", str(w.get("variant_used", w["variant"]))]
        if max_tasks:
            cmd += ["--cpu-max-tasks", str(max_tasks)]
        out = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=1800)
        if out.returncode != 0:
            raise RuntimeError(out.stderr[-2000:])
        return json.loads(out.stdout.strip().splitlines()[-1])


def cpu_sample_batch(path, seconds):
    """Times the oracle on the first matrices of the batch with their tuned configs."""
    import numpy as np

    from oracle import bidiag as OB

    data = np.load(path)
    flops = 0.0
    done = 0
    t0, c0 = time.perf_counter(), time.process_time()
    k = 0
    while f"A{k}" in data.files:
        A = data[f"A{k}"]
        nb, ib, tree, variant = (int(x) for x in data[f"cfg{k}"])
        OB.bidiag_band(A, nb, ib, tree, variant, resources=1)
        flops += metric_flops(*A.shape)
        done += 1
        k += 1
        if time.perf_counter() - t0 > seconds:
            break
    return {"tasks": done, "total_tasks": 512, "flops": flops, "seconds": time.perf_counter() - t0,
            "cpu_seconds": time.process_time() - c0}


def reference_batched(args, w, base):
    """The oracle on the batch: each step reduces the next matrices of the batch (nb = 128, ib = 32,
    FlatTS, the variant with the shorter critical path) for a bounded time, BLAS on the host's cores."""
    import numpy as np

    from oracle import trees as OT
    from paper_1611_06892_gb300 import inputs

    shapes = batch_shapes(w["seeds"][0])
    per_step = max(2.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    info = cpu_info()
    res = []
    k = 0
    with tempfile.TemporaryDirectory() as td:
        for _ in range(args.warmup + args.steps):
            path = os.path.join(td, "batch.npz")
            sample = {}
            for j in range(64):
                m, n = shapes[(k + j) % len(shapes)]
                p, q = -(-m // 128), -(-n // 128)
                v = OT.BIDIAG if OT.critical_path(p, q, OT.FLATTS, OT.BIDIAG) <= \
                    OT.critical_path(p, q, OT.FLATTS, OT.RBIDIAG) else OT.RBIDIAG
                sample[f"A{j}"] = inputs.gaussian(m, n, seed=w["seeds"][0] + k + j)
                sample[f"cfg{j}"] = np.array([128, 32, OT.FLATTS, v])
            np.savez(path, **sample)
            out = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-sample-batch", path,
                                  "--cpu-seconds", str(per_step)], env=cpu_env(info["threads"]),
                                 capture_output=True, text=True, timeout=600, check=True)
            r = json.loads(out.stdout.strip().splitlines()[-1])
            k += r["tasks"]
            res.append(r)
    timed = res[args.warmup:]
    val = sum(r["flops"] for r in timed) / sum(r["seconds"] for r in timed) / 1e12
    sample = (f"{sum(r['tasks'] for r in timed)} of the 512 matrices over {len(timed)} steps "
              f"(~{per_step:.0f} s each), nb 128, FlatTS")
    tot = {"seconds": sum(r["seconds"] for r in timed), "cpu_seconds": sum(r["cpu_seconds"] for r in timed)}
    line = dict(base, impl="reference", value=val, ms_per_step=1e3 * statistics.mean(r["seconds"] for r in timed),
                cpu_baseline=cpu_baseline_entry(val, info, tot, sample),
                e2e={"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
                gpu_launches=0)
    print(json.dumps(line), flush=True)
    return 0


def cpu_sample_grad(path, seconds):
    """The oracle forward + adjoint on the sample matrix of the differentiation workload."""
    import numpy as np

    from oracle import adjoint as OA
    from oracle import bidiag as OB
    from oracle import trees as OT

    data = np.load(path)
    A, W = data["A"], data["W"]
    nb, ib = (int(x) for x in data["cfg"])
    done, t0, c0 = 0, time.perf_counter(), time.process_time()
    while True:
        res = OB.bidiag_band(A, nb, ib, OT.GREEDY, OT.BIDIAG)
        OA.band_vjp(res, W)
        done += 1
        if time.perf_counter() - t0 > seconds:
            break
    m, n = A.shape
    return {"tasks": done, "flops": done * metric_flops(m, n), "seconds": time.perf_counter() - t0,
            "cpu_seconds": time.process_time() - c0, "m": m, "n": n}


def grad_cpu_leg(w, seconds):
    """Bounded oracle sample for the differentiation workload: the leading 1024 x 256 block with
    nb = 64 (the same 4:1 shape and 16 x 4 tile grid), forward + adjoint, BLAS on the host's cores."""
    import numpy as np

    from paper_1611_06892_gb300 import inputs
    m, n, nb, ib = 1024, 256, 64, 16
    A = inputs.gaussian(m, n, seed=w["seeds"][0])
    W = inputs.gaussian(nb + 1, n, seed=w["seeds"][1])
    with tempfile.TemporaryDirectory() as td:
        path = os.path.join(td, "grad.npz")
        np.savez(path, A=A, W=W, cfg=np.array([nb, ib]))
        out = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-sample-grad", path, "--cpu-seconds",
                              str(seconds)], env=cpu_env(cpu_info()["threads"]), capture_output=True, text=True,
                             timeout=900, check=True)
    r = json.loads(out.stdout.strip().splitlines()[-1])
    r["sample"] = (f"{r['tasks']} forward + adjoint passes of the oracle on the leading {m} x {n} block "
                   f"(nb {nb}, ib {ib}, Greedy; {r['seconds']:.1f} s)")
    return r


def run_grad(args, w, base, config, world, rank, local, device, G, torch):
    """The differentiation workload: one step = the forward reduction and its adjoint."""
    f32 = args.precision == "f32"
    dt = torch.float32 if f32 else torch.float64
    m, n, nb, ib = w["m"], w["n"], w["nb"], w["ib"]
    from paper_1611_06892_gb300 import inputs
    A = inputs.torch_gaussian(m, n, w["seeds"][0] + 1000 * rank, device)
    if f32:
        A = A.float().t().contiguous().t()
    gen = torch.Generator(device=device)
    gen.manual_seed(w["seeds"][1] + 1000 * rank)
    W = torch.randn((n, nb + 1), dtype=dt, device=device, generator=gen).t()
    tree = config["tree"]
    h = G.Handle(device=local)
    h.set_option(G.OPT_TIMING, 1)
    peaks = measure_peaks(G, torch, local, f32)

    def step():
        r = h.band(A, nb, ib, tree, w["variant"])
        h.sync()
        fms = h.last_exec_ms()
        Ab = r.backward(W)
        h.sync()
        bms = h.last_exec_ms()
        r.free()
        del Ab
        return fms, bms

    for _ in range(args.warmup):
        step()
    sampler = ClockSampler(local) if rank == 0 else None
    barrier(world)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(h.stream)
    ms = [step() for _ in range(args.steps)]
    e1.record(h.stream)
    torch.cuda.synchronize()
    barrier(world)
    clocks = sampler.stop() if sampler else None
    el_ms = max_over_ranks(e0.elapsed_time(e1), world, device)
    flops = metric_flops(m, n)
    ms_per_step = el_ms / args.steps
    value = world * flops / (ms_per_step * 1e-3) / 1e12
    # end to end: A from pinned host memory, forward, adjoint, dL/dA back to pinned host memory
    A_host = torch.empty((n, m), dtype=dt, pin_memory=True).t()
    A_host.copy_(A)
    G_host = torch.empty((n, m), dtype=dt, pin_memory=True).t()
    e2e_t = []
    for _ in range(args.e2e_steps):
        barrier(world)
        t0 = time.perf_counter()
        Ad = A_host.to(device, non_blocking=True)
        r = h.band(Ad, nb, ib, tree, w["variant"])
        Ab = r.backward(W)
        G_host.copy_(Ab, non_blocking=True)
        h.sync()
        torch.cuda.current_stream(device).synchronize()
        e2e_t.append(time.perf_counter() - t0)
        r.free()
    e2e_s = max_over_ranks(statistics.mean(e2e_t), world, device) if e2e_t else None
    fwd_ms = statistics.mean(x[0] for x in ms)
    bwd_ms = statistics.mean(x[1] for x in ms)
    # the adjoint executor's algorithmic work: every update block is undone on the state and on the
    # gradient and contributes its partial products (three times the forward's update flops)
    alg = table1_flops(G, m, n, nb, G.TREES[tree], G.VARIANTS[w["variant"]], 1)
    bwd_flops = 3.0 * alg
    achieved = bwd_flops / (bwd_ms * 1e-3) / 1e9
    peak, bound, src = roofline_peak(peaks, f32)
    line = dict(base, config=config, dtype="f32" if f32 else "f64", value=value, ms_per_step=ms_per_step,
                e2e={"value": world * flops / e2e_s / 1e12 if e2e_s else None, "unit": "TFLOP/s",
                     "h2d_bytes_per_step": m * n * A.element_size(), "d2h_bytes_per_step": m * n * A.element_size()},
                roofline={"bound": bound, "achieved": achieved, "peak": peak, "unit": "GFLOP/s",
                          "frac": achieved / peak, "traffic": None,
                          "kernel": "exec_kernel adjoint instantiation (reverse sweep), 3 x the forward's Table 1 flops",
                          "algorithmic_flops": bwd_flops, "peak_source": src, "peaks_measured": peaks},
                forward_exec_ms=fwd_ms, backward_exec_ms=bwd_ms, backward_over_forward=bwd_ms / fwd_ms,
                gpu_launches=(7 if w["variant"] == "bidiag" else 8) * args.steps, clocks=clocks)
    if world == 1 and rank == 0 and not args.no_cpu and not f32:
        r = grad_cpu_leg(w, CPU_SAMPLE_SECONDS)
        line["cpu_baseline"] = cpu_baseline_entry(r["flops"] / r["seconds"] / 1e12, cpu_info(), r, r["sample"])
    if rank == 0:
        print(json.dumps(line), flush=True)
    h.close()
    return 0


def run_batched(args, w, base, config, world, rank, local, device, G, torch):
    """The batched workload: 512 uneven matrices reduced in one persistent launch per step."""
    import numpy as np

    f32 = args.precision == "f32"
    dt = torch.float32 if f32 else torch.float64
    shapes = batch_shapes(w["seeds"][0] + 1000 * rank)
    gen = torch.Generator(device=device)
    gen.manual_seed(w["seeds"][0] + 1000 * rank)
    As = [torch.randn(n, m, dtype=dt, device=device, generator=gen).t() for m, n in shapes]
    flops = sum(metric_flops(m, n) for m, n in shapes)
    h = G.Handle(device=local)
    h.set_option(G.OPT_TIMING, 1)
    peaks = measure_peaks(G, torch, local, f32)
    nsm = torch.cuda.get_device_properties(local).multi_processor_count
    if args.batch_config:        # one fixed (nb, ib, tree) for every matrix; variant by critical path
        fnb, fib, ftree = args.batch_config.split(",")
        fixed = dict(nb=[int(fnb)] * len(As), ib=[int(fib)] * len(As), tree=[ftree] * len(As),
                     variant=["auto"] * len(As))
        cfgs = []
        for m, n in shapes:
            p, q = -(-m // int(fnb)), -(-n // int(fnb))
            R = max(1, nsm * min(int(fnb), 32) * (2 if f32 else 1) // int(fnb))
            cfgs.append((int(fnb), int(fib), G.TREES[ftree], G.bidiag_plan_choose_variant(p, q, G.TREES[ftree], R)[0]))
    else:
        fixed = {}
        cfgs = [G.bidiag_autotune(m, n, nsm, 4 if f32 else 8) for m, n in shapes]

    def step():
        res = h.band_batched(As, **fixed)
        h.sync()
        ms = h.last_exec_ms()
        for r in res:
            r.free()
        return ms

    for _ in range(args.warmup):
        step()
    sampler = ClockSampler(local) if rank == 0 else None
    barrier(world)
    torch.cuda.synchronize()
    stream = h.stream
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    exec_ms = [step() for _ in range(args.steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clocks = sampler.stop() if sampler else None
    el_ms = max_over_ranks(e0.elapsed_time(e1), world, device)
    ms_per_step = el_ms / args.steps
    value = world * flops / (ms_per_step * 1e-3) / 1e12
    # end to end: H2D of the 512 inputs from pinned memory, the batched call, D2H of the 512 bands
    hosts = [torch.empty((A.shape[1], A.shape[0]), dtype=dt, pin_memory=True).t().copy_(A) for A in As]
    e2e_t = []
    for _ in range(args.e2e_steps):
        barrier(world)
        t0 = time.perf_counter()
        dev = [x.to(device, non_blocking=True) for x in hosts]
        res = h.band_batched(dev, **fixed)
        bands = [r.band().cpu() for r in res]
        e2e_t.append(time.perf_counter() - t0)
        d2h = sum(x.numel() * x.element_size() for x in bands)
        for r in res:
            r.free()
        del dev, bands
    e2e_s = max_over_ranks(statistics.mean(e2e_t), world, device) if e2e_t else None
    h2d = sum(m * n for m, n in shapes) * (4 if f32 else 8)
    if not e2e_t:
        d2h = 0
    exec_mean = statistics.mean(exec_ms)
    alg = sum(table1_flops(G, m, n, c[0], c[2], c[3], max(1, nsm * min(c[0], 32) * (2 if f32 else 1) // c[0]))
              for (m, n), c in zip(shapes, cfgs))
    achieved = alg / (exec_mean * 1e-3) / 1e9
    peak, bound, src = roofline_peak(peaks, f32)
    if args.batch_config:
        config = dict(config, nb=int(fnb), ib=int(fib), tree=ftree, workload=config["workload"].replace(
            "autotuned nb / ib / tree / variant per matrix", f"fixed nb={fnb} ib={fib} tree={ftree}, variant by critical path"))
    line = dict(base, config=config, dtype="f32" if f32 else "f64", value=value, ms_per_step=ms_per_step,
                e2e={"value": world * flops / e2e_s / 1e12 if e2e_s else None, "unit": "TFLOP/s",
                     "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
                roofline={"bound": bound, "achieved": achieved, "peak": peak, "unit": "GFLOP/s",
                          "frac": achieved / peak, "traffic": None,
                          "kernel": "exec_kernel (persistent dataflow executor, whole batch)",
                          "algorithmic_flops": alg, "peak_source": src, "peaks_measured": peaks},
                exec_ms=exec_ms, gpu_launches=3 * args.steps, clocks=clocks)
    if world == 1 and rank == 0 and not args.no_cpu and not f32:
        with tempfile.TemporaryDirectory() as td:
            path = os.path.join(td, "batch.npz")
            sample = {}
            for k in range(8):
                sample[f"A{k}"] = As[k].double().cpu().numpy()
                sample[f"cfg{k}"] = np.array(cfgs[k])
            np.savez(path, **sample)
            info = cpu_info()
            out = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-sample-batch", path,
                                  "--cpu-seconds", str(CPU_SAMPLE_SECONDS)], env=cpu_env(info["threads"]),
                                 capture_output=True, text=True, timeout=600)
            if out.returncode == 0:
                r = json.loads(out.stdout.strip().splitlines()[-1])
                line["cpu_baseline"] = cpu_baseline_entry(
                    r["flops"] / r["seconds"] / 1e12, info, r,
                    f"first {r['tasks']} of 512 matrices with their tuned configurations ({r['seconds']:.1f} s)")
    if rank == 0:
        print(json.dumps(line), flush=True)
    h.close()
    return 0


AUTOTUNE_CONFIGS = [(32, 8), (32, 16), (32, 32), (64, 8), (64, 16), (64, 32), (128, 8), (128, 16), (128, 32)]
AUTOTUNE_CLASSES = ["PF GE", "PF TS", "PF TT", "PU GE", "PU TS", "PU TT", "UNMQR strip", "TSMQR strip",
                    "TTMQR strip"]


def calibrate_autotune(args, w, G, torch, local, device, path):
    """Calibration table of the batched form's autotuner: mean execution time of each sub-task class
    (panel factor / panel update per panel kind, update strip per kernel) for every candidate (nb, ib),
    measured on the 512-matrix batch reduced with that (nb, ib) for all matrices, once with FlatTS (TS
    kernels) and once with Greedy (TT kernels), traced.  Rows of this storage precision replace those
    in `path` (a C include file compiled into the planner)."""
    import numpy as np
    f32 = args.precision == "f32"
    dt = torch.float32 if f32 else torch.float64
    esize = 4 if f32 else 8
    shapes = batch_shapes(w["seeds"][0])
    gen = torch.Generator(device=device)
    gen.manual_seed(w["seeds"][0])
    As = [torch.randn(n, m, dtype=dt, device=device, generator=gen).t() for m, n in shapes]
    count = len(As)
    h = G.Handle(device=local)
    rows = []
    for nb, ib in AUTOTUNE_CONFIGS:
        durs = {c: [] for c in AUTOTUNE_CLASSES}
        for tree in ("flatts", "greedy"):
            cfg = dict(nb=[nb] * count, ib=[ib] * count, tree=[tree] * count, variant=["auto"] * count)
            for r in h.band_batched(As, **cfg):      # warm-up (plans the batch)
                r.free()
            h.sync()
            h.set_option(G.OPT_TRACE, 1)
            res = h.band_batched(As, **cfg)
            h.sync()
            h.set_option(G.OPT_TRACE, 0)
            tr = h.trace()
            for r in res:
                r.free()
            for (t0, t1, _, op) in tr:
                c = subtask_class(int(op))
                if c in durs:
                    durs[c].append(1e-3 * (t1 - t0))
        rows.append((nb, ib, [float(np.mean(durs[c])) if durs[c] else 0.0 for c in AUTOTUNE_CLASSES],
                     [len(durs[c]) for c in AUTOTUNE_CLASSES]))
    h.close()
    keep = []
    if os.path.exists(path):
        with open(path) as fh:
            keep = [l for l in fh if l.startswith("{") and not l.startswith("{%d," % esize)]
    nsm = torch.cuda.get_device_properties(local).multi_processor_count
    with open(path, "w") as fh:
        fh.write("// Autotuner calibration (generated): mean execution time in microseconds of each executor\n"
                 "// sub-task class, {element bytes, nb, ib, {PF GE, PF TS, PF TT, PU GE, PU TS, PU TT,\n"
                 "// UNMQR strip, TSMQR strip, TTMQR strip}}, measured on a GPU with %d SMs (%s) reducing the\n"
                 "// 512-matrix batch (m ~ U[64, 1024], n ~ U[32, m], N(0,1), seed 6) with one (nb, ib) for all\n"
                 "// matrices, FlatTS and Greedy, traced.  Written by\n"
                 "//   python bench.py --workload batched512 [--precision f32] --calibrate-autotune <this file>\n"
                 % (nsm, torch.cuda.get_device_name(local)))
        for l in keep:
            fh.write(l)
        for nb, ib, us, _ in rows:
            fh.write("{%d, %d, %d, {%s}},\n" % (esize, nb, ib, ", ".join("%.2f" % x for x in us)))
    print(json.dumps({"calibrated": path, "esize": esize,
                      "rows": [{"nb": nb, "ib": ib, "us": dict(zip(AUTOTUNE_CLASSES, us)),
                                "samples": dict(zip(AUTOTUNE_CLASSES, cnt))} for nb, ib, us, cnt in rows]}))
    return 0


def workload_config(args, w, config):
    """The `config` object of both arms (ours and the reference) for the batched and the
    differentiation workloads; the single-matrix workloads keep the generic one."""
    f32 = args.precision == "f32"
    if w["kind"] == "grad":
        m, n = w["m"], w["n"]
        config = dict(config, workload=w["desc"].replace("FP64", "FP32 storage (3xTF32 updates)") if f32 else w["desc"],
                      tree=w.get("tree", "greedy") if args.tree == "auto" else args.tree,
                      l2=f"input {m * n * (4 if f32 else 8) / 2**20:.0f} MiB (the adjoint's working set, 3 copies "
                         "of A plus partial sums, exceeds the 129 MB L2; no flush)")
        config.pop("auto_resources", None)
    elif w["kind"] == "batch":
        config = dict(config, workload=w["desc"] + (", FP32 storage (3xTF32 updates)" if f32 else ", FP64"),
                      count=512, m="U[64,1024]", n="U[32,m]", nb="autotuned", ib="autotuned",
                      tree="autotuned", variant="critical path",
                      l2="inputs 1.1 GB total > 129 MB L2 (no flush needed)")
        config.pop("auto_resources", None)
    return config


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="square8192", choices=sorted(WORKLOADS))
    ap.add_argument("--tree", default="auto", choices=("flatts", "flattt", "greedy", "auto"))
    ap.add_argument("--variant", default=None,
                    help="bidiag | rbidiag | auto | threestep (best split) | threestep:S (default: the workload's)")
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--precision", default="f64", choices=("f64", "f32"),
                    help="f32: FP32 storage with 3xTF32 tensor-core updates and FP64 reflector norms")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-sample", default=None)
    ap.add_argument("--cpu-seconds", type=float, default=CPU_SAMPLE_SECONDS)
    ap.add_argument("--cpu-max-tasks", type=int, default=None)
    ap.add_argument("--cpu-sample-batch", default=None)
    ap.add_argument("--cpu-sample-grad", default=None)
    ap.add_argument("--calibrate-autotune", default=None,
                    help="batched512 only: measure the autotuner's per-sub-task times for every candidate (nb, ib) "
                         "and write them to this C include file (instead of the benchmark)")
    ap.add_argument("--batch-config", default=None,
                    help="batched512 only: nb,ib,tree for every matrix instead of the autotuner's choices")
    ap.add_argument("--f32-updates", type=int, default=None,
                    help="FP32 storage: 0 = tcgen05 + warp-level tensor cores (default), 1 = FFMA, 2 = warp-level only")
    ap.add_argument("--strip-width", type=int, default=None,
                    help="column-strip width of the update sub-tasks (16, 32 or 64; default: the library's 32)")
    ap.add_argument("--trace-summary", default=None,
                    help="after the timed region, trace one more reduction and append its per-sub-task summary "
                         "(markdown) to this file")
    ap.add_argument("--auto-resources", type=int, default=None,
                    help="R of the Auto tree (default: SMs * 32 / nb, twice that for FP32 storage, as the library chooses)")
    args = ap.parse_args()
    w = dict(WORKLOADS[args.workload], name=args.workload)
    if args.variant:
        w["variant"] = args.variant
    if args.workload == "square512" and args.tree == "auto":
        args.tree = "flatts"

    w["resources"] = args.auto_resources
    if args.cpu_sample_grad:
        print(json.dumps(cpu_sample_grad(args.cpu_sample_grad, args.cpu_seconds)))
        return 0
    if args.cpu_sample_batch:
        print(json.dumps(cpu_sample_batch(args.cpu_sample_batch, args.cpu_seconds)))
        return 0
    if args.cpu_sample:
        r = cpu_sample(args.cpu_sample, w, args.tree, args.cpu_seconds, args.cpu_max_tasks)
        print(json.dumps(r))
        return 0

    world, rank, local = dist_setup()
    import numpy as np
    import torch

    if torch.cuda.is_available():
        torch.cuda.set_device(local)
        device = f"cuda:{local}"
    else:
        device = "cpu"          # only the reference (oracle) arm runs without a GPU
    if w["resources"] is None and w["nb"]:
        # the library's default R of the Auto tree: SMs x strip width / nb, twice that for FP32 storage
        nsm = torch.cuda.get_device_properties(local).multi_processor_count if torch.cuda.is_available() else 152
        w["resources"] = max(1, nsm * 32 * (2 if args.precision == "f32" else 1) // w["nb"])
    m, n, nb, ib = w["m"], w["n"], w["nb"], w["ib"]
    flops = metric_flops(m, n)
    f32 = args.precision == "f32"
    desc = w["desc"].replace("FP64", "FP32 storage (3xTF32 updates)") if f32 else w["desc"]
    config = {"workload": desc + f", tree={args.tree}" + (f", variant={args.variant}" if args.variant else ""),
              "m": m, "n": n, "nb": nb, "ib": ib,
              "tree": args.tree, "variant": w["variant"], "auto_resources": w["resources"],
              "l2": f"input {m * n * 8 / 2**20:.0f} MiB > 129 MB L2 (no flush needed)" if m * n * 8 > 129e6
              else "input smaller than L2"}
    config = workload_config(args, w, config)
    base = {"metric": "GE2BND TFLOP/s (4mn^2 - 4n^3/3 flops)", "unit": "TFLOP/s", "higher_is_better": True,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if f32 else "f64", "data": "synthetic", "config": config}

    if args.impl == "reference" and w["kind"] == "batch":
        if rank != 0:
            return 0
        return reference_batched(args, w, base)
    if args.impl == "reference" and w["kind"] == "grad":
        if rank != 0:
            return 0
        per_step = max(2.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
        res = [grad_cpu_leg(w, per_step) for _ in range(args.warmup + args.steps)][args.warmup:]
        val = sum(r["flops"] for r in res) / sum(r["seconds"] for r in res) / 1e12
        tot = {"seconds": sum(r["seconds"] for r in res), "cpu_seconds": sum(r["cpu_seconds"] for r in res)}
        line = dict(base, impl="reference", value=val, ms_per_step=1e3 * statistics.mean(r["seconds"] for r in res),
                    cpu_baseline=cpu_baseline_entry(val, cpu_info(), tot, res[0]["sample"]),
                    e2e={"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
                    gpu_launches=0)
        print(json.dumps(line), flush=True)
        return 0
    if args.impl == "reference":
        # the plain CPU oracle on bounded samples of the same workload; rank 0 only
        if rank != 0:
            return 0
        A = make_input(w, 0, device)
        A_host = A.cpu().numpy()
        del A
        torch.cuda.empty_cache()
        per_step = max(2.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
        if args.cpu_seconds != CPU_SAMPLE_SECONDS:
            per_step = args.cpu_seconds
        info = cpu_info()
        full = w["name"] == "square512"      # the oracle's size: every step is the whole reduction
        res = [run_cpu_sample_subprocess(A_host, w, args.tree, 1e9 if full else per_step, threads=info["threads"])
               for _ in range(args.warmup + args.steps)]
        timed = res[args.warmup:]
        val = sum(r["flops"] for r in timed) / sum(r["seconds"] for r in timed) / 1e12
        sample = (f"the whole task list ({timed[0]['total_tasks']} tasks) each step" if full else
                  f"first {timed[0]['tasks']} of {timed[0]['total_tasks']} tasks of the task list "
                  f"(~{per_step:.0f} s each step)")
        tot = {"seconds": sum(r["seconds"] for r in timed), "cpu_seconds": sum(r["cpu_seconds"] for r in timed)}
        line = dict(base, impl="reference", value=val, ms_per_step=1e3 * statistics.mean(r["seconds"] for r in timed),
                    cpu_baseline=cpu_baseline_entry(val, info, tot, sample),
                    e2e={"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
                    gpu_launches=0)
        print(json.dumps(line), flush=True)
        return 0

    import paper_1611_06892_gb300 as G
    if not os.path.exists(G.LIB_PATH):
        from paper_1611_06892_gb300 import build
        build.build()
    G.load_library()
    if w["kind"] == "batch" and args.calibrate_autotune:
        return calibrate_autotune(args, w, G, torch, local, device, args.calibrate_autotune)
    if w["kind"] == "batch":
        return run_batched(args, w, base, config, world, rank, local, device, G, torch)
    if w["kind"] == "grad":
        return run_grad(args, w, base, config, world, rank, local, device, G, torch)

    A = make_input(w, rank, device)
    if f32:
        A = A.float().t().contiguous().t()
    h = G.Handle(device=local)
    h.set_option(G.OPT_TIMING, 1)
    h.set_option(G.OPT_AUTO_RESOURCES, w["resources"])
    if args.strip_width:
        h.set_option(G.OPT_STRIP, args.strip_width)
        config["strip_width"] = args.strip_width
    if args.f32_updates is not None:
        h.set_option(G.OPT_F32_UPDATES, args.f32_updates)
        config["f32_updates"] = args.f32_updates
    stream = h.stream
    peaks = measure_peaks(G, torch, local, f32)

    vcode = variant_code(w["variant"])

    def step():
        r = h.band(A, nb, ib, args.tree, vcode)
        h.sync()
        ms = h.last_exec_ms()
        w["variant_used"] = int(r.desc.variant)
        r.free()
        return ms

    for _ in range(args.warmup):
        step()
    sampler = ClockSampler(local) if rank == 0 else None
    barrier(world)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    exec_ms = [step() for _ in range(args.steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clocks = sampler.stop() if sampler else None
    el_ms = max_over_ranks(e0.elapsed_time(e1), world, device)
    ms_per_step = el_ms / args.steps
    value = world * flops / (ms_per_step * 1e-3) / 1e12

    # end to end with host buffers, copies inside the timed region: FP64 through the host-buffer entry
    # point (bidiag_band_host), FP32 storage through the binding (pinned H2D, bidiag_band_f32, band D2H)
    dt = torch.float32 if f32 else torch.float64
    A_host = torch.empty((n, m), dtype=dt, pin_memory=True).t()
    A_host.copy_(A)
    ab_host = torch.empty((n, nb + 1), dtype=dt, pin_memory=True).t()
    e2e_t = []
    for _ in range(args.e2e_steps):
        barrier(world)
        t0 = time.perf_counter()
        if f32:
            Ad = A_host.to(device, non_blocking=True)
            r = h.band(Ad, nb, ib, args.tree, vcode)
            ab_host.copy_(r.band(), non_blocking=True)
            h.sync()
            torch.cuda.current_stream(device).synchronize()
            r.free()
        else:
            G.bidiag_band_host(h.h, m, n, A_host.data_ptr(), m, nb, ib, G.TREES[args.tree], vcode,
                               ab_host.data_ptr(), nb + 1)
        e2e_t.append(time.perf_counter() - t0)
    e2e_s = max_over_ranks(statistics.mean(e2e_t), world, device) if e2e_t else None
    if args.trace_summary and rank == 0:
        h.set_option(G.OPT_TRACE, 1)
        r = h.band(A, nb, ib, args.tree, vcode)
        h.sync()
        r.free()
        h.set_option(G.OPT_TRACE, 0)
        nsm = torch.cuda.get_device_properties(local).multi_processor_count
        title = f"{config['workload']}" + (f", R = {w['resources']}" if args.tree == "auto" else "")
        with open(args.trace_summary, "a") as fh:
            fh.write(trace_report(h, nb, ib, A.element_size(), nsm, title) + "\n")

    exec_mean = statistics.mean(exec_ms)
    alg = table1_flops(G, m, n, nb, G.TREES[args.tree], w.get("variant_used", vcode), w["resources"])
    achieved = alg / (exec_mean * 1e-3) / 1e9
    peak, bound, peak_src = roofline_peak(peaks, f32)
    unit = "GFLOP/s"
    line = dict(base, value=value, ms_per_step=ms_per_step,
                variant_used=w.get("variant_used"),       # the library's code (4 + s: three-step, split s)
                e2e={"value": world * flops / e2e_s / 1e12 if e2e_s else None, "unit": "TFLOP/s",
                     "h2d_bytes_per_step": m * n * A.element_size(),
                     "d2h_bytes_per_step": (nb + 1) * n * A.element_size()},
                roofline={"bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
                          "frac": achieved / peak, "traffic": EXEC_TRAFFIC_BYTES if (not f32 and w["name"] == "square8192" and args.tree == "auto") else None,
                          "kernel": "exec_kernel (persistent dataflow executor)", "algorithmic_flops": alg,
                          "peak_source": peak_src, "peaks_measured": peaks},
                exec_ms=exec_ms, gpu_launches=3 * args.steps, clocks=clocks)
    if world == 1 and rank == 0 and not args.no_cpu and not f32:
        A_np = A.cpu().numpy()
        info = cpu_info()
        full = w["name"] == "square512"      # the oracle's size: timed on the whole reduction
        r = run_cpu_sample_subprocess(A_np, w, args.tree, 1e9 if full else CPU_SAMPLE_SECONDS, threads=info["threads"])
        sample = (f"the whole reduction ({r['total_tasks']} tasks, {r['seconds']:.1f} s)" if full else
                  f"first {r['tasks']} of {r['total_tasks']} tasks of the same task list ({r['seconds']:.1f} s)")
        line["cpu_baseline"] = cpu_baseline_entry(r["flops"] / r["seconds"] / 1e12, info, r, sample)
        if full:
            r1 = run_cpu_sample_subprocess(A_np, w, args.tree, 1e9, threads=1)
            line["cpu_baseline_one_thread"] = cpu_baseline_entry(
                r1["flops"] / r1["seconds"] / 1e12, dict(info, threads=1), r1,
                f"the whole reduction, one BLAS thread ({r1['seconds']:.1f} s)")
    if rank == 0:
        print(json.dumps(line), flush=True)
    h.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
