"""Host model of the executor's claim protocol (no GPU).

The persistent executor's CTAs take sub-tasks with `next_task`: flag words 0 (unclaimed) / 2 (claimed)
/ 1 (done), a look-ahead scan of `window` queue entries from the head for a ready one (claimed with a
compare-and-swap), the head moved over a claimed prefix, and otherwise an in-order claim (atomic
increment of the head, skipping entries claimed out of order) whose dependencies the CTA then waits
for.  This test replays that protocol as a discrete-event simulation on real device programs from the
planner, with random sub-task durations and interleavings, and checks what the protocol promises:
every sub-task runs exactly once, never before its dependencies are done, and the simulation always
finishes (no deadlock) for any number of CTAs and any window, including windows of 0 (strict order).
"""
import heapq
import random

import pytest

import paper_1611_06892_gb300 as G


def simulate(deps_of, n, nctas, window, seed, mutant=None):
    """Runs the claim protocol with nctas agents; returns (start, end, runs) per sub-task.  mutant
    plants a mistake: "no_ready_check" (the scan claims without checking the dependencies and runs at
    once), "no_wait" (a sub-task claimed in queue order runs without waiting for its dependencies).
    CTAs act one at a time (each scan and claim is one step), so races between concurrent scans are not
    modelled."""
    rng = random.Random(seed)
    flag = [0] * n                  # 0 unclaimed, 2 claimed, 1 done
    head = 0
    start = [None] * n
    end = [None] * n
    events = []                     # (time, seq, cta, task or -1 for "look for work")
    seq = 0
    for c in range(nctas):
        heapq.heappush(events, (rng.random() * 1e-3, seq, c, -1))
        seq += 1
    waiting = {}                    # cta -> task it claimed in order and waits for
    runs = [0] * n

    def ready(i):
        return all(flag[d] == 1 for d in deps_of[i])

    def next_task():
        nonlocal head
        h = head                    # one head value for the whole scan
        for base in range(0, window, 32):
            if h >= n:
                return None
            lanes = [h + base + l for l in range(32) if base + l < window and h + base + l < n]
            st = [flag[i] for i in lanes]
            if base == 0:           # move the head over a claimed prefix of the inspected entries
                lane_st = []
                for l in range(32):
                    i = h + base + l
                    if i < n and base + l < window:
                        lane_st.append(flag[i])
                    else:           # not inspected: stops the prefix
                        lane_st.append(0)
                skip = lane_st.index(0) if 0 in lane_st else 32
                if skip and h + skip <= n and head == h:
                    head = h + skip
            for i, s in zip(lanes, st):
                if s == 0 and (mutant == "no_ready_check" or ready(i)) and flag[i] == 0:
                    flag[i] = 2
                    return i
        while True:                 # in-order claim
            i = head
            head += 1
            if i >= n:
                return None
            if flag[i] == 0:
                flag[i] = 2
                return i

    def look_for_work(c, t):
        nonlocal seq
        i = next_task()
        if i is None:
            return                  # queue exhausted: the CTA leaves
        if ready(i) or mutant in ("no_ready_check", "no_wait"):
            runs[i] += 1
            start[i] = t
            heapq.heappush(events, (t + rng.uniform(0.5, 2.0), seq, c, i))
            seq += 1
        else:
            waiting[c] = i          # in-order claim: wait for its dependencies

    steps = 0
    while events:
        steps += 1
        assert steps < 50 * n + 10000, "simulation does not finish"
        t, _, c, task = heapq.heappop(events)
        if task >= 0:               # the sub-task is done: publish, wake waiters whose sub-task is ready
            flag[task] = 1
            end[task] = t
            for cc, wt in sorted(waiting.items()):
                if ready(wt):
                    del waiting[cc]
                    runs[wt] += 1
                    start[wt] = t
                    heapq.heappush(events, (t + rng.uniform(0.5, 2.0), seq, cc, wt))
                    seq += 1
        look_for_work(c, t)
        assert events or not waiting, "CTAs left waiting with nothing running (deadlock)"
    return start, end, runs


def program(shape):
    m, n_, nb, ib, tree, variant, R = shape
    prog, deps, _ = G.bidiag_plan_program(m, n_, nb, ib, G.TREES[tree], G.VARIANTS[variant], R)
    return [list(deps[prog[i, 5]:prog[i, 6]]) for i in range(len(prog))]


def protocol_holds(deps_of, nctas, window, seed, mutant=None):
    n = len(deps_of)
    try:
        start, end, runs = simulate(deps_of, n, nctas, window, seed, mutant)
    except AssertionError:
        return False
    if any(r != 1 for r in runs) or any(e is None for e in end):
        return False
    return all(end[d] <= start[i] for i in range(n) for d in deps_of[i])


SHAPES = [(768, 768, 256, 32, "auto", "bidiag", 3), (640, 384, 128, 32, "greedy", "rbidiag", 1),
          (512, 512, 128, 32, "flatts", "bidiag", 1)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("nctas,window", [(1, 0), (3, 0), (3, 64), (16, 16), (16, 32), (16, 1024), (152, 512)])
def test_claim_protocol_runs_each_task_once_in_dependency_order(shape, nctas, window):
    deps_of = program(shape)
    for i in range(len(deps_of)):
        assert all(d < i for d in deps_of[i])          # the queue order is topological
    for seed in range(3):
        assert protocol_holds(deps_of, nctas, window, seed)


@pytest.mark.parametrize("mutant", ["no_ready_check", "no_wait"])
def test_claim_protocol_model_catches_planted_mistakes(mutant):
    deps_of = program(SHAPES[0])
    assert not all(protocol_holds(deps_of, nctas, window, seed, mutant)
                   for seed in range(3) for nctas, window in ((16, 16), (16, 64), (152, 512)))
