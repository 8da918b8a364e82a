"""Reduction trees, canonical task lists and the task-DAG model of tiled BiDiag / R-BiDiag.

ORACLE - test infrastructure only.  Nothing in the product path imports this module; it is used by
``tests/``, by ``__graft_entry__.smoke()`` and by the ``cpu_baseline`` / reference legs of ``bench.py``.
It shares no code with the CUDA path (the C++ planner is an independent implementation of the same
rules, and the tests compare the two).

Everything is written from the paper (Faverge, Langou, Robert, Dongarra, "Bidiagonalization with
parallel tiled algorithms", arXiv 1611.06892):

* Algorithm 1 (tiled QR(p,q)), Algorithm 2 (elim via TS kernels), Algorithm 3 (elim via TT kernels),
  and the rule that a tile already in triangle form is not factored again (end of Sec. 3.2).
* Sec. 3.3: the FlatTS, FlatTT and Greedy trees.
* Sec. 3.4: BiDiag = QR(1); LQ(1); QR(2); ...; LQ(q-1); QR(q), LQ(k) per Algorithm 4.
* Sec. 3.5: R-BiDiag = QR(p,q); LQ(1); QR(2); ...; QR(q).
* Sec. 5: the Auto tree (FlatTS groups of size a joined by a Greedy tree of TT kernels, with a chosen
  per step so that ceil(rows/a) * cols >= gamma * resources, gamma = 2).
* Table 1: kernel weights in units of nb^3/3 flops, used by the critical-path model of Sec. 4.

Conventions (0-based tile indices).  Each step is described in *oriented* coordinates: a QR step k
works on tile column k of its matrix; an LQ step k works on the transpose, so oriented tile (a, b) of
an LQ step is actual tile (b, a).  A task is a tuple ``(type, phase, k, i, piv, j)``:

* ``type``  - one of GEQRT, UNMQR, TSQRT, TSMQR, TTQRT, TTMQR (LQ steps use the same kernels on the
  transposed geometry; their paper names are GELQT, UNMLQ, ...), or COPY (R-BiDiag only).
* ``phase`` - PQR (R-BiDiag pre-QR on the m x n matrix), QR or LQ (BiDiag steps; in R-BiDiag these run
  on the separate n x n matrix holding R).
* ``k`` step, ``i`` oriented row of the factored / eliminated tile, ``piv`` oriented pivot row,
  ``j`` oriented column of the updated tile; -1 where unused.  COPY(i, j) copies the R part of actual
  tile (i, j), i <= j < q, into the n x n matrix of the second phase.

Readings where the paper is silent (each also listed in the design notes):

* Greedy pairing (one step): with ready rows r_0 < ... < r_{z-1} and h = floor(z/2), rows
  r_{z-h+t} are eliminated into r_{z-2h+t}, t = 0..h-1; the eliminated rows are dropped and this repeats
  while z > 1.  It has depth ceil(log2 z), as Sec. 4 requires.
* Greedy for the multi-column pre-QR of R-BiDiag: time-stepped; at time s the rows ready in column k are
  those eliminated in column k-1 at a time < s (every row for k = 0) and not yet eliminated in column k;
  the halving rule is applied to that set.  Program order is by (s, k).
* Auto: u and v are the live counts of panel tiles and trailing tiles of the step; a is the largest
  value in [1, u] with ceil(u/a) * v >= gamma * R, else 1; groups are consecutive; the heads are joined
  by the halving Greedy rule with TT kernels.
* LQ(k) (Algorithm 4): panel = tile row k, tiles k+1..q-1; the diagonal pivot is tile (k, k+1).
* R-BiDiag second phase runs on rows 0..q-1 only, on a separate copy of R (the pre-QR reflectors keep
  their storage, Sec. 3.6 "Memory usage").
"""
from __future__ import annotations

import math

# tree codes
FLATTS, FLATTT, GREEDY, AUTO = 0, 1, 2, 3
TREE_NAMES = {FLATTS: "flatts", FLATTT: "flattt", GREEDY: "greedy", AUTO: "auto"}
# variant codes; three-step with split s (Sec. 4.5: s BiDiag steps, then R-BiDiag on the trailing
# (p - s) x (q - s) tiles) is THREESTEP + s
BIDIAG, RBIDIAG = 0, 1
THREESTEP = 4
# phases
QR, LQ, PQR = 0, 1, 2
# task types
GEQRT, UNMQR, TSQRT, TSMQR, TTQRT, TTMQR, COPY = 0, 1, 2, 3, 4, 5, 6
TYPE_NAMES = {GEQRT: "GEQRT", UNMQR: "UNMQR", TSQRT: "TSQRT", TSMQR: "TSMQR",
              TTQRT: "TTQRT", TTMQR: "TTMQR", COPY: "COPY"}
LQ_NAMES = {GEQRT: "GELQT", UNMQR: "UNMLQ", TSQRT: "TSLQT", TSMQR: "TSMLQ",
            TTQRT: "TTLQT", TTMQR: "TTMLQ"}
# elimination kinds
TS, TT = 0, 1

# Table 1 weights, unit nb^3/3 flops.  COPY is a data move, weight 0.
WEIGHT = {GEQRT: 4, UNMQR: 6, TSQRT: 6, TSMQR: 12, TTQRT: 2, TTMQR: 6, COPY: 0}

PANEL_TYPES = (GEQRT, TSQRT, TTQRT)


def greedy_rounds(rows):
    """Halving Greedy tree on sorted panel rows; list of rounds, each a list of (i, piv)."""
    rows = list(rows)
    rounds = []
    while len(rows) > 1:
        z = len(rows)
        h = z // 2
        rnd = [(rows[z - h + t], rows[z - 2 * h + t]) for t in range(h)]
        rounds.append(rnd)
        gone = {i for i, _ in rnd}
        rows = [r for r in rows if r not in gone]
    return rounds


def auto_group_size(u, v, resources, gamma=2):
    """Sec. 5: largest a in [1, u] with ceil(u/a) * v >= gamma * resources; 1 if none qualifies."""
    for a in range(u, 0, -1):
        if -(-u // a) * v >= gamma * resources:
            return a
    return 1


def step_eliminations(rows, v, tree, resources=None, gamma=2):
    """Eliminations (i, piv, kind) of one QR/LQ step on panel rows ``rows`` (sorted), ``v`` trailing tiles."""
    rows = list(rows)
    if tree == FLATTS:
        return [(r, rows[0], TS) for r in rows[1:]]
    if tree == FLATTT:
        return [(r, rows[0], TT) for r in rows[1:]]
    if tree == GREEDY:
        return [(i, piv, TT) for rnd in greedy_rounds(rows) for (i, piv) in rnd]
    if tree == AUTO:
        if resources is None:
            raise ValueError("Auto tree needs the resource count")
        a = auto_group_size(len(rows), v, resources, gamma)
        groups = [rows[s:s + a] for s in range(0, len(rows), a)]
        el = [(r, g[0], TS) for g in groups for r in g[1:]]
        heads = [g[0] for g in groups]
        el += [(i, piv, TT) for rnd in greedy_rounds(heads) for (i, piv) in rnd]
        return el
    raise ValueError(f"unknown tree {tree}")


def greedy_multicolumn(p, q):
    """Time-stepped Greedy for the full QR(p, q) (R-BiDiag pre-QR).  Returns [(k, i, piv)] in (s, k) order."""
    kmax = min(p, q)
    elim_time = {}          # (row, col) -> time step of its elimination in that column
    remaining = [p - 1 - k for k in range(kmax)]   # eliminations still to do per column
    out = []
    s = 0
    while any(remaining):
        for k in range(kmax):
            if not remaining[k]:
                continue
            if k == 0:
                ready = [i for i in range(p) if (i, 0) not in elim_time]
            else:
                ready = [i for i in range(k, p)
                         if elim_time.get((i, k - 1), s) < s and (i, k) not in elim_time]
            z = len(ready)
            h = z // 2
            for t in range(h):
                i, piv = ready[z - h + t], ready[z - 2 * h + t]
                elim_time[(i, k)] = s
                out.append((k, i, piv))
                remaining[k] -= 1
        s += 1
    return out


def split_of(variant):
    """Number of BiDiag steps before the switch to R-BiDiag: 0 for R-BiDiag, s for THREESTEP + s,
    None for BiDiag (no second phase)."""
    if variant == BIDIAG:
        return None
    if variant == RBIDIAG:
        return 0
    if variant >= THREESTEP:
        return variant - THREESTEP
    raise ValueError(f"unknown variant {variant}")


def task_buffer(phase, k, variant):
    """Matrix a task works on: 0 = A (m x n), 1 = the R copy of the second phase.  The second phase is
    the BiDiag of the trailing R: its LQ steps k >= s and QR steps k >= s + 1 (QR(s) is the pre-QR)."""
    s = split_of(variant)
    if s is None or phase == PQR:
        return 0
    return 1 if (phase == LQ and k >= s) or (phase == QR and k > s) else 0


def _steps(p, q, variant):
    """(first-phase steps, second-phase steps), each a list of (phase, k, panel_rows, ntrail) in
    sequence order (Sec. 3.4 / 3.5; the three-step of Sec. 4.5 runs s BiDiag steps on A, the pre-QR of
    the trailing tiles, then BiDiag on their R)."""
    first, second = [], []
    s = split_of(variant)
    if s is not None and not 0 <= s < q:
        raise ValueError("three-step split must be in [0, q)")
    for k in range(q if s is None else s):
        first.append((QR, k, list(range(k, p)), q - k - 1))
        if k < q - 1:
            first.append((LQ, k, list(range(k + 1, q)), p - k - 1))
    if s is not None:
        for k in range(s, q - 1):
            second.append((LQ, k, list(range(k + 1, q)), q - k - 1))
            second.append((QR, k + 1, list(range(k + 1, q)), q - k - 2))
    return first, second


def _elim_tasks(phase, k, elims, ntrail_cols, tasks, tri):
    """Expand eliminations into kernel tasks (Algorithms 2 and 3, skipping already-triangular tiles)."""
    jcols = list(range(k + 1, k + 1 + ntrail_cols))

    def factor(r):
        if (phase, k, r) in tri:
            return False
        tri.add((phase, k, r))
        tasks.append((GEQRT, phase, k, r, -1, -1))
        return True

    for (i, piv, kind) in elims:
        if kind == TS:
            fp = factor(piv)
            tasks.append((TSQRT, phase, k, i, piv, -1))
            for j in jcols:
                if fp:
                    tasks.append((UNMQR, phase, k, piv, -1, j))
                tasks.append((TSMQR, phase, k, i, piv, j))
        else:
            fp = factor(piv)
            fi = factor(i)
            for j in jcols:
                if fp:
                    tasks.append((UNMQR, phase, k, piv, -1, j))
                if fi:
                    tasks.append((UNMQR, phase, k, i, -1, j))
            tasks.append((TTQRT, phase, k, i, piv, -1))
            for j in jcols:
                tasks.append((TTMQR, phase, k, i, piv, j))


def _single_tile(phase, k, row, ntrail_cols, tasks, tri):
    """A step whose panel has one tile: GEQRT plus its UNMQR updates."""
    if (phase, k, row) in tri:
        return
    tri.add((phase, k, row))
    tasks.append((GEQRT, phase, k, row, -1, -1))
    for j in range(k + 1, k + 1 + ntrail_cols):
        tasks.append((UNMQR, phase, k, row, -1, j))


def _preqr_eliminations(p, q, s, tree, resources, gamma):
    """Eliminations [(k, i, piv, kind)] of the pre-QR of tiles s..p-1 x s..q-1, in program order."""
    if tree == GREEDY:
        return [(k + s, i + s, piv + s, TT) for (k, i, piv) in greedy_multicolumn(p - s, q - s)]
    return [(k, i, piv, kind) for k in range(s, q)
            for (i, piv, kind) in step_eliminations(range(k, p), q - k - 1, tree, resources, gamma)]


def eliminations(p, q, tree, variant, resources=None, gamma=2):
    """Canonical elimination list [(phase, k, i, piv, kind)] in program order."""
    out = []
    first, second = _steps(p, q, variant)
    for (phase, k, rows, ntrail) in first:
        for (i, piv, kind) in step_eliminations(rows, ntrail, tree, resources, gamma):
            out.append((phase, k, i, piv, kind))
    s = split_of(variant)
    if s is not None:
        for (k, i, piv, kind) in _preqr_eliminations(p, q, s, tree, resources, gamma):
            out.append((PQR, k, i, piv, kind))
    for (phase, k, rows, ntrail) in second:
        for (i, piv, kind) in step_eliminations(rows, ntrail, tree, resources, gamma):
            out.append((phase, k, i, piv, kind))
    return out


def task_list(p, q, tree, variant, resources=None, gamma=2):
    """Canonical kernel task list [(type, phase, k, i, piv, j)] in program order."""
    if not (p >= q >= 1):
        raise ValueError("need p >= q >= 1 tiles")
    tasks = []
    tri = set()

    def run_steps(steps):
        for (phase, k, rows, ntrail) in steps:
            el = step_eliminations(rows, ntrail, tree, resources, gamma)
            if el:
                _elim_tasks(phase, k, el, ntrail, tasks, tri)
            else:
                _single_tile(phase, k, rows[0], ntrail, tasks, tri)

    first, second = _steps(p, q, variant)
    run_steps(first)
    s = split_of(variant)
    if s is not None:
        if tree == GREEDY:
            # time-stepped multi-column greedy: program order by (time, column)
            by_col = set()
            for (k, i, piv, kind) in _preqr_eliminations(p, q, s, tree, resources, gamma):
                _elim_tasks(PQR, k, [(i, piv, kind)], q - k - 1, tasks, tri)
                by_col.add(k)
            for k in range(s, q):
                if k not in by_col:       # single-tile column (p == q, last column)
                    _single_tile(PQR, k, k, q - k - 1, tasks, tri)
        else:
            for k in range(s, q):
                el = step_eliminations(range(k, p), q - k - 1, tree, resources, gamma)
                if el:
                    _elim_tasks(PQR, k, el, q - k - 1, tasks, tri)
                else:
                    _single_tile(PQR, k, k, q - k - 1, tasks, tri)
        for a in range(s, q):
            for b in range(a, q):
                tasks.append((COPY, PQR, -1, a, -1, b))
    run_steps(second)
    return tasks


# ----------------------------------------------------------------------------------------------
# Task-DAG model.  Data items: each tile of each matrix is split into its strict upper part (SU),
# its diagonal (D) and its strict lower part (SL); each panel task also writes its own T factor.
# Dependencies are read-after-write, write-after-write and write-after-read on those items.
# Oriented "upper" of an LQ step is the actual lower triangle, so a TTQRT of an LQ step touches
# D and SL of the actual tile.
# ----------------------------------------------------------------------------------------------
SU, D, SL = 0, 1, 2


def _item(buf, a, b, part):
    return (buf, a, b, part)


def task_access(task, variant):
    """(reads, writes) item sets of a task; matrix 0 is A (m x n), matrix 1 the R copy of R-BiDiag."""
    typ, phase, k, i, piv, j = task
    buf = task_buffer(phase, k, variant)
    lq = phase == LQ

    def act(a, b):
        return (b, a) if lq else (a, b)

    def up(a, b):
        x, y = act(a, b)
        return {_item(buf, x, y, D), _item(buf, x, y, SL if lq else SU)}

    def lo(a, b):
        x, y = act(a, b)
        return {_item(buf, x, y, SU if lq else SL)}

    def full(a, b):
        x, y = act(a, b)
        return {_item(buf, x, y, SU), _item(buf, x, y, D), _item(buf, x, y, SL)}

    if typ == GEQRT:
        return set(), full(i, k)
    if typ == UNMQR:
        return lo(i, k), full(i, j)
    if typ == TSQRT:
        return set(), up(piv, k) | full(i, k)
    if typ == TSMQR:
        return full(i, k), full(piv, j) | full(i, j)
    if typ == TTQRT:
        return set(), up(piv, k) | up(i, k)
    if typ == TTMQR:
        return up(i, k), full(piv, j) | full(i, j)
    if typ == COPY:
        a, b = i, j
        src = ({_item(0, a, a, D), _item(0, a, a, SU)} if a == b else
               {_item(0, a, b, SU), _item(0, a, b, D), _item(0, a, b, SL)})
        dst = {_item(1, a, b, SU), _item(1, a, b, D), _item(1, a, b, SL)}
        return src, dst
    raise ValueError(typ)


def _panel_of(tasks):
    """Map each update task index to the index of the panel task whose reflectors it applies."""
    last = {}
    owner = {}
    for idx, (typ, phase, k, i, piv, j) in enumerate(tasks):
        if typ == GEQRT:
            last[(GEQRT, phase, k, i)] = idx
        elif typ == TSQRT:
            last[(TSQRT, phase, k, i)] = idx
        elif typ == TTQRT:
            last[(TTQRT, phase, k, i)] = idx
        elif typ == UNMQR:
            owner[idx] = last[(GEQRT, phase, k, i)]
        elif typ == TSMQR:
            owner[idx] = last[(TSQRT, phase, k, i)]
        elif typ == TTMQR:
            owner[idx] = last[(TTQRT, phase, k, i)]
    return owner


def dag(tasks, variant, weights=WEIGHT, want_edges=False):
    """Walk the tasks in program order; returns (levels, finish_times, critical_path[, edges]).

    level(t) = 0 without predecessors, else 1 + max level of its predecessors.
    finish(t) = weight(t) + max finish of its predecessors; the critical path is the max finish.
    The reflector object (T factor) of a panel task is an extra item read by its updates.
    """
    owner = _panel_of(tasks)
    last_w = {}                 # item -> task index of the last writer
    readers = {}                # item -> task indices that read it since its last write
    levels = [0] * len(tasks)
    finish = [0] * len(tasks)
    edges = [] if want_edges else None
    for idx, t in enumerate(tasks):
        reads, writes = task_access(t, variant)
        preds = set()
        for it in reads | writes:
            w = last_w.get(it)
            if w is not None:
                preds.add(w)
        for it in writes:
            preds.update(readers.get(it, ()))
        if idx in owner:
            preds.add(owner[idx])   # reflector object (V and T) of the panel task
        preds.discard(idx)
        lv = 0
        fs = 0
        for d in preds:
            lv = max(lv, levels[d] + 1)
            fs = max(fs, finish[d])
        levels[idx] = lv
        finish[idx] = fs + weights[t[0]]
        if want_edges:
            edges.append(sorted(preds))
        for it in reads:
            readers.setdefault(it, []).append(idx)
        for it in writes:
            last_w[it] = idx
            readers[it] = []
    cp = max(finish) if finish else 0
    if want_edges:
        return levels, finish, cp, edges
    return levels, finish, cp


def critical_path(p, q, tree, variant, resources=None):
    """Critical path length (Table 1 units) of the task DAG, unbounded resources (Sec. 4 model)."""
    tasks = task_list(p, q, tree, variant, resources)
    return dag(tasks, variant)[2]


def best_split(p, q, tree, resources=None):
    """Sec. 4.5: the three-step split with the shortest critical path, found by trying every
    s in [0, q); ties keep the smallest s.  Returns (s, critical path)."""
    best = None
    for s in range(q):
        c = critical_path(p, q, tree, THREESTEP + s, resources)
        if best is None or c < best[1]:
            best = (s, c)
    return best


def weight_total(tasks):
    """Sum of Table 1 weights over the tasks (total work in nb^3/3 units)."""
    return sum(WEIGHT[t[0]] for t in tasks)
