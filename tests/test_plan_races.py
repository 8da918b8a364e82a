"""Host-side race check of the executor's device program (no GPU).

Every sub-task's element-level memory footprint is modelled from what the CUDA sub-task loads and
stores (tile rows/columns, orientation, triangular masks, T blocks).  Two sub-tasks that touch the same
element, one of them writing it, must be ordered by the dependency DAG: otherwise the persistent
executor could run them concurrently on different SMs.
"""
import numpy as np
import pytest

import paper_1611_06892_gb300 as G

UNMQR, TSMQR, TTMQR, COPY, PF, PU = 1, 3, 5, 6, 7, 8
GE, TS, TT = 0, 1, 2


def footprint(t, nb, ib, w, grids):
    """(reads, writes): sets of (buffer, tile, row, col) / ('T', slot, index) for one sub-task."""
    op, x, a, c, tslot = (int(v) for v in t[:5])
    typ, tr, strip, blk, kind = op & 15, (op >> 4) & 1, (op >> 8) & 0xFF, (op >> 16) & 0xFF, (op >> 24) & 3
    reads, writes = set(), set()

    def tile(ref):
        return (ref >> 28, ref & 0x0FFFFFFF)

    def region(ref, r0, c0, rows, cols, mask, out, is_store):
        buf, idx = tile(ref)
        for r in range(rows):
            for cc in range(cols):
                R, C = r0 + r, c0 + cc
                if mask == "upper" and R > C:
                    continue
                if mask == "unitlower" and R <= C and not is_store:
                    continue
                out.add((buf, idx) + ((C, R) if tr else (R, C)))

    def t_block(slot, b, out):
        for o in range(ib * ib):
            out.add(("T", slot, b * ib * ib + o))

    def update(utype, V, Cp, C, blk0, blk1, col0, ncols, notrans=False):
        row_lo = blk0 * ib if utype == UNMQR else 0
        row_hi = blk1 * ib if utype == TTMQR else nb
        region(C, row_lo, col0, row_hi - row_lo, ncols, None, reads, False)
        for b in range(blk0, blk1):
            c0 = b * ib
            if utype == UNMQR:
                region(V, c0, c0, nb - c0, ib, "unitlower", reads, False)
            else:
                vrows = nb if utype == TSMQR else c0 + ib
                region(V, 0, c0, vrows, ib, None if utype == TSMQR else "upper", reads, False)
                region(Cp, c0, col0, ib, ncols, None, reads, False)
                region(Cp, c0, col0, ib, ncols, None, writes, True)
            t_block(tslot, b, reads)
        region(C, row_lo, col0, row_hi - row_lo, ncols, None, writes, True)

    nblk = nb // ib
    if typ == PF:
        c0 = blk * ib
        if kind == GE:
            region(x, c0, c0, nb - c0, ib, None, reads, False)
            region(x, c0, c0, nb - c0, ib, None, writes, True)
        else:
            vrows = nb if kind == TS else c0 + ib
            m = None if kind == TS else "upper"
            region(a, c0, c0, ib, ib, "upper", reads, False)
            region(x, 0, c0, vrows, ib, m, reads, False)
            region(a, c0, c0, ib, ib, "upper", writes, True)
            region(x, 0, c0, vrows, ib, m, writes, True)
        t_block(tslot, blk, writes)
    elif typ == PU:
        utype = {GE: UNMQR, TS: TSMQR, TT: TTMQR}[kind]
        update(utype, x, a, x, blk, blk + 1, strip * ib, ib)
    elif typ in (UNMQR, TSMQR, TTMQR):
        col0 = strip * w
        update(typ, x, a, c, 0, nblk, col0, min(w, nb - col0))
    elif typ == COPY:
        diag = int(t[7]) & 1
        for r in range(nb):
            for cc in range(nb):
                if not (diag and r > cc):
                    reads.add(tile(x) + (r, cc))
                writes.add(tile(c) + (r, cc))
    else:
        raise AssertionError(f"unexpected sub-task type {typ}")
    return reads, writes


def check_program(m, n, nb, ib, tree, variant, strip_w=32):
    prog, deps, w = G.bidiag_plan_program(m, n, nb, ib, tree, variant, resources=2, strip_w=strip_w)
    nsub = len(prog)
    anc = [0] * nsub
    for y in range(nsub):
        b, e = int(prog[y, 5]), int(prog[y, 6])
        acc = 0
        for d in deps[b:e]:
            d = int(d)
            assert d < y, "dependency must point to an earlier queue position"
            acc |= anc[d] | (1 << d)
        anc[y] = acc
    acc_by_elem = {}
    for y in range(nsub):
        rd, wr = footprint(prog[y], nb, ib, w, None)
        for e in rd:
            acc_by_elem.setdefault(e, []).append((y, False))
        for e in wr:
            acc_by_elem.setdefault(e, []).append((y, True))
    for e, lst in acc_by_elem.items():
        writers = [y for y, isw in lst if isw]
        if not writers:
            continue
        others = sorted({y for y, _ in lst})
        for wtr in writers:
            for o in others:
                if o == wtr:
                    continue
                lo, hi = min(o, wtr), max(o, wtr)
                assert (anc[hi] >> lo) & 1, f"unordered conflict on {e} between sub-tasks {lo} and {hi}"
    return nsub


@pytest.mark.parametrize("variant", (0, 1), ids=("bidiag", "rbidiag"))
@pytest.mark.parametrize("tree", (0, 1, 2, 3), ids=("flatts", "flattt", "greedy", "auto"))
def test_device_program_is_race_free(tree, variant):
    # 3 x 3 tiles (ragged), nb = 8 with 2 inner blocks and strips of 4 columns (2 strips per tile)
    assert check_program(22, 20, 8, 4, tree, variant, strip_w=4) > 0
    # 4 x 2 tiles, inner block = tile, strips = tile
    assert check_program(16, 8, 4, 4, tree, variant, strip_w=32) > 0


def test_program_counts():
    prog, deps, w = G.bidiag_plan_program(512, 512, 64, 16, 0, 0, resources=152, strip_w=32)
    assert w == 32
    types = prog[:, 0] & 15
    assert set(np.unique(types)) <= {UNMQR, TSMQR, PF, PU}
    # every panel task has nb/ib factor sub-tasks and (nb/ib)(nb/ib - 1)/2 update sub-tasks
    assert (types == PU).sum() == (types == PF).sum() // 4 * 6


def test_checker_catches_a_missing_dependency(monkeypatch):
    """Drop the dependencies of one factor sub-task: the checker must report an unordered conflict."""
    real = G.bidiag_plan_program

    def broken(*args, **kw):
        prog, deps, w = real(*args, **kw)
        prog = prog.copy()
        pf = [y for y in range(len(prog)) if (prog[y, 0] & 15) == PF and ((prog[y, 0] >> 16) & 0xFF) == 1]
        y = pf[0]
        prog[y, 6] = prog[y, 5]          # no dependencies left
        return prog, deps, w

    monkeypatch.setattr(G, "bidiag_plan_program", broken)
    with pytest.raises(AssertionError, match="unordered conflict"):
        check_program(22, 20, 8, 4, 2, 0, strip_w=4)


@pytest.mark.parametrize("split", (1, 2))
@pytest.mark.parametrize("tree", (0, 1, 2, 3), ids=("flatts", "flattt", "greedy", "auto"))
def test_three_step_program_is_race_free(tree, split):
    """Three-step (Sec. 4.5): BiDiag steps on A, pre-QR of the trailing tiles, BiDiag on their R copy."""
    assert check_program(22, 20, 8, 4, tree, 4 + split, strip_w=4) > 0
    assert check_program(40, 24, 8, 4, tree, 4 + split, strip_w=8) > 0
