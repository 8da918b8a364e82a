"""Host-side checks of the adjoint program (the reverse sweep of bidiag_band_backward), no GPU.

* Every forward sub-task is undone exactly once, by the adjoint sub-task of the matching kind.
* Race and order check: every element of the working state / gradient that two adjoint sub-tasks
  touch (one writing it) is ordered by the dependency DAG, and in the REVERSE of the forward order of
  their counterparts; every partial slot is written by one sub-task that precedes the factor sub-task
  reading it.  Footprints are modelled from what the CUDA sub-tasks load and store.
* The slot table covers each panel task's update strips and panel-block updates exactly once.
* Panels with at least eight update strips get a reduced slot: reduction sub-tasks, which follow every
  update strip of the panel, sum the strips' partials block by block over row chunks that tile the
  block's rows, and the factor sub-task of a block follows its reductions.
* Slot storage is recycled: logical slots that share storage have the same size and range, distinct
  storage ranges never overlap, and for consecutive owners of one range every reader and writer of the
  earlier owner precedes every writer of the later one in the DAG.
"""
import numpy as np
import pytest

import paper_1611_06892_gb300 as G

UNMQR, TSMQR, TTMQR, COPY, PF, PU = 1, 3, 5, 6, 7, 8
BPF, BPU, BUPD, BCOPY, BRED = 9, 10, 11, 12, 13
RED_ELEMS, RED_MIN = 2048, 8
GE, TS, TT = 0, 1, 2


def fields(t):
    op = int(t[0])
    return dict(typ=op & 15, tr=(op >> 4) & 1, half=(op >> 5) & 1, strip=(op >> 8) & 0xFF, blk=(op >> 16) & 0xFF, kind=(op >> 24) & 3,
                x=int(t[1]), a=int(t[2]), c=int(t[3]), tslot=int(t[4]), flags=int(t[7]))


def state_footprint(f, nb, ib, w, pus=1):
    """Elements (tile, row, col) of the working state / gradient an adjoint sub-task reads or writes."""
    tr = f["tr"]
    out = set()

    def region(ref, r0, c0, rows, cols, upper=False, orient=True):
        buf = ref >> 28
        assert buf in (2, 3), "adjoint sub-tasks address the state buffers"
        idx = ref & 0x0FFFFFFF
        for r in range(rows):
            for cc in range(cols):
                R, C = r0 + r, c0 + cc
                if upper and R > C:
                    continue
                out.add((buf, idx) + ((C, R) if (tr and orient) else (R, C)))

    def update(utype, Cp, C, blk0, blk1, col0, ncols):
        row_lo = blk0 * ib if utype == UNMQR else 0
        row_hi = blk1 * ib if utype == TTMQR else nb
        region(C, row_lo, col0, row_hi - row_lo, ncols)
        if utype != UNMQR:
            for b in range(blk0, blk1):
                region(Cp, b * ib, col0, ib, ncols)

    nblk = nb // ib
    typ, blk, kind = f["typ"], f["blk"], f["kind"]
    if typ == BPF:
        c0 = blk * ib
        if kind == GE:
            region(f["c"], c0, c0, nb - c0, ib)
        else:
            region(f["a"], c0, c0, ib, ib, upper=True)
            region(f["c"], 0, c0, nb if kind == TS else c0 + ib, ib, upper=(kind == TT))
    elif typ == BPU:
        utype = {GE: UNMQR, TS: TSMQR, TT: TTMQR}[kind]
        pw = ib // pus
        update(utype, f["a"], f["c"], blk, blk + 1, f["strip"] * ib + f["half"] * pw, pw)
    elif typ == BUPD:
        utype = (UNMQR, TSMQR, TTMQR)[kind]
        col0 = f["strip"] * w
        update(utype, f["a"], f["c"], 0, nblk, col0, min(w, nb - col0))
    elif typ == BCOPY:
        diag = f["flags"] & 1
        region(f["x"], 0, 0, nb, nb, upper=bool(diag), orient=False)
        region(f["c"], 0, 0, nb, nb, upper=bool(diag), orient=False)
    return out


def check_backward(m, n, nb, ib, tree, variant, strip_w, state=True):
    fprog, fdeps, w = G.bidiag_plan_program(m, n, nb, ib, tree, variant, resources=2, strip_w=strip_w)
    prog, fwd, deps, slot_off, pinfo, wb = G.bidiag_plan_backward(m, n, nb, ib, tree, variant, resources=2,
                                                                  strip_w=strip_w)
    nsub = len(prog)
    nblk = nb // ib
    # every forward sub-task is undone: once, or (update strips) by column pieces of width wb that
    # tile its columns exactly
    assert set(fwd.tolist()) == set(range(len(fprog)))
    split = w // wb
    assert split in (1, 2) and wb * split == w
    # panel-block updates with ib >= 16 are undone as two column halves (op bit 5 = half)
    pus = 2 if any(fields(t)["typ"] == BPU and fields(t)["half"] for t in prog) else 1
    if nb > ib:
        assert pus == (2 if ib >= 16 and ib % 2 == 0 else 1)
    for y in range(len(fprog)):
        ys = [z for z in range(nsub) if fwd[z] == y and fields(prog[z])["typ"] != BRED]
        g = fields(fprog[y])
        if g["typ"] in (UNMQR, TSMQR, TTMQR):
            cols = sorted(fields(prog[z])["strip"] for z in ys)
            want = [g["strip"] * split + hh for hh in range(split) if (g["strip"] * split + hh) * wb < nb]
            assert cols == want
        elif g["typ"] == PU:
            assert sorted(fields(prog[z])["half"] for z in ys) == list(range(pus))
        else:
            assert len(ys) == 1
    # kinds match the forward sub-tasks they undo
    kind_map = {PF: BPF, PU: BPU, UNMQR: BUPD, TSMQR: BUPD, TTMQR: BUPD, COPY: BCOPY}
    for y in range(nsub):
        f, g = fields(prog[y]), fields(fprog[fwd[y]])
        if f["typ"] == BRED:        # serves the factor sub-task of the same block
            assert g["typ"] == PF and (f["blk"], f["kind"], f["tslot"]) == (g["blk"], g["kind"], g["tslot"])
            continue
        assert f["typ"] == kind_map[g["typ"]]
        if f["typ"] in (BPF, BPU):
            assert (f["blk"], f["kind"], f["tslot"], f["x"]) == (g["blk"], g["kind"], g["tslot"], g["x"])
            assert f["c"] == g["x"] + (2 << 28) and f["a"] == (g["a"] + (2 << 28) if g["a"] >= 0 else -1)
        if f["typ"] == BUPD:
            assert f["kind"] == {UNMQR: 0, TSMQR: 1, TTMQR: 2}[g["typ"]] and f["strip"] // split == g["strip"]
    # ancestors in the adjoint DAG
    anc = [0] * nsub
    for y in range(nsub):
        acc = 0
        for d in deps[prog[y, 5]:prog[y, 6]]:
            d = int(d)
            assert d < y
            acc |= anc[d] | (1 << d)
        anc[y] = acc
    # state / gradient: conflicts ordered in reverse forward order
    touch = {}
    for y in range(nsub if state else 0):
        for e in state_footprint(fields(prog[y]), nb, ib, wb, pus):
            touch.setdefault(e, []).append(y)
    for e, ys in touch.items():
        ys = sorted(ys, key=lambda y: -fwd[y])        # the order the reverse sweep must follow
        for i in range(1, len(ys)):
            assert (anc[ys[i]] >> ys[i - 1]) & 1, f"state element {e}: adjoint {ys[i - 1]} must precede {ys[i]}"
    # slots: one writer each, before the factor sub-task of the block that reads it
    writer = {}
    for y in range(nsub):
        f = fields(prog[y])
        if f["typ"] in (BPU, BUPD):
            assert f["flags"] not in writer, "a partial slot with two writers"
            writer[f["flags"]] = y
            t = pinfo[f["tslot"]]
            if f["typ"] == BUPD:
                assert t[0] <= f["flags"] < t[0] + t[1]
            else:
                b, s = f["blk"], f["strip"]
                assert f["flags"] == t[2] + (b * nblk - b * (b + 1) // 2 + (s - b - 1)) * pus + f["half"]
    # reductions: (panel, block) -> chunk -> sub-task; each follows every update strip of its panel
    red = {}
    readers, writers = {}, {sl: [y] for sl, y in writer.items()}
    for y in range(nsub):
        f = fields(prog[y])
        if f["typ"] != BRED:
            continue
        t = pinfo[f["tslot"]]
        writers.setdefault(int(t[3]), []).append(y)
        for sl in range(t[0], t[0] + t[1]):
            readers.setdefault(sl, []).append(y)
        assert t[3] >= 0 and t[1] >= RED_MIN
        chunks = red.setdefault((f["tslot"], f["blk"]), {})
        assert f["strip"] not in chunks
        chunks[f["strip"]] = y
        for sl in range(t[0], t[0] + t[1]):
            assert (anc[y] >> writer[sl]) & 1, f"reduction {y} before update slot {sl}"
    nred = 0
    for y in range(nsub):
        f = fields(prog[y])
        if f["typ"] != BPF:
            continue
        t = pinfo[f["tslot"]]
        b = f["blk"]
        assert (t[3] >= 0) == (t[1] >= RED_MIN)
        if t[3] >= 0:
            vrows = nb - b * ib if f["kind"] == GE else (nb if f["kind"] == TS else (b + 1) * ib)
            rows = max(1, RED_ELEMS // ib)
            chunks = red.pop((f["tslot"], b))
            assert sorted(chunks) == list(range(-(-vrows // rows)))
            for z in chunks.values():
                assert (anc[y] >> z) & 1, f"factor sub-task {y} before its reduction {z}"
            reads = [int(t[3])]
            nred += b == 0
        else:
            reads = list(range(t[0], t[0] + t[1]))
        reads += [t[2] + (b * nblk - b * (b + 1) // 2 + (s - b - 1)) * pus + hh for s in range(b + 1, nblk)
                  for hh in range(pus)]
        for sl in reads:
            readers.setdefault(sl, []).append(y)
            if sl == t[3]:          # its block's reductions precede it (checked above)
                continue
            assert sl in writer and (anc[y] >> writer[sl]) & 1, f"slot {sl} not written before its reader {y}"
    assert not red, "a reduction without its factor sub-task"
    assert len(writer) + nred == len(slot_off) - 1
    # slot storage: sizes nb^2 + nb ib (update strips, reduced slots) and nb ib + ib^2 (panel-block
    # updates); logical slots sharing storage are its consecutive owners (in the order of their first
    # writers), each owner's readers and writers precede the next owner's writers
    nlog = len(slot_off) - 1
    size = np.zeros(nlog, dtype=np.int64)
    npu = nblk * (nblk - 1) // 2 * pus
    for t in pinfo:
        size[t[0]:t[0] + t[1]] = nb * nb + nb * ib
        size[t[2]:t[2] + npu] = nb * ib + ib * ib
        if t[3] >= 0:
            size[t[3]] = nb * nb + nb * ib
    assert (size > 0).all()
    groups = {}
    for sl in range(nlog):
        groups.setdefault(int(slot_off[sl]), []).append(sl)
    ends = sorted((off, off + int(size[g[0]])) for off, g in groups.items())
    for (o0, e0), (o1, _) in zip(ends, ends[1:]):
        assert e0 <= o1, "storage ranges overlap"
    assert ends[-1][1] <= slot_off[-1]
    for off, g in groups.items():
        assert len({int(size[sl]) for sl in g}) == 1
        g = sorted(g, key=lambda sl: min(writers[sl]))
        for a, b in zip(g, g[1:]):
            for wy in writers[b]:
                for z in writers[a] + readers.get(a, []):
                    assert (anc[wy] >> z) & 1, f"storage at {off}: owner {a} (sub-task {z}) not before {b} ({wy})"
    return nsub


@pytest.mark.parametrize("variant", (0, 1), ids=("bidiag", "rbidiag"))
@pytest.mark.parametrize("tree", (0, 1, 2, 3), ids=("flatts", "flattt", "greedy", "auto"))
def test_adjoint_program_order(tree, variant):
    # 3 x 3 ragged tiles, nb = 8, two inner blocks, strips of 4 columns
    assert check_backward(22, 20, 8, 4, tree, variant, strip_w=4) > 0
    # nb = 32 with strips of 16 columns: undone as two 8-column halves each, the last tile ragged
    assert check_backward(70, 40, 32, 8, tree, variant, strip_w=16) > 0
    # ib = 16: the panel-block update adjoints are split into two 8-column halves too
    assert check_backward(70, 40, 32, 16, tree, variant, strip_w=16) > 0
    # 5 x 2 tiles, inner block = tile
    assert check_backward(20, 8, 4, 4, tree, variant, strip_w=32) > 0
    # three inner blocks per tile, strips of two blocks
    assert check_backward(30, 18, 6, 2, tree, variant, strip_w=4) > 0


def test_checker_catches_a_reversed_edge(monkeypatch):
    """Drop the dependencies of one factor adjoint: the checker must report it."""
    real = G.bidiag_plan_backward

    def broken(*args, **kw):
        prog, fwd, deps, slot_off, pinfo, wb = real(*args, **kw)
        prog = prog.copy()
        y = [i for i in range(len(prog)) if (prog[i, 0] & 15) == BPF and prog[i, 6] > prog[i, 5]][-1]
        prog[y, 6] = prog[y, 5]
        return prog, fwd, deps, slot_off, pinfo, wb

    monkeypatch.setattr(G, "bidiag_plan_backward", broken)
    with pytest.raises(AssertionError):
        check_backward(22, 20, 8, 4, 2, 0, strip_w=4)


@pytest.mark.parametrize("split", (1, 2))
@pytest.mark.parametrize("tree", (0, 1, 2, 3), ids=("flatts", "flattt", "greedy", "auto"))
def test_adjoint_program_order_three_step(tree, split):
    assert check_backward(22, 20, 8, 4, tree, 4 + split, strip_w=4) > 0
    assert check_backward(30, 18, 6, 2, tree, 4 + split, strip_w=4) > 0


@pytest.mark.parametrize("variant", (0, 1), ids=("bidiag", "rbidiag"))
@pytest.mark.parametrize("tree", (0, 2), ids=("flatts", "greedy"))
def test_adjoint_program_reductions(tree, variant):
    """Tall enough that panels have many update strips: reductions appear and are ordered."""
    prog = G.bidiag_plan_backward(100, 40, 8, 4, tree, variant, resources=2, strip_w=4)[0]
    assert any((int(op) & 15) == BRED for op in prog[:, 0])
    assert check_backward(100, 40, 8, 4, tree, variant, strip_w=4) > 0
    # ib = 2: 1024-row chunks cover a block in one chunk; ib = 8 with nb = 32: 256-row chunks
    assert check_backward(130, 24, 6, 2, tree, variant, strip_w=2) > 0
    assert check_backward(300, 64, 32, 8, tree, variant, strip_w=16) > 0
    # nb = 256, ib = 32: 64-row chunks, four per block (slot and order checks only)
    assert check_backward(1600, 512, 256, 32, tree, variant, strip_w=32, state=False) > 0


def test_checker_catches_shared_live_storage(monkeypatch):
    """Give two update strips of the same panel (independent sub-tasks, both live until the panel's
    factor adjoints) the same storage: the storage check must report it."""
    real = G.bidiag_plan_backward

    def broken(*args, **kw):
        prog, fwd, deps, slot_off, pinfo, wb = real(*args, **kw)
        slot_off = slot_off.copy()
        t = next(t for t in pinfo if t[1] >= 2)
        slot_off[t[0] + 1] = slot_off[t[0]]
        return prog, fwd, deps, slot_off, pinfo, wb

    monkeypatch.setattr(G, "bidiag_plan_backward", broken)
    with pytest.raises(AssertionError):
        check_backward(100, 40, 8, 4, 0, 1, strip_w=4)
