"""Host-side checks of the C ABI library (no GPU): it loads, exports every declared symbol, and its
planner reproduces the oracle's elimination lists, task lists, DAG levels and critical paths."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_1611_06892_gb300 as G
from oracle import trees as T

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session", autouse=True)
def built_library():
    if not os.path.exists(G.LIB_PATH):
        from paper_1611_06892_gb300 import build
        build.build()
    return G.load_library()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "bidiag.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bidiag_[a-z_0-9]+)\s*\(", src)))


def test_exports_every_declared_symbol():
    lib = ctypes.CDLL(G.LIB_PATH)
    names = declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name


@pytest.mark.parametrize("variant", (T.BIDIAG, T.RBIDIAG), ids=("bidiag", "rbidiag"))
@pytest.mark.parametrize("tree", (T.FLATTS, T.FLATTT, T.GREEDY, T.AUTO), ids=("flatts", "flattt", "greedy", "auto"))
def test_planner_matches_oracle(tree, variant):
    """Canonical elimination list, task list and level of every task match bit-exact (p, q <= 11)."""
    for p in range(1, 12):
        for q in range(1, p + 1):
            for R in (1, 3, 40):
                el_o = np.array(T.eliminations(p, q, tree, variant, R), dtype=np.int32).reshape(-1, 5)
                el_c = G.bidiag_plan_eliminations(p, q, tree, variant, R)
                assert np.array_equal(el_o, el_c), (p, q, R)
                tasks = T.task_list(p, q, tree, variant, R)
                tk_c, lv_c, cp_c = G.bidiag_plan_tasks(p, q, tree, variant, R)
                assert np.array_equal(np.array(tasks, dtype=np.int32).reshape(-1, 6), tk_c), (p, q, R)
                lv_o, _, cp_o = T.dag(tasks, variant)
                assert np.array_equal(np.array(lv_o, dtype=np.int32), lv_c) and cp_o == cp_c, (p, q, R)


def test_planner_cfg_sizes_match_oracle():
    """The bench's tile grids: 32 x 32 (8192^2, nb 256) and 256 x 4 (65536 x 1024)."""
    for (p, q, variant) in ((32, 32, T.BIDIAG), (256, 4, T.RBIDIAG)):
        for tree in (T.FLATTS, T.GREEDY, T.AUTO):
            tasks = T.task_list(p, q, tree, variant, 152)
            tk_c, lv_c, cp_c = G.bidiag_plan_tasks(p, q, tree, variant, 152)
            assert np.array_equal(np.array(tasks, dtype=np.int32).reshape(-1, 6), tk_c)
            lv_o, _, cp_o = T.dag(tasks, variant)
            assert np.array_equal(np.array(lv_o, dtype=np.int32), lv_c) and cp_o == cp_c


def test_planner_printed_critical_paths():
    """The planner's own DAG reproduces the printed R-BiDiagGreedy values (Sec. 4.3.2)."""
    for p, q, val in ((65, 5, 262), (66, 5, 260), (134, 10, 680), (133, 10, 682), (535, 50, 4946), (534, 50, 4948)):
        assert G.bidiag_plan_tasks(p, q, T.GREEDY, T.RBIDIAG)[2] == val


def test_switch_ratio_q100():
    """Sec. 4.3.3: for q = 100 the BiDiagGreedy / R-BiDiagGreedy crossover is delta_s = 5.67, i.e. it
    lies between p = 566 and p = 568 tiles."""
    q = 100

    def better_r(p):
        return G.bidiag_plan_tasks(p, q, T.GREEDY, T.RBIDIAG)[2] < G.bidiag_plan_tasks(p, q, T.GREEDY, T.BIDIAG)[2]

    assert not better_r(560)
    assert better_r(575)
    lo, hi = 560, 575
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if better_r(mid):
            hi = mid
        else:
            lo = mid
    assert 5.66 <= hi / q <= 5.68


def test_planner_argument_errors():
    lib = G.load_library()
    cnt = ctypes.c_int64()
    assert lib.bidiag_plan_tasks(3, 4, 0, 0, 1, None, None, 0, ctypes.byref(cnt), None) == -1   # q > p
    assert lib.bidiag_plan_tasks(4, 3, 7, 0, 1, None, None, 0, ctypes.byref(cnt), None) == -3
    assert lib.bidiag_plan_tasks(4, 3, 0, 2, 1, None, None, 0, ctypes.byref(cnt), None) == -4    # auto: not a plan
    assert lib.bidiag_plan_tasks(4, 3, 0, 7, 1, None, None, 0, ctypes.byref(cnt), None) == -4    # split 3 >= q
    assert lib.bidiag_plan_eliminations(4, 3, 0, 0, 1, None, 0, None) == -8


def test_choose_variant_follows_critical_paths():
    """BIDIAG_AUTO_VARIANT picks the variant with the shorter critical path (Sec. 4.3.3): BiDiag for
    square matrices, R-BiDiag for tall ones, switching between p = 566 and 568 for q = 100."""
    for (p, q) in ((1, 1), (5, 5), (9, 4), (13, 3), (17, 2), (40, 40)):
        for tree in (T.FLATTS, T.FLATTT, T.GREEDY):
            v, cb, cr = G.bidiag_plan_choose_variant(p, q, tree, 1)
            assert cb == T.critical_path(p, q, tree, T.BIDIAG)
            assert cr == T.critical_path(p, q, tree, T.RBIDIAG)
            assert v == (T.RBIDIAG if cr < cb else T.BIDIAG)
    assert G.bidiag_plan_choose_variant(32, 32, T.AUTO, 19)[0] == T.BIDIAG
    assert G.bidiag_plan_choose_variant(256, 4, T.AUTO, 19)[0] == T.RBIDIAG
    assert G.bidiag_plan_choose_variant(560, 100, T.GREEDY, 1)[0] == T.BIDIAG
    assert G.bidiag_plan_choose_variant(575, 100, T.GREEDY, 1)[0] == T.RBIDIAG


def test_autotune_choices():
    """The batched form's autotuner searches the calibrated (nb, ib) pairs and the FlatTS / Greedy / Auto
    trees: its choice is one of those candidates, the variant is the one with the shorter critical path
    for that tree (Sec. 4.3.3), no tile is larger than needed to cover the matrix's width, and each
    storage precision has its own calibration."""
    cands = {(nb, ib) for nb in (32, 64, 128) for ib in (8, 16, 32) if ib <= nb}
    for es in (8, 4):
        for (m, n) in ((32, 1), (64, 32), (100, 100), (1024, 1024), (1024, 200), (4096, 1024), (70000, 64)):
            nb, ib, tree, variant = G.bidiag_autotune(m, n, 152, es)
            assert (nb, ib) in cands and tree in (T.FLATTS, T.GREEDY, T.AUTO)
            assert nb < 2 * max(32, n)          # never more than one size above the matrix's width
            w = min(nb, max(ib, 32 // ib * ib))
            R = max(1, 152 * w * (2 if es == 4 else 1) // nb)
            assert variant == G.bidiag_plan_choose_variant(-(-m // nb), -(-n // nb), tree, R)[0]
    with pytest.raises(G.BidiagError):
        G.bidiag_autotune(100, 100, 152, 2)


def test_three_step_planner_matches_oracle():
    """Three-step with every split s (Sec. 4.5): elimination list, task list, levels and critical path
    bit-exact against the oracle; the best split agrees."""
    for tree in (T.FLATTS, T.FLATTT, T.GREEDY, T.AUTO):
        for p in range(1, 9):
            for q in range(1, p + 1):
                for s in range(q):
                    v = T.THREESTEP + s
                    tasks = T.task_list(p, q, tree, v, 3)
                    tk, lv, cp = G.bidiag_plan_tasks(p, q, tree, v, 3)
                    assert np.array_equal(np.array(tasks, dtype=np.int32).reshape(-1, 6), tk), (tree, p, q, s)
                    lv_o, _, cp_o = T.dag(tasks, v)
                    assert np.array_equal(np.array(lv_o, dtype=np.int32), lv) and cp == cp_o
                    el_o = np.array(T.eliminations(p, q, tree, v, 3), dtype=np.int32).reshape(-1, 5)
                    assert np.array_equal(el_o, G.bidiag_plan_eliminations(p, q, tree, v, 3))
                assert G.bidiag_plan_best_split(p, q, tree, 3) == T.best_split(p, q, tree, 3)


def test_three_step_end_points():
    """Split 0 is R-BiDiag (same task list); split q-1 has BiDiag's critical path; so the best split is
    never worse than either variant (Sec. 4.5)."""
    for tree in (T.FLATTS, T.FLATTT, T.GREEDY, T.AUTO):
        for (p, q) in ((5, 5), (9, 4), (13, 3), (7, 1), (20, 6)):
            assert T.task_list(p, q, tree, T.RBIDIAG, 3) == T.task_list(p, q, tree, T.THREESTEP, 3)
            cb = G.bidiag_plan_tasks(p, q, tree, T.BIDIAG, 3)[2]
            cr = G.bidiag_plan_tasks(p, q, tree, T.RBIDIAG, 3)[2]
            assert G.bidiag_plan_tasks(p, q, tree, T.THREESTEP + q - 1, 3)[2] == cb
            assert G.bidiag_plan_best_split(p, q, tree, 3)[1] <= min(cb, cr)


def test_three_step_figure_q30():
    """Sec. 4.5, q = 30 tile columns, Greedy: the three-step equals BiDiag for square matrices, beats
    both BiDiag and R-BiDiag in the middle region (p = 60 .. 260) and equals R-BiDiag beyond it (the
    planner's critical paths; the planner is checked against the oracle above)."""
    q = 30

    def cps(p):
        cb = G.bidiag_plan_tasks(p, q, T.GREEDY, T.BIDIAG)[2]
        cr = G.bidiag_plan_tasks(p, q, T.GREEDY, T.RBIDIAG)[2]
        return cb, cr, G.bidiag_plan_best_split(p, q, T.GREEDY)

    cb, cr, (s, c3) = cps(30)
    assert c3 == cb < cr
    for p in (60, 100, 150, 200, 260):
        cb, cr, (s, c3) = cps(p)
        assert c3 < min(cb, cr) and 0 < s < q - 1, (p, cb, cr, s, c3)
    cb, cr, (s, c3) = cps(300)
    assert c3 == cr < cb and s == 0
