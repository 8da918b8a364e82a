"""GPU parity: the CUDA path (through the C ABI) against the oracle, element by element.

Tolerances: band entries within 1e-12 * ||A||_F (the target for FP64 B with the same tree); the
in-place Householder vectors (|v| <= ~1) within 1e-11 absolute; the T factors within 1e-10 * max|T|.
The canonical task list must match bit-exact.
"""
import numpy as np
import pytest

import paper_1611_06892_gb300 as G
from oracle import bidiag as OB
from oracle import trees as T
from paper_1611_06892_gb300 import inputs

pytestmark = pytest.mark.gpu

TREES = {"flatts": T.FLATTS, "flattt": T.FLATTT, "greedy": T.GREEDY, "auto": T.AUTO}
R_AUTO = 3


@pytest.fixture(scope="module")
def torch_mod():
    import torch
    return torch


@pytest.fixture(scope="module")
def handle(torch_mod):
    h = G.Handle()
    h.set_option(G.OPT_AUTO_RESOURCES, R_AUTO)
    yield h
    h.close()


def to_dev(torch_mod, A):
    return torch_mod.from_numpy(np.asfortranarray(A)).cuda()


def gpu_reduce(handle, torch_mod, A, nb, ib, tree, variant):
    res = handle.band(to_dev(torch_mod, A), nb, ib, tree, variant)
    handle.sync()
    return res


def tiles_to_dense(tiles, m, n):
    t = tiles.cpu().numpy()
    p, q, nb, _ = t.shape
    D = t.transpose(0, 2, 1, 3).reshape(p * nb, q * nb)
    return D[:m, :n]


def compare(res_g, res_o, A, nb, ib):
    m, n = A.shape
    nA = np.linalg.norm(A)
    # task list
    assert np.array_equal(res_g.tasks(), np.array(res_o["tasks"], dtype=np.int32).reshape(-1, 6))
    # band
    ab_g = res_g.band().cpu().numpy()
    err_b = np.abs(ab_g - res_o["ab"]).max()
    assert err_b <= 1e-12 * nA, f"band error {err_b:.3e} vs {1e-12 * nA:.3e}"
    ii, jj = np.indices(ab_g.shape)
    assert np.all(ab_g[(jj - (nb - ii)) < 0] == 0.0)          # rows above B's first row
    # in-place reflectors and R/L
    W_g = tiles_to_dense(res_g.tiles(), m, n)
    err_w = np.abs(W_g - res_o["work"]).max()
    assert err_w <= 1e-11 * max(1.0, nA), f"work error {err_w:.3e}"
    if res_o["work2"] is not None:
        W2 = tiles_to_dense(res_g.tiles(second=True), n, n)
        assert np.abs(W2 - res_o["work2"]).max() <= 1e-11 * max(1.0, nA)
    # T factors
    Tg = res_g.T().cpu().numpy()
    slots = res_g.tslot()
    for idx, rec in res_o["refl"].items():
        s = slots[idx]
        assert s >= 0
        K = len(rec["tau"])
        for b0 in range(0, K, ib):
            kb = min(ib, K - b0)
            got = Tg[s][:kb, b0:b0 + kb]
            ref = rec["T"][:kb, b0:b0 + kb]
            assert np.abs(got - ref).max() <= 1e-10 * max(1.0, np.abs(ref).max()), (idx, b0)


CASES = [
    # m, n, nb, ib
    (8, 8, 4, 2),
    (96, 96, 16, 4),
    (200, 136, 32, 8),      # ragged rows and columns, 7 x 5 tiles
    (300, 90, 32, 16),      # tall
    (64, 64, 64, 16),       # one tile
    (130, 1, 32, 8),        # one column
    (5, 3, 1, 1),           # nb = 1
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c)))
@pytest.mark.parametrize("tree", list(TREES), ids=list(TREES))
@pytest.mark.parametrize("variant", ("bidiag", "rbidiag"))
def test_parity_small(handle, torch_mod, case, tree, variant):
    m, n, nb, ib = case
    A = inputs.gaussian(m, n, seed=m * 7 + n)
    v = G.VARIANTS[variant]
    res_o = OB.bidiag_band(A, nb, ib, TREES[tree], v, resources=R_AUTO)
    res_g = gpu_reduce(handle, torch_mod, A, nb, ib, tree, variant)
    compare(res_g, res_o, A, nb, ib)
    res_g.free()


def test_parity_cfg1(handle, torch_mod):
    """512 x 512 N(0,1), nb = 64, ib = 16, BiDiag with FlatTS (the small bench configuration)."""
    A = inputs.gaussian(512, 512, seed=1)
    res_o = OB.bidiag_band(A, 64, 16, T.FLATTS, T.BIDIAG)
    res_g = gpu_reduce(handle, torch_mod, A, 64, 16, "flatts", "bidiag")
    compare(res_g, res_o, A, 64, 16)


@pytest.mark.parametrize("tree", ("greedy", "auto"))
def test_parity_nb256_ragged(handle, torch_mod, tree):
    """The bench's tile size (nb = 256, ib = 32) over 3 x 3 tiles with ragged edges."""
    A = inputs.gaussian(600, 520, seed=17)
    for variant in ("bidiag", "rbidiag"):
        res_o = OB.bidiag_band(A, 256, 32, TREES[tree], G.VARIANTS[variant], resources=R_AUTO)
        res_g = gpu_reduce(handle, torch_mod, A, 256, 32, tree, variant)
        compare(res_g, res_o, A, 256, 32)


@pytest.mark.parametrize("m,n,variant", ((1536, 1536, "bidiag"), (1792, 1280, "rbidiag")))
def test_parity_nb256_auto_groups(handle, torch_mod, m, n, variant):
    """nb = 256, ib = 32 on 6 x 6 (BiDiag) and 7 x 5 (R-BiDiag) tiles with R = 3, where Auto's first
    steps have 1 < a < u: FlatTS groups joined by a Greedy TT tree (Sec. 5), compared element-wise at
    the bench's tile size."""
    p, q = -(-m // 256), -(-n // 256)
    a0 = T.auto_group_size(p, q - 1, R_AUTO)
    assert 1 < a0 < p          # the first QR step mixes TS groups and TT joins
    A = inputs.gaussian(m, n, seed=m + n)
    res_o = OB.bidiag_band(A, 256, 32, T.AUTO, G.VARIANTS[variant], resources=R_AUTO)
    res_g = gpu_reduce(handle, torch_mod, A, 256, 32, "auto", variant)
    compare(res_g, res_o, A, 256, 32)
    res_g.free()


@pytest.mark.parametrize("variant", ("bidiag", "rbidiag"))
def test_apply_q_p(handle, torch_mod, variant):
    A = inputs.gaussian(150, 100, seed=23)
    res_o = OB.bidiag_band(A, 32, 8, T.GREEDY, G.VARIANTS[variant])
    res_g = gpu_reduce(handle, torch_mod, A, 32, 8, "greedy", variant)
    C = inputs.gaussian(150, 37, seed=3)
    D = inputs.gaussian(45, 100, seed=4)
    for trans in (0, 1):
        got = res_g.apply_q(to_dev(torch_mod, C), trans)
        handle.sync()
        assert np.abs(got.cpu().numpy() - OB.apply_q(res_o, C, trans)).max() <= 1e-11 * np.abs(C).max()
        got = res_g.apply_p(to_dev(torch_mod, D), trans)
        handle.sync()
        assert np.abs(got.cpu().numpy() - OB.apply_p(res_o, D, trans)).max() <= 1e-11 * np.abs(D).max()


def test_determinism(handle, torch_mod):
    A = inputs.gaussian(333, 333, seed=31)
    r1 = gpu_reduce(handle, torch_mod, A, 32, 8, "auto", "bidiag").band()
    r2 = gpu_reduce(handle, torch_mod, A, 32, 8, "auto", "bidiag").band()
    assert torch_mod.equal(r1, r2)


@pytest.mark.parametrize("m,n,nb,ib,tree,variant,dtype", [
    (1536, 1536, 256, 32, "auto", "bidiag", "f64"),
    (1536, 1536, 256, 32, "flatts", "bidiag", "f64"),
    (1792, 1280, 256, 32, "greedy", "rbidiag", "f64"),
    (700, 500, 32, 8, "auto", "bidiag", "f64"),
    (1536, 1536, 256, 32, "auto", "bidiag", "f32"),
])
def test_window_does_not_change_results(torch_mod, m, n, nb, ib, tree, variant, dtype):
    """The executor's look-ahead (out-of-order claims of ready sub-tasks) and the priority weights of
    the queue order change only timing: the band is bitwise the same with strict queue order, several
    windows and both weightings."""
    A = inputs.gaussian(m, n, seed=57)
    dA = to_dev(torch_mod, A)
    if dtype == "f32":
        dA = dA.float().t().contiguous().t()
    bands = {}
    settings = [(0, 1), (16, 1), (32, 1), (512, 1), (1024, 1), (0, 0), (512, 0)]
    for window, prio in settings:
        h = G.Handle()
        h.set_option(G.OPT_AUTO_RESOURCES, R_AUTO)
        h.set_option(G.OPT_WINDOW, window)
        h.set_option(G.OPT_PRIORITY, prio)
        res = h.band(dA, nb, ib, tree, variant)
        h.sync()
        bands[(window, prio)] = res.band().cpu()
        res.free()
        h.close()
    for key in settings[1:]:
        assert torch_mod.equal(bands[key], bands[(0, 1)]), key
    bands[0] = bands[(0, 1)]
    if dtype == "f64":
        ref = OB.bidiag_band(A, nb, ib, TREES[tree], T.BIDIAG if variant == "bidiag" else T.RBIDIAG,
                             resources=R_AUTO) if m * n <= 1 << 20 else None
        if ref is not None:
            assert np.abs(bands[0].numpy() - ref["ab"]).max() <= 1e-12 * np.linalg.norm(A)


def test_host_entry_point(handle, torch_mod):
    """bidiag_band_host (host buffers, copies inside) gives the same band as the device entry point."""
    A = inputs.gaussian(160, 96, seed=41)
    m, n, nb, ib = 160, 96, 32, 8
    ref = gpu_reduce(handle, torch_mod, A, nb, ib, "greedy", "bidiag").band().cpu().numpy()
    hA = np.asfortranarray(A)
    ab = np.zeros((n, nb + 1)).T            # (nb+1) x n column-major
    assert ab.flags["F_CONTIGUOUS"]
    G.bidiag_band_host(handle.h, m, n, hA.ctypes.data, m, nb, ib, G.GREEDY, G.BIDIAG, ab.ctypes.data, nb + 1)
    assert np.array_equal(ab, ref)


def test_argument_errors(handle, torch_mod):
    lib = G.load_library()
    import ctypes
    A = to_dev(torch_mod, inputs.gaussian(10, 8, seed=1))
    r = ctypes.c_void_p()
    p = ctypes.c_void_p(A.data_ptr())
    assert lib.bidiag_band(handle.h, 0, 8, p, 10, 4, 2, 0, 0, ctypes.byref(r)) == -2
    assert lib.bidiag_band(handle.h, 10, 8, p, 9, 4, 2, 0, 0, ctypes.byref(r)) == -5
    assert lib.bidiag_band(handle.h, 10, 8, p, 10, 300, 2, 0, 0, ctypes.byref(r)) == -6
    assert lib.bidiag_band(handle.h, 10, 8, p, 10, 4, 3, 0, 0, ctypes.byref(r)) == -7
    assert lib.bidiag_band(handle.h, 10, 8, p, 10, 4, 2, 9, 0, ctypes.byref(r)) == -8
    assert lib.bidiag_band(handle.h, 10, 8, p, 10, 4, 2, 0, -1, ctypes.byref(r)) == -9
    assert lib.bidiag_band(handle.h, 10, 8, p, 10, 4, 2, 0, 6, ctypes.byref(r)) == -9    # split 2 >= q
    assert lib.bidiag_band(handle.h, 8, 10, p, 10, 4, 2, 0, 0, ctypes.byref(r)) == G.ERR_UNSUPPORTED
    # shared memory limit: nb = 256 with ib = 64 does not fit
    big = to_dev(torch_mod, inputs.gaussian(256, 256, seed=2))
    assert lib.bidiag_band(handle.h, 256, 256, ctypes.c_void_p(big.data_ptr()), 256, 256, 64, 0, 0,
                           ctypes.byref(r)) == G.ERR_UNSUPPORTED


@pytest.mark.parametrize("window", [0, -1, 64])
def test_wait_timeout_is_reported(handle, torch_mod, window):
    """Failure path without a GPU fault: a dependency on a flag nothing sets makes the bounded wait
    run out; bidiag_sync reports BIDIAG_ERR_TIMEOUT and the handle keeps working (strict queue order
    and look-ahead scheduling)."""
    h = G.Handle()
    h.set_option(G.OPT_WINDOW, window)
    h.set_option(G.OPT_WAIT_LIMIT_NS, 50_000_000)
    h.set_option(G.OPT_DEBUG_UNSET_DEP, 1)
    A = to_dev(torch_mod, inputs.gaussian(64, 48, seed=5))
    res = h.band(A, 16, 4, "greedy", "bidiag")
    with pytest.raises(G.BidiagError) as ei:
        h.sync()
    assert ei.value.code == G.ERR_TIMEOUT
    res.free()
    res = h.band(A, 16, 4, "greedy", "bidiag")
    h.sync()
    A_h = inputs.gaussian(64, 48, seed=5)
    ref = OB.bidiag_band(A_h, 16, 4, T.GREEDY, T.BIDIAG)
    assert np.abs(res.band().cpu().numpy() - ref["ab"]).max() <= 1e-12 * np.linalg.norm(A_h)
    h.close()


def test_auto_variant(handle, torch_mod):
    """variant = auto runs R-BiDiag on a tall matrix and BiDiag on a square one (critical-path switch)."""
    for (m, n, expect) in ((640, 64, T.RBIDIAG), (96, 96, T.BIDIAG)):
        A = inputs.gaussian(m, n, seed=m + n)
        res_g = gpu_reduce(handle, torch_mod, A, 16, 4, "greedy", "auto")
        assert res_g.desc.variant == expect
        res_o = OB.bidiag_band(A, 16, 4, T.GREEDY, expect)
        compare(res_g, res_o, A, 16, 4)


THREE_STEP_CASES = [
    # m, n, nb, ib, split
    (200, 136, 32, 8, 1),     # ragged 7 x 5 tiles
    (200, 136, 32, 8, 3),
    (300, 90, 32, 16, 1),     # tall, 10 x 3
    (96, 96, 16, 4, 2),       # square 6 x 6
    (600, 520, 256, 32, 1),   # the bench's tile size, 3 x 3 ragged
]


@pytest.mark.parametrize("case", THREE_STEP_CASES, ids=lambda c: "x".join(map(str, c)))
@pytest.mark.parametrize("tree", list(TREES), ids=list(TREES))
def test_parity_three_step(handle, torch_mod, case, tree):
    """Three-step (Sec. 4.5) with a fixed split: band, tiles of both buffers, T and task list."""
    m, n, nb, ib, s = case
    A = inputs.gaussian(m, n, seed=m * 3 + n + s)
    v = G.threestep_split(s)
    res_o = OB.bidiag_band(A, nb, ib, TREES[tree], v, resources=R_AUTO)
    res_g = gpu_reduce(handle, torch_mod, A, nb, ib, tree, v)
    compare(res_g, res_o, A, nb, ib)
    res_g.free()


def test_three_step_best_split(handle, torch_mod):
    """BIDIAG_THREESTEP picks the split with the shortest critical path and records it."""
    m, n, nb, ib = 640, 160, 32, 8       # 20 x 5 tiles
    A = inputs.gaussian(m, n, seed=77)
    s, _ = G.bidiag_plan_best_split(20, 5, G.GREEDY, R_AUTO)
    res_g = gpu_reduce(handle, torch_mod, A, nb, ib, "greedy", "threestep")
    want = G.RBIDIAG if s == 0 else G.threestep_split(s)
    assert res_g.desc.variant == want
    res_o = OB.bidiag_band(A, nb, ib, T.GREEDY, T.THREESTEP + s, resources=R_AUTO)
    compare(res_g, res_o, A, nb, ib)
    res_g.free()


EDGE_CASES = [
    # m, n, nb, ib: a 1 x 1 matrix, one row of tiles narrower than the tile, a tile larger than the
    # matrix, one extra row past a tile boundary, two columns
    (1, 1, 4, 2), (3, 1, 8, 4), (7, 7, 8, 8), (33, 32, 32, 32), (9, 2, 4, 4), (17, 16, 4, 1),
]


@pytest.mark.parametrize("case", EDGE_CASES, ids=lambda c: "x".join(map(str, c)))
@pytest.mark.parametrize("tree", list(TREES), ids=list(TREES))
@pytest.mark.parametrize("variant", ("bidiag", "rbidiag"))
def test_parity_edge_sizes(handle, torch_mod, case, tree, variant):
    m, n, nb, ib = case
    A = inputs.gaussian(m, n, seed=m * 11 + n)
    res_o = OB.bidiag_band(A, nb, ib, TREES[tree], G.VARIANTS[variant], resources=R_AUTO)
    res_g = gpu_reduce(handle, torch_mod, A, nb, ib, tree, variant)
    compare(res_g, res_o, A, nb, ib)
    res_g.free()
