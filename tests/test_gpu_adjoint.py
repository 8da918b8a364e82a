"""GPU adjoint (bidiag_band_backward, through the C ABI) against the oracle adjoint, element by element,
plus the checks that hold at any size: finite differences of the GPU forward, the closed form
d(sum sigma)/dA = U V^T, and the reconstruction of A by the reverse sweep.

Tolerance (FP64): both sides evaluate the same chain rule on reflectors that agree to ~1e-15; the
adjoint multiplies by 1/beta and 1/(beta tau) per step, so dL/dA is compared at 1e-10 of its largest
entry (1e-11 measured margin on these inputs is not assumed).
"""
import numpy as np
import pytest

import paper_1611_06892_gb300 as G
from oracle import adjoint as AD
from oracle import bidiag as OB
from oracle import trees as T
from paper_1611_06892_gb300 import inputs

pytestmark = pytest.mark.gpu

TREES = {"flatts": T.FLATTS, "flattt": T.FLATTT, "greedy": T.GREEDY, "auto": T.AUTO}
R_AUTO = 3
TOL = 1e-10


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


def dev(torch, X):
    return torch.from_numpy(np.asfortranarray(X)).cuda()


CASES = [
    # m, n, nb, ib
    (8, 8, 4, 2),
    (96, 96, 16, 4),
    (200, 136, 32, 8),      # ragged rows and columns, 7 x 5 tiles
    (300, 90, 32, 16),      # tall
    (64, 64, 64, 16),       # one tile
    (130, 1, 32, 8),        # one column
    (64, 32, 16, 4),        # the finite-difference size
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c)))
@pytest.mark.parametrize("tree", list(TREES), ids=list(TREES))
@pytest.mark.parametrize("variant", ("bidiag", "rbidiag"))
def test_adjoint_parity(handle, torch_mod, case, tree, variant):
    torch = torch_mod
    m, n, nb, ib = case
    A = inputs.gaussian(m, n, seed=m * 5 + n)
    W = inputs.gaussian(nb + 1, n, seed=m + 3 * n)
    res_o = OB.bidiag_band(A, nb, ib, TREES[tree], G.VARIANTS[variant], resources=R_AUTO)
    Ab_o, _ = AD.band_vjp(res_o, W)
    res_g = handle.band(dev(torch, A), nb, ib, tree, variant)
    Ab_g, Arec = res_g.backward(dev(torch, W), reconstruct=True)
    handle.sync()
    Ab_g = Ab_g.cpu().numpy()
    scale = max(1.0, np.abs(Ab_o).max())
    assert np.abs(Ab_g - Ab_o).max() <= TOL * scale
    assert np.abs(Arec.cpu().numpy() - A).max() <= 1e-12 * max(1.0, np.linalg.norm(A))
    res_g.free()


@pytest.mark.parametrize("tree", ("greedy", "auto"))
@pytest.mark.parametrize("variant", ("bidiag", "rbidiag"))
def test_adjoint_parity_nb256(handle, torch_mod, tree, variant):
    """The bench's tile size (nb = 256, ib = 32) over 3 x 3 ragged tiles."""
    torch = torch_mod
    A = inputs.gaussian(600, 520, seed=17)
    W = inputs.gaussian(257, 520, seed=18)
    res_o = OB.bidiag_band(A, 256, 32, TREES[tree], G.VARIANTS[variant], resources=R_AUTO)
    Ab_o, _ = AD.band_vjp(res_o, W)
    res_g = handle.band(dev(torch, A), 256, 32, tree, variant)
    Ab_g = res_g.backward(dev(torch, W))
    handle.sync()
    assert np.abs(Ab_g.cpu().numpy() - Ab_o).max() <= TOL * max(1.0, np.abs(Ab_o).max())
    res_g.free()


def test_adjoint_finite_differences_64x32(handle, torch_mod):
    """L = <W, B> + sum sigma(B) on 64 x 32 (nb = 16): <dL/dA, E> from the GPU adjoint against central
    differences of the GPU forward."""
    torch = torch_mod
    m, n, nb, ib = 64, 32, 16, 4
    A = inputs.gaussian(m, n, seed=7)
    W = inputs.gaussian(nb + 1, n, seed=8)

    def loss(X):
        r = handle.band(dev(torch, X), nb, ib, "greedy", "bidiag")
        handle.sync()
        ab = r.band().cpu().numpy()
        r.free()
        B = OB.band_to_dense(ab, n)
        return float((W * ab).sum()) + float(np.linalg.svd(B, compute_uv=False).sum()), B

    _, B = loss(A)
    U, _, Vt = np.linalg.svd(B)
    ab_bar = W + OB.band_of(U @ Vt, nb)
    res = handle.band(dev(torch, A), nb, ib, "greedy", "bidiag")
    Ab = res.backward(dev(torch, ab_bar)).cpu().numpy()
    res.free()
    rng = np.random.default_rng(9)
    h = 1e-6
    for _ in range(6):
        E = rng.standard_normal((m, n))
        fd = (loss(A + h * E)[0] - loss(A - h * E)[0]) / (2 * h)
        an = float((Ab * E).sum())
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an))


@pytest.mark.parametrize("variant", ("bidiag", "rbidiag"))
def test_sum_of_singular_values_4096x1024(torch_mod, variant):
    """The differentiation workload's size: d(sum sigma(B))/dA = U V^T of A's thin SVD."""
    torch = torch_mod
    m, n, nb, ib = 4096, 1024, 256, 32
    A = inputs.torch_gaussian(m, n, 7)
    h = G.Handle()
    try:
        res = h.band(A, nb, ib, "greedy", variant)
        h.sync()
        ab = res.band()
        from paper_1611_06892_gb300.autograd import dense_from_band
        B = dense_from_band(ab)
        U, _, Vh = torch.linalg.svd(B)
        Bbar = U @ Vh
        ab_bar = torch.zeros_like(ab)
        j = torch.arange(n, device=ab.device)
        for d in range(nb + 1):
            i = j + d - nb
            ok = i >= 0
            ab_bar[d, ok] = Bbar[i[ok], j[ok]]
        Ab, Arec = res.backward(ab_bar, reconstruct=True)
        h.sync()
        Ua, _, Vha = torch.linalg.svd(A, full_matrices=False)
        assert (Ab - Ua @ Vha).abs().max().item() <= 1e-9
        assert (Arec - A).abs().max().item() <= 1e-12 * torch.linalg.norm(A).item()
        res.free()
    finally:
        h.close()


def test_autograd_checkpointed_and_recomputed(torch_mod):
    """torch.autograd through band_bidiag: the kept and the recomputed reflector store give the same
    gradient, equal to the oracle adjoint."""
    torch = torch_mod
    from paper_1611_06892_gb300.autograd import band_bidiag
    m, n, nb, ib = 150, 100, 32, 8
    A_np = inputs.gaussian(m, n, seed=51)
    W_np = inputs.gaussian(nb + 1, n, seed=52)
    W = dev(torch, W_np)
    grads = []
    for budget in (None, 0):
        A = dev(torch, A_np).requires_grad_(True)
        ab = band_bidiag(A, nb, ib, "auto", "bidiag", memory_budget=budget)
        (ab * W).sum().backward()
        grads.append(A.grad.cpu().numpy())
    assert np.array_equal(grads[0], grads[1])
    # the Auto tree's R is the library's default, SMs x (strip width 32) / nb
    R = max(1, torch.cuda.get_device_properties(0).multi_processor_count * 32 // nb)
    res_o = OB.bidiag_band(A_np, nb, ib, T.AUTO, T.BIDIAG, resources=R)
    Ab_o, _ = AD.band_vjp(res_o, W_np)
    assert np.abs(grads[0] - Ab_o).max() <= TOL * max(1.0, np.abs(Ab_o).max())


def test_batched_result_backward(handle, torch_mod):
    """A result of the batched form differentiates like the one-matrix result with its configuration."""
    torch = torch_mod
    shapes = [(120, 70), (64, 64), (200, 40)]
    As = [dev(torch, inputs.gaussian(m, n, seed=m + n)) for m, n in shapes]
    res = handle.band_batched(As, nb=[32, 16, 32], ib=[8, 4, 16], tree=["greedy", "flatts", "flattt"],
                              variant=["bidiag", "rbidiag", "rbidiag"])
    handle.sync()
    for (m, n), A, r, nb, ib, tree, var in zip(shapes, As, res, [32, 16, 32], [8, 4, 16],
                                                ["greedy", "flatts", "flattt"], ["bidiag", "rbidiag", "rbidiag"]):
        W = dev(torch, inputs.gaussian(nb + 1, n, seed=3 * n))
        got = r.backward(W)
        one = handle.band(A, nb, ib, tree, var)
        ref = one.backward(W)
        handle.sync()
        assert torch.equal(got, ref)
        one.free()
        r.free()


def test_backward_argument_errors(handle, torch_mod):
    import ctypes
    torch = torch_mod
    lib = G.load_library()
    A = dev(torch, inputs.gaussian(40, 30, seed=1))
    res = handle.band(A, 8, 4, "greedy", "bidiag")
    handle.sync()
    W = torch.zeros((9, 30), dtype=torch.float64, device="cuda").t().contiguous().t()
    out = torch.zeros((30, 40), dtype=torch.float64, device="cuda").t()
    p = ctypes.c_void_p
    assert lib.bidiag_band_backward(handle.h, None, p(W.data_ptr()), 9, p(out.data_ptr()), 40, None, 1) == -2
    assert lib.bidiag_band_backward(handle.h, res.r, None, 9, p(out.data_ptr()), 40, None, 1) == -3
    assert lib.bidiag_band_backward(handle.h, res.r, p(W.data_ptr()), 8, p(out.data_ptr()), 40, None, 1) == -4
    assert lib.bidiag_band_backward(handle.h, res.r, p(W.data_ptr()), 9, None, 40, None, 1) == -5
    assert lib.bidiag_band_backward(handle.h, res.r, p(W.data_ptr()), 9, p(out.data_ptr()), 39, None, 1) == -6
    assert lib.bidiag_band_backward_f32(handle.h, res.r, p(W.data_ptr()), 9, p(out.data_ptr()), 40, None, 1) == -2
    res.free()


SPLIT_TOL = 1e-4


@pytest.mark.parametrize("case", [(200, 136, 32, 16), (320, 96, 32, 32), (600, 400, 256, 32)],
                         ids=lambda c: "x".join(map(str, c)))
@pytest.mark.parametrize("variant", ("bidiag", "rbidiag"))
def test_adjoint_split_fp32(handle, torch_mod, case, variant):
    """FP32 storage (3xTF32 updates, FP64 reflector scalars): dL/dA against the FP64 oracle adjoint of
    the same FP32-rounded matrix, within SPLIT_TOL of the largest entry."""
    torch = torch_mod
    m, n, nb, ib = case
    A32 = inputs.gaussian(m, n, seed=m + n).astype(np.float32)
    W32 = inputs.gaussian(nb + 1, n, seed=2 * n).astype(np.float32)
    res_o = OB.bidiag_band(A32.astype(np.float64), nb, ib, T.GREEDY, G.VARIANTS[variant], resources=R_AUTO)
    Ab_o, _ = AD.band_vjp(res_o, W32.astype(np.float64))
    res_g = handle.band(dev(torch, A32), nb, ib, "greedy", variant)
    Ab_g, Arec = res_g.backward(dev(torch, W32), reconstruct=True)
    handle.sync()
    err = np.abs(Ab_g.cpu().numpy().astype(np.float64) - Ab_o).max() / np.abs(Ab_o).max()
    assert err <= SPLIT_TOL, err
    rec = np.abs(Arec.cpu().numpy().astype(np.float64) - A32).max() / np.abs(A32).max()
    assert rec <= 1e-5, rec
    res_g.free()


@pytest.mark.parametrize("case", [(200, 136, 32, 8, 1), (300, 90, 32, 16, 2), (600, 520, 256, 32, 1)],
                         ids=lambda c: "x".join(map(str, c)))
@pytest.mark.parametrize("tree", ("flatts", "greedy", "auto"))
def test_adjoint_parity_three_step(handle, torch_mod, case, tree):
    torch = torch_mod
    m, n, nb, ib, s = case
    A = inputs.gaussian(m, n, seed=m + n + s)
    W = inputs.gaussian(nb + 1, n, seed=5 * n)
    v = G.threestep_split(s)
    res_o = OB.bidiag_band(A, nb, ib, TREES[tree], v, resources=R_AUTO)
    Ab_o, _ = AD.band_vjp(res_o, W)
    res_g = handle.band(dev(torch, A), nb, ib, tree, v)
    Ab_g, Arec = res_g.backward(dev(torch, W), reconstruct=True)
    handle.sync()
    assert np.abs(Ab_g.cpu().numpy() - Ab_o).max() <= TOL * max(1.0, np.abs(Ab_o).max())
    assert np.abs(Arec.cpu().numpy() - A).max() <= 1e-12 * max(1.0, np.linalg.norm(A))
    res_g.free()


@pytest.mark.parametrize("case", [(1, 1, 4, 2), (3, 1, 8, 4), (7, 7, 8, 8), (33, 32, 32, 32), (9, 2, 4, 4),
                                  (17, 16, 4, 1)], ids=lambda c: "x".join(map(str, c)))
@pytest.mark.parametrize("tree", ("flatts", "greedy", "auto"))
@pytest.mark.parametrize("variant", ("bidiag", "rbidiag"))
def test_adjoint_edge_sizes(handle, torch_mod, case, tree, variant):
    torch = torch_mod
    m, n, nb, ib = case
    A = inputs.gaussian(m, n, seed=m * 13 + n)
    W = inputs.gaussian(nb + 1, n, seed=m + 7 * n)
    res_o = OB.bidiag_band(A, nb, ib, TREES[tree], G.VARIANTS[variant], resources=R_AUTO)
    Ab_o, _ = AD.band_vjp(res_o, W)
    res_g = handle.band(dev(torch, A), nb, ib, tree, variant)
    Ab_g, Arec = res_g.backward(dev(torch, W), reconstruct=True)
    handle.sync()
    assert np.abs(Ab_g.cpu().numpy() - Ab_o).max() <= TOL * max(1.0, np.abs(Ab_o).max())
    assert np.abs(Arec.cpu().numpy() - A).max() <= 1e-12 * max(1.0, np.linalg.norm(A))
    res_g.free()
