"""Split-precision form (FP32 storage, updates as three TF32 tensor-core products, FP64 reflector norms)
against the FP64 oracle, at the stated accuracy: residual, orthogonality, singular-value error and the
band itself within 5e-6 relative (FP32 carries 2^-24 = 6e-8 per rounding).

The input is rounded to FP32 once; the oracle reduces that same rounded matrix in FP64.
"""
import numpy as np
import pytest

import paper_1611_06892_gb300 as G
from oracle import bidiag as OB
from oracle import trees as T
from paper_1611_06892_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL = 5e-6
TREES = {"flatts": T.FLATTS, "flattt": T.FLATTT, "greedy": T.GREEDY, "auto": T.AUTO}


@pytest.fixture(scope="module")
def torch_mod():
    import torch
    return torch


@pytest.fixture(scope="module")
def handle(torch_mod):
    h = G.Handle()
    h.set_option(G.OPT_AUTO_RESOURCES, 3)
    yield h
    h.close()


def dense_band(ab, n):
    nb = ab.shape[0] - 1
    B = np.zeros((n, n))
    for j in range(n):
        for d in range(nb + 1):
            i = j + d - nb
            if i >= 0:
                B[i, j] = ab[d, j]
    return B


def check(torch, handle, A32, nb, ib, tree, variant):
    m, n = A32.shape
    A64 = A32.astype(np.float64)
    res = handle.band(torch.from_numpy(np.asfortranarray(A32)).cuda(), nb, ib, tree, variant)
    handle.sync()
    assert res.esize == 4
    ab = res.band().cpu().numpy().astype(np.float64)
    ref = OB.bidiag_band(A64, nb, ib, TREES[tree], G.VARIANTS[variant], resources=3)
    nA = np.linalg.norm(A64)
    # the band, elementwise against the FP64 oracle with the same tree
    assert np.abs(ab - ref["ab"]).max() <= TOL * nA
    # singular values of B against those of A
    sb = np.linalg.svd(dense_band(ab, n), compute_uv=False)
    sa = np.linalg.svd(A64, compute_uv=False)
    assert np.abs(sb - sa).max() <= TOL * sa[0]
    # residual A P X = Q B X and orthogonality, through the FP32 apply entry points
    rng = np.random.default_rng(3)
    X = rng.standard_normal((n, 3)).astype(np.float32)
    Z = torch.from_numpy(np.asfortranarray(X.T)).cuda()
    res.apply_p(Z, 1)
    handle.sync()
    PX = Z.cpu().numpy().T.astype(np.float64)
    Y = np.zeros((m, 3), dtype=np.float32)
    Y[:n] = (dense_band(ab, n) @ X.astype(np.float64)).astype(np.float32)
    Yd = torch.from_numpy(np.asfortranarray(Y)).cuda()
    res.apply_q(Yd, 0)
    handle.sync()
    QBX = Yd.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(A64 @ PX - QBX) <= TOL * nA * np.linalg.norm(X)
    W = Yd.clone()
    res.apply_q(W, 1)
    handle.sync()
    # Q^T (Q Y) = Y: two FP32 applications, each within the target
    assert np.linalg.norm(W.cpu().numpy() - Y) <= 2 * TOL * np.linalg.norm(Y)
    # tau (diagonal of T) from the FP64 norms
    Tg = res.T().cpu().numpy()
    slots = res.tslot()
    worst = 0.0
    for idx, rec in ref["refl"].items():
        K = len(rec["tau"])
        got = np.array([Tg[slots[idx]][j % ib, j] for j in range(K)])
        worst = max(worst, np.abs(got - rec["tau"]).max())
    assert worst <= 1e-4
    res.free()


@pytest.mark.parametrize("case", [(200, 136, 32, 16), (320, 96, 32, 32), (96, 96, 16, 4), (130, 33, 32, 16)],
                         ids=lambda c: "x".join(map(str, c)))
@pytest.mark.parametrize("tree", ("flatts", "greedy", "auto"))
@pytest.mark.parametrize("variant", ("bidiag", "rbidiag"))
def test_split_fp32_against_fp64_oracle(handle, torch_mod, case, tree, variant):
    m, n, nb, ib = case
    A32 = inputs.gaussian(m, n, seed=m + 3 * n).astype(np.float32)
    check(torch_mod, handle, A32, nb, ib, tree, variant)


def test_split_fp32_nb256(handle, torch_mod):
    """The bench's tile size over ragged 3 x 2 tiles (tensor-core path: ib = 32)."""
    A32 = inputs.gaussian(600, 400, seed=9).astype(np.float32)
    check(torch_mod, handle, A32, 256, 32, "greedy", "rbidiag")


def test_split_fp32_scalar_modes(torch_mod):
    """The reflector scalars (beta, tau, tail scale) of the FP32 path in float-pair arithmetic (default)
    and in FP64 (BIDIAG_OPT_F32_SCALARS = 1): both meet the FP64-oracle checks, and their bands agree
    to a few FP32 roundings (the two compute the same FP32 values up to rounding ties)."""
    torch = torch_mod
    A32 = inputs.gaussian(600, 400, seed=9).astype(np.float32)
    bands = []
    for mode in (0, 1):
        h = G.Handle()
        h.set_option(G.OPT_AUTO_RESOURCES, 3)
        h.set_option(G.OPT_F32_SCALARS, mode)
        try:
            check(torch, h, A32, 256, 32, "auto", "bidiag")
            res = h.band(torch.from_numpy(np.asfortranarray(A32)).cuda(), 256, 32, "auto", "bidiag")
            h.sync()
            bands.append(res.band().cpu().numpy().astype(np.float64))
            res.free()
        finally:
            h.close()
    nA = np.linalg.norm(A32.astype(np.float64))
    assert np.abs(bands[0] - bands[1]).max() <= 64 * 2.0 ** -24 * nA


def test_split_fp32_update_modes(torch_mod):
    """The FP32-storage updates with the C -= V W product on tcgen05 (default, one matrix, 64-column
    strips), on the warp-level tensor cores only (BIDIAG_OPT_F32_UPDATES = 2) and by FFMA (= 1): each meets
    the FP64-oracle checks; the trace shows that the default really ran updates on tcgen05 and the other
    modes none; the two three-TF32 forms agree to a few FP32 roundings."""
    torch = torch_mod
    A32 = inputs.gaussian(700, 520, seed=21).astype(np.float32)
    nA = np.linalg.norm(A32.astype(np.float64))
    bands = {}
    for mode in (0, 2, 1):
        h = G.Handle()
        h.set_option(G.OPT_AUTO_RESOURCES, 3)
        h.set_option(G.OPT_F32_UPDATES, mode)
        try:
            check(torch, h, A32, 256, 32, "auto", "bidiag")
            h.set_option(G.OPT_TRACE, 1)
            res = h.band(torch.from_numpy(np.asfortranarray(A32)).cuda(), 256, 32, "auto", "bidiag")
            h.sync()
            bands[mode] = res.band().cpu().numpy().astype(np.float64)
            res.free()
            tc5 = int(((h.trace()[:, 3] >> 32) & 1).sum())
            assert (tc5 > 0) == (mode == 0), (mode, tc5)
        finally:
            h.close()
    assert np.abs(bands[0] - bands[2]).max() <= 64 * 2.0 ** -24 * nA


@pytest.mark.parametrize("m,n,tree,variant,seed", [(65536, 1024, "greedy", "rbidiag", 4),
                                                   (65536, 2048, "auto", "rbidiag", 5),
                                                   (8192, 8192, "auto", "bidiag", 2)],
                         ids=("tall1024", "tall2048", "square8192"))
def test_split_fp32_full_size(torch_mod, m, n, tree, variant, seed):
    """The split form at the bench's sizes, each result's accuracy against FP64 stated and checked at
    5e-6: singular values of B against those of the (FP32-rounded) A relative to sigma_1, the residual
    ||A P X - Q B X|| / (||A|| ||X||) and the orthogonality round trip ||Q^T Q Y - Y|| / ||Y|| through
    the FP32 apply entry points (two applications, each within 5e-6).  Inputs: N(0,1) for the tall shapes, U diag(s) V^T with s geometric
    from 1 to 1e-8 for the square one."""
    torch = torch_mod
    nb, ib = 256, 32
    if m == n:
        A = inputs.torch_prescribed_singular_values(m, n, inputs.geometric_sv(n), seed, seed + 1)
    else:
        A = inputs.torch_gaussian(m, n, seed)
    A32 = A.float().t().contiguous().t()
    del A
    h = G.Handle()
    try:
        res = h.band(A32, nb, ib, tree, variant)
        h.sync()
        ab = res.band().double()
        B = torch.zeros((n, n), dtype=torch.float64, device="cuda")
        j = torch.arange(n, device="cuda")
        for d in range(nb + 1):
            i = j + d - nb
            ok = i >= 0
            B[i[ok], j[ok]] = ab[d, ok]
        A64 = A32.double()
        sa = torch.linalg.svdvals(A64)
        sb = torch.linalg.svdvals(B)
        err_sv = (sa - sb).abs().max().item() / sa[0].item()
        gen = torch.Generator(device="cuda")
        gen.manual_seed(5)
        X = torch.randn((n, 4), dtype=torch.float32, device="cuda", generator=gen)
        Z = torch.empty((n, 4), dtype=torch.float32, device="cuda").t()
        Z.copy_(X.t())
        res.apply_p(Z, 1)
        h.sync()
        Y = torch.zeros((4, m), dtype=torch.float32, device="cuda").t()
        Y[:n] = (B @ X.double()).float()
        Y0 = Y.clone()
        res.apply_q(Y, 0)
        h.sync()
        err_res = torch.linalg.norm(A64 @ Z.t().double() - Y.double()).item() / (
            torch.linalg.norm(A64).item() * torch.linalg.norm(X.double()).item())
        res.apply_q(Y, 1)
        h.sync()
        err_orth = torch.linalg.norm((Y - Y0).double()).item() / torch.linalg.norm(Y0.double()).item()
        print(f"\nsplit-FP32 accuracy {m}x{n} {tree} {variant}: sigma {err_sv:.2e}, residual {err_res:.2e}, "
              f"orthogonality {err_orth:.2e}")
        # the round trip is two FP32 applications, each held to the target
        assert err_sv <= TOL and err_res <= TOL and err_orth <= 2 * TOL
        res.free()
    finally:
        h.close()
