"""Full-size GPU checks at the bench's workloads (8192^2 square BiDiag with each of the four trees,
65536 x 1024 and 65536 x 2048 tall R-BiDiag), in the launch configuration bench.py times.

At these sizes the oracle cannot run the whole reduction, so the checks are properties that hold at
any size (band structure, orthogonal invariance of the Frobenius norm, singular values of B equal to
those of A within 30 max(m, n) eps ||A||_2 (Weyl; Sec. 6.1 states singular values accurate to machine
precision), A P X = Q B X through the library's own apply_q / apply_p, orthogonality of Q) plus one
sampled output the oracle computes exactly: the first diagonal block of B, which only depends on the
panel tasks of the first tile column (Sec. 3.4: QR(1) factors that column before anything else).
An 8192^2 SVD takes about 85 s on the GPU, so at 8192^2 the singular values are compared for the
bench's tree (Auto); every tree is compared on sigma at 4096^2 with the same geometric spectrum.
"""
import numpy as np
import pytest

import paper_1611_06892_gb300 as G
from oracle import bidiag as OB
from oracle import trees as T
from paper_1611_06892_gb300 import inputs

pytestmark = pytest.mark.gpu
EPS = 2.0 ** -53


@pytest.fixture(scope="module")
def torch_mod():
    import torch
    return torch


def dense_band(torch, ab, n, nb):
    """Dense n x n B from the (nb+1) x n band on the device."""
    B = torch.zeros((n, n), dtype=torch.float64, device=ab.device)
    j = torch.arange(n, device=ab.device)
    for d in range(nb + 1):
        i = j + d - nb
        ok = i >= 0
        B[i[ok], j[ok]] = ab[d, ok]
    return B


def run(torch, A, nb, ib, tree, variant, resources):
    h = G.Handle()
    h.set_option(G.OPT_AUTO_RESOURCES, resources)
    res = h.band(A, nb, ib, tree, variant)
    h.sync()
    return h, res


def check_properties(torch, h, res, A, nb, s_ref, tol_sv, check_sv=True):
    m, n = A.shape
    ab = res.band()
    # rows above B's first row are exact zeros
    d = torch.arange(nb + 1, device=ab.device)[:, None]
    j = torch.arange(n, device=ab.device)[None, :]
    assert torch.all(ab[(j + d - nb) < 0] == 0)
    B = dense_band(torch, ab, n, nb)
    nA = torch.linalg.norm(A).item()
    assert abs(torch.linalg.norm(B).item() - nA) <= 1e-12 * nA * max(m, n) ** 0.5
    # singular values of B against those of A, on sigma itself (absolute, relative to ||A||_2)
    if check_sv:
        sb = torch.linalg.svdvals(B)
        err_sv = (sb - s_ref).abs().max().item()
        assert err_sv <= tol_sv, f"singular values: {err_sv:.3e} > {tol_sv:.3e}"
    # A (P X) = Q [B X; 0]
    gen = torch.Generator(device="cuda")
    gen.manual_seed(11)
    X = torch.randn((n, 4), dtype=torch.float64, device="cuda", generator=gen)
    PXt = torch.empty((n, 4), dtype=torch.float64, device="cuda").t()   # 4 x n, column-major
    PXt.copy_(X.t())
    res.apply_p(PXt, 1)                                  # X^T P^T = (P X)^T
    h.sync()
    y1 = A @ PXt.t()
    Y = torch.zeros((4, m), dtype=torch.float64, device="cuda").t()       # m x 4, column-major
    Y[:n] = B @ X
    res.apply_q(Y, 0)
    h.sync()
    err = torch.linalg.norm(y1 - Y).item() / (nA * torch.linalg.norm(X).item())
    assert err <= 30 * max(m, n) * EPS, err
    # Q^T Q X = X
    Z = Y.clone()
    res.apply_q(Z, 1)
    h.sync()
    Z2 = Z.clone()
    res.apply_q(Z2, 0)
    h.sync()
    assert torch.linalg.norm(Z2 - Y).item() <= 30 * m * EPS * torch.linalg.norm(Y).item()


@pytest.mark.parametrize("tree", ("auto", "flatts", "flattt", "greedy"))
def test_square_8192(torch_mod, tree):
    torch = torch_mod
    m = n = 8192
    nb, ib = 256, 32
    s = inputs.geometric_sv(n)
    A = inputs.torch_prescribed_singular_values(m, n, s, 2, 3)
    R = max(1, torch.cuda.get_device_properties(0).multi_processor_count * 32 // nb)
    h, res = run(torch, A, nb, ib, tree, "bidiag", R)
    s_ref = torch.as_tensor(np.sort(s)[::-1].copy(), device="cuda")
    check_properties(torch, h, res, A, nb, s_ref, 30 * n * EPS * float(s_ref[0]), check_sv=(tree == "auto"))
    # sampled output: the first diagonal block of B from the oracle's column-0 panel tasks
    tasks = T.task_list(m // nb, n // nb, G.TREES[tree], T.BIDIAG, R)
    col0 = [(x, t) for x, t in enumerate(tasks)
            if t[1] == T.QR and t[2] == 0 and t[0] in (T.GEQRT, T.TSQRT, T.TTQRT)]
    A0 = A[:, :nb].cpu().numpy()
    st = OB.new_state(np.zeros((m, nb)), nb, ib, G.TREES[tree], T.BIDIAG, resources=R)
    st["A"].M[...] = A0
    OB.run_tasks(st, col0)
    R00 = np.triu(st["A"].M[:nb, :nb])
    B00 = np.triu(dense_band(torch, res.band(), n, nb)[:nb, :nb].cpu().numpy())
    assert np.abs(B00 - R00).max() <= 1e-12 * torch.linalg.norm(A).item()
    res.free()
    h.close()


@pytest.mark.parametrize("tree", ("auto", "flatts", "flattt", "greedy"))
def test_square_4096_singular_values(torch_mod, tree):
    """Every tree at 4096^2 with the 8192^2 workload's spectrum (s geometric from 1 to 1e-8): the
    singular values of B within 30 n eps ||A||_2 of the prescribed s, and the other properties."""
    torch = torch_mod
    m = n = 4096
    nb, ib = 256, 32
    s = inputs.geometric_sv(n)
    A = inputs.torch_prescribed_singular_values(m, n, s, 2, 3)
    R = max(1, torch.cuda.get_device_properties(0).multi_processor_count * 32 // nb)
    h, res = run(torch, A, nb, ib, tree, "bidiag", R)
    s_ref = torch.as_tensor(np.sort(s)[::-1].copy(), device="cuda")
    check_properties(torch, h, res, A, nb, s_ref, 30 * n * EPS * float(s_ref[0]))
    res.free()
    h.close()


@pytest.mark.parametrize("n,seed", ((1024, 4), (2048, 5)))
@pytest.mark.parametrize("tree", ("greedy", "auto"))
def test_tall_65536_rbidiag(torch_mod, tree, n, seed):
    torch = torch_mod
    m, nb, ib = 65536, 256, 32
    A = inputs.torch_gaussian(m, n, seed)
    R = max(1, torch.cuda.get_device_properties(0).multi_processor_count * 32 // nb)
    h, res = run(torch, A, nb, ib, tree, "rbidiag", R)
    s_ref = torch.linalg.svdvals(A)
    check_properties(torch, h, res, A, nb, s_ref, 30 * m * EPS * s_ref[0].item())
    res.free()
    h.close()


def test_adjoint_8192_bounded_memory(torch_mod):
    """The adjoint at the headline size (8192^2 N(0,1), Auto, nb = 256, FP64): its device workspace
    stays within 10 GB (partial-sum storage recycled in queue order), the directional derivative
    <dL/dA, E> of L = <W, B> matches central differences of the forward, and the reverse sweep
    reconstructs A.

    The band is a piecewise smooth function of A: a Householder reflector switches branch where its
    pivot entry alpha crosses zero (the sign of beta follows alpha), and with ~16K reflectors a
    perturbation of 1e-5 per entry already crosses such a switch.  The difference step is therefore
    1e-7 (relative to ||A||), and a direction is used only if both one-sided differences agree (no
    switch crossed); otherwise the next seeded direction is tried."""
    torch = torch_mod
    m = n = 8192
    nb, ib = 256, 32
    A = inputs.torch_gaussian(m, n, 12)
    R = max(1, torch.cuda.get_device_properties(0).multi_processor_count * 32 // nb)
    h, res = run(torch, A, nb, ib, "auto", "bidiag", R)
    ws = res.backward_workspace()
    assert ws <= 10 * 2 ** 30, f"adjoint workspace {ws / 2**30:.1f} GiB"
    gen = torch.Generator(device="cuda")
    gen.manual_seed(13)
    W = torch.randn((n, nb + 1), dtype=torch.float64, device="cuda", generator=gen).t()
    Abar, Arec = res.backward(W, reconstruct=True)
    h.sync()
    nA = torch.linalg.norm(A).item()
    assert torch.linalg.norm(Arec - A).item() <= 30 * n * EPS * nA

    def loss(X):
        r = h.band(X.t().contiguous().t(), nb, ib, "auto", "bidiag")
        h.sync()
        v = (r.band() * W).sum().item()
        r.free()
        return v

    L0 = loss(A)
    checked = 0
    for seed in (14, 15, 16):
        gen.manual_seed(seed)
        E = torch.randn((n, m), dtype=torch.float64, device="cuda", generator=gen).t()
        dL = (Abar * E).sum().item()
        step = 1e-7 * nA / torch.linalg.norm(E).item()
        up, down = loss(A + step * E) - L0, L0 - loss(A - step * E)
        if abs(up - down) > 1e-3 * max(abs(up), abs(down)):
            continue                     # a branch switch lies within the step: try another direction
        fd = (up + down) / (2 * step)
        assert abs(fd - dL) <= 1e-5 * abs(dL), (seed, fd, dL)
        checked += 1
        if checked == 2:
            break
    assert checked >= 1, "every direction crossed a branch switch"
    res.free()
    h.close()
