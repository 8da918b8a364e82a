"""Pins of the oracle adjoint (oracle/adjoint.py) against things it does not compute itself:
central finite differences of the oracle forward reduction, the closed-form gradient of the sum of
singular values (sigma(B) = sigma(A), so d(sum sigma)/dA = U V^T for the thin SVD A = U S V^T), and the
reconstruction of A by the backward walk."""
import numpy as np
import pytest

from oracle import adjoint as AD
from oracle import bidiag as OB
from oracle import kernels as K
from oracle import trees as T

TREES = (T.FLATTS, T.FLATTT, T.GREEDY, T.AUTO)
VARIANTS = (T.BIDIAG, T.RBIDIAG)


def loss_band(A, W, nb, ib, tree, variant):
    return float((W * OB.bidiag_band(A, nb, ib, tree, variant, resources=2)["ab"]).sum())


@pytest.mark.parametrize("x", [[3.0, 1.0, -2.0, 0.5], [-0.7, 0.2, 0.1], [1e-3, 2.0, -1.0, 4.0, 0.3], [2.0, -1e-2]])
def test_house_vjp_finite_differences(x):
    """house_vjp against central differences of oracle.kernels.house (tau and the reflector tail)."""
    x = np.array(x)
    rng = np.random.default_rng(len(x))
    vb = rng.standard_normal(len(x) - 1)
    tb = float(rng.standard_normal())

    def f(y):
        _, tau, v = K.house(y)
        return tb * tau + vb @ v

    h = 1e-6
    fd = np.array([(f(x + h * e) - f(x - h * e)) / (2 * h) for e in np.eye(len(x))])
    got = AD.house_vjp(x, vb, tb)
    assert np.allclose(got, fd, rtol=1e-7, atol=1e-8)


def test_house_vjp_identity_branch():
    """sigma = 0 (zero tail): house returns the identity reflector, whose derivative is taken as 0."""
    assert np.all(AD.house_vjp(np.array([2.0, 0.0, 0.0]), np.ones(2), 1.0) == 0.0)


@pytest.mark.parametrize("variant", VARIANTS, ids=("bidiag", "rbidiag"))
@pytest.mark.parametrize("tree", TREES, ids=("flatts", "flattt", "greedy", "auto"))
def test_full_jacobian_tiny(tree, variant):
    """Every entry of dL/dA, L = <W, band>, against central differences on a 9 x 7 matrix of 3 x 2 tiles
    (nb = 4, ragged last tile row and column)."""
    rng = np.random.default_rng(10 + tree + 4 * variant)
    m, n, nb, ib = 9, 7, 4, 2
    A = rng.standard_normal((m, n))
    W = rng.standard_normal((nb + 1, n))
    res = OB.bidiag_band(A, nb, ib, tree, variant, resources=2)
    Ab, _ = AD.band_vjp(res, W)
    h = 1e-6
    fd = np.zeros((m, n))
    for i in range(m):
        for j in range(n):
            E = np.zeros((m, n))
            E[i, j] = h
            fd[i, j] = (loss_band(A + E, W, nb, ib, tree, variant) - loss_band(A - E, W, nb, ib, tree, variant)) / (2 * h)
    assert np.abs(Ab - fd).max() <= 1e-7 * max(1.0, np.abs(fd).max())


@pytest.mark.parametrize("variant", VARIANTS, ids=("bidiag", "rbidiag"))
@pytest.mark.parametrize("tree", TREES, ids=("flatts", "flattt", "greedy", "auto"))
def test_directional_derivatives_64x32(tree, variant):
    """The differentiation check size: 64 x 32, nb = 16, ib = 4 (4 x 2 tiles), L = <W, B> + sum sigma(B);
    <dL/dA, E> against central differences along random directions E."""
    rng = np.random.default_rng(20 + tree + 4 * variant)
    m, n, nb, ib = 64, 32, 16, 4
    A = rng.standard_normal((m, n))
    W = rng.standard_normal((nb + 1, n))

    def loss(X):
        r = OB.bidiag_band(X, nb, ib, tree, variant, resources=2)
        B = OB.band_to_dense(r["ab"], n)
        return float((W * r["ab"]).sum()) + float(np.linalg.svd(B, compute_uv=False).sum())

    res = OB.bidiag_band(A, nb, ib, tree, variant, resources=2)
    B = OB.band_to_dense(res["ab"], n)
    U, _, Vt = np.linalg.svd(B)
    ab_bar = W + AD.band_of_dense_grad(U @ Vt, nb)
    Ab, _ = AD.band_vjp(res, ab_bar)
    h = 1e-6
    for _ in range(4):
        E = rng.standard_normal((m, n))
        fd = (loss(A + h * E) - loss(A - h * E)) / (2 * h)
        an = float((Ab * E).sum())
        assert abs(fd - an) <= 1e-7 * max(1.0, abs(an))


@pytest.mark.parametrize("case", [(64, 32, 16, 4, T.GREEDY, T.BIDIAG), (100, 70, 16, 8, T.FLATTS, T.BIDIAG),
                                  (120, 40, 16, 4, T.GREEDY, T.RBIDIAG), (75, 75, 8, 4, T.AUTO, T.BIDIAG),
                                  (90, 33, 16, 16, T.FLATTT, T.RBIDIAG)],
                         ids=lambda c: "x".join(map(str, c)))
def test_sum_of_singular_values_closed_form(case):
    """sigma(B) = sigma(A), so the gradient of sum sigma(B), pushed back through the reduction, is U V^T."""
    m, n, nb, ib, tree, variant = case
    rng = np.random.default_rng(m + n)
    A = rng.standard_normal((m, n))
    res = OB.bidiag_band(A, nb, ib, tree, variant, resources=2)
    B = OB.band_to_dense(res["ab"], n)
    U, _, Vt = np.linalg.svd(B)
    Ab, Arec = AD.band_vjp(res, AD.band_of_dense_grad(U @ Vt, nb))
    Ua, _, Vta = np.linalg.svd(A, full_matrices=False)
    assert np.abs(Ab - Ua @ Vta).max() <= 1e-12
    assert np.abs(Arec - A).max() <= 1e-13 * np.linalg.norm(A)


def test_zero_band_gradient():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((40, 24))
    res = OB.bidiag_band(A, 8, 4, T.GREEDY, T.BIDIAG, resources=2)
    Ab, _ = AD.band_vjp(res, np.zeros((9, 24)))
    assert np.all(Ab == 0.0)
