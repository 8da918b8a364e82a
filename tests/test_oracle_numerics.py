"""Pins of the oracle's arithmetic against what the mathematics fixes (no GPU).

B = Q^T A P must hold to roundoff with Q, P orthogonal; B keeps A's singular values (checked against
LAPACK's SVD and against an independent one-sided Jacobi SVD); special cases reduce to library QR;
|B| does not depend on the tree or the variant (panel QR/LQ factors are unique up to signs); every
reflector satisfies its textbook invariants.  A dropped term, a wrong sign or a transposed operand in
any kernel breaks one of these.
"""
import numpy as np
import pytest

from oracle import bidiag as OB
from oracle import jacobi as OJ
from oracle import kernels as OK
from oracle import trees as T
from paper_1611_06892_gb300 import inputs

EPS = 2.0 ** -53
TREES = (T.FLATTS, T.FLATTT, T.GREEDY, T.AUTO)

SHAPES = [(8, 8, 4, 2), (13, 9, 4, 2), (20, 7, 3, 1), (37, 23, 8, 4), (64, 64, 16, 4), (50, 50, 16, 8),
          (100, 36, 16, 4), (71, 71, 32, 8), (9, 9, 16, 4), (33, 1, 8, 2)]


def dense_b(res):
    return OB.band_to_dense(res["ab"], res["n"])


def check_invariants(A, res, tol=30.0):
    m, n = A.shape
    B = dense_b(res)
    Q = OB.dense_q(res)
    P = OB.dense_p(res)
    Bf = np.zeros((m, n))
    Bf[:n, :n] = B
    nA = np.linalg.norm(A)
    scale = max(m, n) * EPS
    assert np.linalg.norm(A - Q @ Bf @ P.T) <= tol * nA * scale           # P1 residual
    assert np.linalg.norm(Q.T @ Q - np.eye(m)) <= tol * m * EPS             # P2
    assert np.linalg.norm(P.T @ P - np.eye(n)) <= tol * n * EPS
    QtAP = Q.T @ A @ P                                                      # P3 dense mode
    QtAP[:n, :n] -= B
    assert np.abs(QtAP).max() <= tol * nA * scale
    s_a = np.linalg.svd(A, compute_uv=False)                                # P4
    s_b = np.linalg.svd(B, compute_uv=False)
    assert np.abs(s_a - s_b).max() <= tol * scale * s_a[0]
    nb = res["nb"]
    ii, jj = np.indices(B.shape)
    assert np.all(B[(jj < ii) | (jj - ii > nb)] == 0.0)                     # band structure


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("variant", (T.BIDIAG, T.RBIDIAG), ids=("bidiag", "rbidiag"))
def test_residual_orthogonality_singular_values(shape, variant):
    m, n, nb, ib = shape
    A = inputs.gaussian(m, n, seed=m * 1000 + n)
    for tree in TREES:
        res = OB.bidiag_band(A, nb, ib, tree, variant, resources=2)
        check_invariants(A, res)


def test_known_singular_values():
    """A = U diag(s) V^T with Haar U, V: B has exactly the prescribed s (to roundoff)."""
    n = 48
    s = np.logspace(0, -8, n)
    A = inputs.prescribed_singular_values(n, n, s, seed_u=2, seed_v=3)
    for tree in TREES:
        res = OB.bidiag_band(A, 16, 4, tree, T.BIDIAG, resources=2)
        sb = np.linalg.svd(dense_b(res), compute_uv=False)
        assert np.abs(sb - s).max() <= 30 * n * EPS


def test_jacobi_svd_independent():
    """One-sided Jacobi SVD of B equals LAPACK's SVD of A on tiny inputs."""
    A = inputs.gaussian(24, 16, seed=11)
    res = OB.bidiag_band(A, 8, 4, T.GREEDY, T.BIDIAG)
    sj = OJ.singular_values(dense_b(res))
    sa = np.linalg.svd(A, compute_uv=False)
    assert np.abs(sj - sa).max() <= 100 * 24 * EPS * sa[0]
    D = np.diag([3.0, -2.0, 0.5])
    assert np.allclose(OJ.singular_values(D), [3.0, 2.0, 0.5], rtol=0, atol=1e-15)


def test_single_tile_is_qr():
    """m = n <= nb: B is the R of a plain QR (rows equal up to sign)."""
    A = inputs.gaussian(12, 12, seed=5)
    res = OB.bidiag_band(A, 16, 4, T.FLATTS, T.BIDIAG)
    R = np.linalg.qr(A, mode="r")
    B = dense_b(res)
    assert np.allclose(np.abs(B), np.abs(R), atol=1e-13)
    assert np.allclose(np.abs(np.diag(B)), np.abs(np.diag(R)), atol=1e-13)


def test_one_tile_column_is_tiled_qr():
    """q = 1 (n <= nb): BiDiag is a tiled QR, so |B| = |R| of numpy's QR, for every tree."""
    A = inputs.gaussian(70, 10, seed=6)
    R = np.linalg.qr(A, mode="r")
    for tree in TREES:
        res = OB.bidiag_band(A, 16, 4, tree, T.BIDIAG, resources=2)
        assert np.allclose(np.abs(dense_b(res)), np.abs(R), atol=1e-12)


def dense_block_bidiag(A, nb):
    """Tree-free reference: QR of each column panel and LQ of each row panel with numpy."""
    A = np.array(A, dtype=np.float64, copy=True)
    m, n = A.shape
    for k0 in range(0, n, nb):
        k1 = min(k0 + nb, n)
        Q, _ = np.linalg.qr(A[k0:, k0:k1], mode="complete")
        A[k0:, k0:] = Q.T @ A[k0:, k0:]
        if k1 < n:
            Q2, _ = np.linalg.qr(A[k0:k1, k1:].T, mode="complete")
            A[k0:, k1:] = A[k0:, k1:] @ Q2
    B = np.triu(A[:n, :n])
    return np.triu(B) - np.triu(B, nb + 1)


@pytest.mark.parametrize("variant", (T.BIDIAG, T.RBIDIAG), ids=("bidiag", "rbidiag"))
def test_abs_band_is_tree_invariant(variant):
    """|B| is the same for every tree and equals the tree-free dense reference (signs aside)."""
    m, n, nb = 45, 30, 8
    A = inputs.gaussian(m, n, seed=7)
    ref = np.abs(dense_block_bidiag(A, nb))
    for tree in TREES:
        B = dense_b(OB.bidiag_band(A, nb, 4, tree, variant, resources=2))
        assert np.allclose(np.abs(B), ref, atol=1e-11 * np.linalg.norm(A))


def test_house_special_cases():
    beta, tau, v = OK.house(np.array([3.0, 0.0, 0.0]))
    assert (beta, tau) == (3.0, 0.0) and not v.any()
    beta, tau, v = OK.house(np.array([-0.0, 3.0, 4.0]))
    assert beta == -5.0                      # sgn(-0) = +1
    beta, tau, v = OK.house(np.array([-3.0, 4.0]))
    assert beta == 5.0 and 1.0 <= tau <= 2.0
    rng = np.random.default_rng(0)
    for _ in range(20):
        x = rng.standard_normal(7)
        beta, tau, v = OK.house(x)
        u = np.concatenate(([1.0], v))
        H = np.eye(7) - tau * np.outer(u, u)
        assert np.allclose(H @ x, beta * np.eye(7)[0], atol=1e-14)
        assert np.allclose(H @ H.T, np.eye(7), atol=1e-14)
        assert 1.0 <= tau <= 2.0


def test_reflector_invariants():
    """P7: 1 <= tau <= 2, T upper triangular with diag(T) = tau, and I - Y T Y^T orthogonal per block."""
    A = inputs.gaussian(40, 24, seed=9)
    ib = 4
    res = OB.bidiag_band(A, 8, ib, T.AUTO, T.BIDIAG, resources=2)
    for rec in res["refl"].values():
        tau = rec["tau"]
        assert np.all((tau == 0) | ((tau >= 1) & (tau <= 2)))
        Tm = rec["T"]
        Y = OK.reflector_matrix(rec["kind"], rec["V"], len(tau), rec["top_rows"])
        for b0 in range(0, len(tau), ib):
            kb = min(ib, len(tau) - b0)
            Tb = Tm[:kb, b0:b0 + kb]
            assert np.allclose(np.tril(Tb, -1), 0)
            assert np.allclose(np.diag(Tb), tau[b0:b0 + kb])
            Yb = Y[:, b0:b0 + kb]
            H = np.eye(Y.shape[0]) - Yb @ Tb @ Yb.T
            assert np.allclose(H.T @ H, np.eye(Y.shape[0]), atol=1e-13)
            # the block equals the product of its reflectors
            Hp = np.eye(Y.shape[0])
            for l in range(kb):
                Hp = Hp @ (np.eye(Y.shape[0]) - tau[b0 + l] * np.outer(Yb[:, l], Yb[:, l]))
            assert np.allclose(H, Hp, atol=1e-13)


def test_apply_q_p_consistency():
    """apply_q / apply_p agree with dense Q, P in all four modes."""
    A = inputs.gaussian(30, 20, seed=12)
    for variant in (T.BIDIAG, T.RBIDIAG):
        res = OB.bidiag_band(A, 8, 4, T.GREEDY, variant)
        Q, P = OB.dense_q(res), OB.dense_p(res)
        C = inputs.gaussian(30, 5, seed=1)
        D = inputs.gaussian(6, 20, seed=2)
        assert np.allclose(OB.apply_q(res, C, 1), Q.T @ C, atol=1e-13)
        assert np.allclose(OB.apply_q(res, C, 0), Q @ C, atol=1e-13)
        assert np.allclose(OB.apply_p(res, D, 0), D @ P, atol=1e-13)
        assert np.allclose(OB.apply_p(res, D, 1), D @ P.T, atol=1e-13)


def test_zero_and_rank_deficient():
    """Zero columns give identity reflectors (tau = 0); the invariants still hold."""
    A = inputs.gaussian(20, 12, seed=13)
    A[:, 3] = 0.0
    A[:, 7] = A[:, 2]
    for tree in TREES:
        res = OB.bidiag_band(A, 4, 2, tree, T.BIDIAG, resources=2)
        check_invariants(A, res)
    Z = np.zeros((9, 6))
    res = OB.bidiag_band(Z, 4, 2, T.GREEDY, T.BIDIAG)
    assert not res["ab"].any()


def _planted(monkeypatch, name, fn):
    monkeypatch.setattr(OK, name, fn)
    A = inputs.gaussian(24, 16, seed=21)
    with pytest.raises(AssertionError):
        for tree in TREES:
            check_invariants(A, OB.bidiag_band(A, 8, 4, tree, T.BIDIAG, resources=2))


def test_pins_catch_planted_mistakes(monkeypatch):
    """Plant plausible mistakes in the oracle (CPU only) and check that the pins above fail."""
    orig_house, orig_tsmqr, orig_ttmqr = OK.house, OK.tsmqr, OK.ttmqr

    def wrong_sign(x):
        beta, tau, v = orig_house(x)
        return -beta, tau, v

    def dropped_top(V, tau, Cp, Ci, trans=True):
        saved = Cp.copy()
        orig_tsmqr(V, tau, Cp, Ci, trans)
        Cp[...] = saved

    def transposed_tt(V, tau, Cp, Ci, trans=True):
        orig_ttmqr(V, tau, Cp, Ci, not trans)

    for name, fn in (("house", wrong_sign), ("tsmqr", dropped_top), ("ttmqr", transposed_tt)):
        with monkeypatch.context() as mp:
            _planted(mp, name, fn)
