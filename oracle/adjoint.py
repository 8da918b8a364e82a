"""Adjoint (reverse-mode derivative) of the tiled BiDiag / R-BiDiag reduction, plain CPU FP64.

ORACLE - test infrastructure only: only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
legs may import it.  It shares no code with the CUDA path.

The reduction of Sec. 3.4 / 3.5 is a sequence of Householder steps.  Written on the whole m x n working
matrix M (with the eliminated entries taken as the exact zeros they stand for), one step is

    x = M[S, c]                      (S: the rows the reflector acts on, c: its pivot column)
    (beta, tau, v) = house(x)        (LAPACK convention, see oracle.kernels.house)
    M[S, :] <- H M[S, :],  H = I - tau v v^T,

and H x = beta e_1, so the step is M' = H(x) M on the rows S.  An LQ step is the same on M^T.  Every
tile kernel of Table 1 (GEQRT, TSQRT, TTQRT and their updates UNMQR, TSMQR, TTMQR) applies one such
step per reflector, to the panel tile's own later columns and to every trailing tile of the same rows,
in the program order of the canonical task list, so the band B is a function of A through this
sequence of steps (the block form T of the compact WY representation does not change the function).

``band_vjp`` walks the steps backwards, one reflector at a time.  With G the gradient of the loss with
respect to the post-step rows M'[S, :]:

* pre-step rows:   M = H M'  (H is its own inverse), so x = M[S, c] = beta (e_1 - tau v);
* through H:       a = M^T v, b = G^T v, tau_bar = -a.b, v_bar = -tau (G a + M b), G_pre = H G;
* through house:   x_bar from (v_bar, tau_bar) (``house_vjp``), added to G_pre[:, c].

A reflector with tau = 0 is the identity (house's sigma = 0 branch) and is treated as constant.
Nothing is blocked or reordered: this is the definition of the chain rule over the step sequence.
The walk starts from the final M = [B; 0] (band of B, zeros elsewhere) and, as a by-product, ends at a
reconstruction of A.
"""
from __future__ import annotations

import numpy as np

from . import bidiag as OB
from . import trees as T


def house_vjp(x, v_bar, tau_bar):
    """Gradient with respect to x of <v_bar, v_tail(x)> + tau_bar tau(x) for (beta, tau, v) = house(x).

    house: alpha = x_0, sigma2 = |x_1:|^2, nu = sqrt(alpha^2 + sigma2), beta = -sgn(alpha) nu,
    tau = (beta - alpha) / beta = 1 - alpha / beta, v_tail = x_1: / (alpha - beta).
    sigma2 = 0 is the identity branch (tau = 0, v = e_1): zero derivative.
    """
    x = np.asarray(x, dtype=np.float64)
    alpha = float(x[0])
    x1 = x[1:]
    sigma2 = float(x1 @ x1)
    if sigma2 == 0.0:
        return np.zeros_like(x)
    nu = np.sqrt(alpha * alpha + sigma2)
    beta = nu if alpha < 0 else -nu
    d = alpha - beta
    g = float(np.asarray(v_bar) @ x1) / (d * d)
    alpha_bar = -tau_bar / beta - g          # d tau / d alpha = -1/beta,  d v_tail / d alpha = -x1 / d^2
    beta_bar = tau_bar * alpha / (beta * beta) + g   # d tau / d beta = alpha/beta^2,  d v_tail / d beta = x1 / d^2
    xb = np.zeros_like(x)
    xb[0] = alpha_bar
    xb[1:] = np.asarray(v_bar) / d
    xb += beta_bar * (beta / (nu * nu)) * x   # d beta / d x = -sgn(alpha) x / nu = (beta / nu^2) x
    return xb


def reflector_support(rec, jj, nb):
    """Rows (oriented coordinates) of reflector jj of a panel-task record, its pivot column, and v over
    those rows (first entry 1).

    GE (GEQRT on oriented tile (i, k)): rows i*nb + jj .. end of the tile, v = [1; V[jj+1:, jj]].
    TS: pivot row piv*nb + jj, then every row of tile i, v = [1; V[:, jj]].
    TT: pivot row piv*nb + jj, then rows 0 .. min(jj+1, rows of tile i) - 1 of tile i.
    """
    V = rec["V"]
    i0 = rec["i"] * nb
    col = rec["k"] * nb + jj
    if rec["kind"] == "GE":
        rows = np.arange(i0 + jj, i0 + V.shape[0])
        v = np.concatenate(([1.0], V[jj + 1:, jj]))
    else:
        ri = V.shape[0]
        l = ri if rec["kind"] == "TS" else min(jj + 1, ri)
        rows = np.concatenate(([rec["piv"] * nb + jj], np.arange(i0, i0 + l)))
        v = np.concatenate(([1.0], V[0:l, jj]))
    return rows, col, v


def reflector_vjp(M, G, rows, col, v, tau):
    """One step backwards: M, G (oriented views) hold the post-step state and its gradient on entry and
    the pre-step state and its gradient on return."""
    Mp = M[rows, :]
    Gp = G[rows, :]
    Mpre = Mp - tau * np.outer(v, v @ Mp)
    a = v @ Mpre
    b = v @ Gp
    tau_bar = -float(a @ b)
    v_bar = -tau * (Gp @ a + Mpre @ b)
    Gpre = Gp - tau * np.outer(v, b)
    Gpre[:, col] += house_vjp(Mpre[:, col], v_bar[1:], tau_bar)
    M[rows, :] = Mpre
    G[rows, :] = Gpre


def band_vjp(res, ab_bar):
    """Gradient of <ab_bar, ab> with respect to A for a result of ``oracle.bidiag.bidiag_band``.

    ab_bar: (nb+1) x n in the band storage of ``res["ab"]`` (entries with row index < 0 are ignored).
    Returns (A_bar, A_rec): the m x n gradient and the reconstruction of A from the band and the
    reflectors (a by-product of the backward walk).
    """
    m, n, nb = res["m"], res["n"], res["nb"]
    M = np.zeros((m, n))
    G = np.zeros((m, n))
    M[:n, :n] = OB.band_to_dense(res["ab"], n)
    G[:n, :n] = OB.band_to_dense(np.asarray(ab_bar, dtype=np.float64), n)
    for idx in sorted(res["refl"], reverse=True):
        rec = res["refl"][idx]
        Mo, Go = (M.T, G.T) if rec["phase"] == T.LQ else (M, G)
        for jj in range(len(rec["tau"]) - 1, -1, -1):
            tau = float(rec["tau"][jj])
            if tau == 0.0:
                continue
            rows, col, v = reflector_support(rec, jj, nb)
            reflector_vjp(Mo, Go, rows, col, v, tau)
    return G, M


def dense_band_grad(ab_bar, n):
    """Dense n x n gradient from a band gradient (zero outside the band)."""
    return OB.band_to_dense(np.asarray(ab_bar, dtype=np.float64), n)


def band_of_dense_grad(Bbar, nb):
    """Band storage of the band part of a dense n x n gradient."""
    return OB.band_of(np.asarray(Bbar, dtype=np.float64), nb)
