"""Tile kernels of the tiled QR / LQ algorithms, one Householder reflector at a time (Level 2), FP64.

ORACLE - test infrastructure only (imported by ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
CPU legs; never by the product path).  It shares no code with the CUDA kernels.

Kernels of Table 1 (Sec. 3.2): GEQRT, UNMQR, TSQRT, TSMQR, TTQRT, TTMQR.  Every function works in place
on numpy views; an LQ kernel is the same function applied to the transposed views.

Readings where the paper is silent:

* Householder convention (LAPACK style): for x = [alpha; x_tail], sigma2 = x_tail . x_tail.  If
  sigma2 == 0 the reflector is the identity (tau = 0, beta = alpha).  Otherwise
  beta = -sgn(alpha) * sqrt(alpha^2 + sigma2) with sgn(alpha) = -1 iff alpha < 0 (so +0 and -0 give +1),
  tau = (beta - alpha) / beta and v = [1; x_tail / (alpha - beta)].  H = I - tau v v^T maps x to beta e_1.
* Norms are a plain sum of squares followed by sqrt (no scaling).
* A panel tile with r rows and c columns produces min(r, c) reflectors (GEQRT); TS and TT panels produce
  c reflectors (their top tile is a triangle of order c).
* The T factor of the compact WY form is built per block of ``ib`` reflectors by the forward recurrence
  T[0:l, l] = -tau_l T[0:l, 0:l] (V[:, 0:l]^T v_l), T[l, l] = tau_l.  The oracle applies reflectors one at a
  time and uses T only for export and comparison.
"""
from __future__ import annotations

import numpy as np


def house(x):
    """Householder reflector of vector x: returns (beta, tau, v_tail)."""
    alpha = float(x[0])
    tail = np.asarray(x[1:], dtype=np.float64)
    sigma2 = float(tail @ tail)
    if sigma2 == 0.0:
        return alpha, 0.0, np.zeros_like(tail)
    nrm = np.sqrt(alpha * alpha + sigma2)
    beta = nrm if alpha < 0 else -nrm
    tau = (beta - alpha) / beta
    return beta, tau, tail / (alpha - beta)


def geqrt(A):
    """QR of tile A (r x c) in place: R in the upper part, reflector tails below the diagonal.

    Returns tau (length min(r, c)).
    """
    r, c = A.shape
    K = min(r, c)
    tau = np.zeros(K)
    for j in range(K):
        beta, t, v = house(A[j:, j])
        A[j, j] = beta
        A[j + 1:, j] = v
        tau[j] = t
        if t != 0.0 and j + 1 < c:
            w = A[j, j + 1:] + v @ A[j + 1:, j + 1:]
            A[j, j + 1:] -= t * w
            A[j + 1:, j + 1:] -= t * np.outer(v, w)
    return tau


def unmqr(V, tau, C, trans=True):
    """C <- Q^T C (trans) or Q C with Q = H_0 ... H_{K-1} from a GEQRT tile V (unit lower part)."""
    K = len(tau)
    order = range(K) if trans else range(K - 1, -1, -1)
    for j in order:
        t = tau[j]
        if t == 0.0:
            continue
        v = V[j + 1:, j]
        w = C[j, :] + v @ C[j + 1:, :]
        C[j, :] -= t * w
        C[j + 1:, :] -= t * np.outer(v, w)


def tsqrt(R, A):
    """Eliminate the square tile A under the triangle R (c x c upper part of the pivot tile), in place.

    R's upper triangle is updated, A is overwritten by the reflector tails (full).  Returns tau (length c).
    """
    c = A.shape[1]
    tau = np.zeros(c)
    for j in range(c):
        x = np.concatenate(([R[j, j]], A[:, j]))
        beta, t, v = house(x)
        R[j, j] = beta
        A[:, j] = v
        tau[j] = t
        if t != 0.0 and j + 1 < c:
            w = R[j, j + 1:] + v @ A[:, j + 1:]
            R[j, j + 1:] -= t * w
            A[:, j + 1:] -= t * np.outer(v, w)
    return tau


def tsmqr(V, tau, Cp, Ci, trans=True):
    """[Cp; Ci] <- Q^T [Cp; Ci] (trans) or Q [Cp; Ci]; reflector j is [e_j; V[:, j]]."""
    K = len(tau)
    order = range(K) if trans else range(K - 1, -1, -1)
    for j in order:
        t = tau[j]
        if t == 0.0:
            continue
        v = V[:, j]
        w = Cp[j, :] + v @ Ci
        Cp[j, :] -= t * w
        Ci -= t * np.outer(v, w)


def ttqrt(R, Ri):
    """Eliminate triangle Ri (upper part, r_i x c) under triangle R (c x c upper part), in place.

    Reflector j has tail Ri[0:min(j+1, r_i), j]; it overwrites that part of Ri.  Returns tau (length c).
    Only upper parts are read or written, so the tiles' strict lower parts keep their GEQRT reflectors.
    """
    ri, c = Ri.shape
    tau = np.zeros(c)
    for j in range(c):
        l = min(j + 1, ri)
        x = np.concatenate(([R[j, j]], Ri[0:l, j]))
        beta, t, v = house(x)
        R[j, j] = beta
        Ri[0:l, j] = v
        tau[j] = t
        if t != 0.0 and j + 1 < c:
            w = R[j, j + 1:] + v @ Ri[0:l, j + 1:]
            R[j, j + 1:] -= t * w
            Ri[0:l, j + 1:] -= t * np.outer(v, w)
    return tau


def ttmqr(V, tau, Cp, Ci, trans=True):
    """Apply TTQRT reflectors: reflector j is [e_j; V[0:min(j+1, r), j]] acting on rows j of Cp and 0.. of Ci."""
    K = len(tau)
    ri = V.shape[0]
    order = range(K) if trans else range(K - 1, -1, -1)
    for j in order:
        t = tau[j]
        if t == 0.0:
            continue
        l = min(j + 1, ri)
        v = V[0:l, j]
        w = Cp[j, :] + v @ Ci[0:l, :]
        Cp[j, :] -= t * w
        Ci[0:l, :] -= t * np.outer(v, w)


def reflector_matrix(kind, V, K, top_rows):
    """Dense reflector vectors (columns) of a panel task, over [top tile rows; tail tile rows].

    GEQRT: the unit lower trapezoid of V (top_rows = 0, rows of V only).
    TS / TT: [e_j over ``top_rows`` rows; tail from V].
    """
    if kind == "GE":
        r = V.shape[0]
        Y = np.zeros((r, K))
        for j in range(K):
            Y[j, j] = 1.0
            Y[j + 1:, j] = V[j + 1:, j]
        return Y
    ri = V.shape[0]
    Y = np.zeros((top_rows + ri, K))
    for j in range(K):
        Y[j, j] = 1.0
        if kind == "TS":
            Y[top_rows:, j] = V[:, j]
        else:
            l = min(j + 1, ri)
            Y[top_rows:top_rows + l, j] = V[0:l, j]
    return Y


def build_t(Y, tau, ib):
    """T factor, ib x K: diagonal ib x ib blocks of the compact WY form, block b in columns b*ib..."""
    K = len(tau)
    T = np.zeros((ib, K))
    for b0 in range(0, K, ib):
        kb = min(ib, K - b0)
        Tb = np.zeros((kb, kb))
        for l in range(kb):
            col = b0 + l
            Tb[l, l] = tau[col]
            if l > 0:
                z = Y[:, b0:col].T @ Y[:, col]
                Tb[0:l, l] = -tau[col] * (Tb[0:l, 0:l] @ z)
        T[0:kb, b0:b0 + kb] = Tb
    return T
