"""Tiled BiDiag / R-BiDiag reduction to band bidiagonal form, plain CPU FP64 (the oracle).

ORACLE - test infrastructure only: only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
``cpu_baseline`` / reference legs may import it.  It shares no code with the CUDA path.

``bidiag_band(A, nb, ib, tree, variant)`` runs the canonical task list of ``oracle.trees`` in program
order with the Level-2 kernels of ``oracle.kernels`` and returns B = Q^T A P in LAPACK upper-band storage
(ldab = nb + 1, B[i, j] at ab[nb + i - j, j] for max(0, j - nb) <= i <= j), the reflectors of every
panel task and the task list.  Sec. 3.4 (BiDiag), Sec. 3.5 (R-BiDiag), Algorithms 1-4.

Tiles are ragged at the bottom and right edges (the paper assumes m = p nb, n = q nb; a last tile of
m - (p-1) nb rows / n - (q-1) nb columns is the reading used here).  m >= n is required (Sec. 3.6 says
m < n is the transposed problem).
"""
from __future__ import annotations

import numpy as np

from . import kernels as K
from . import trees as T


class Tiles:
    """Tile views of a dense column-major-agnostic numpy matrix (row block a, column block b)."""

    def __init__(self, M, nb):
        self.M = M
        self.nb = nb
        self.m, self.n = M.shape

    def rows(self, a):
        return range(a * self.nb, min((a + 1) * self.nb, self.m))

    def cols(self, b):
        return range(b * self.nb, min((b + 1) * self.nb, self.n))

    def tile(self, a, b):
        nb = self.nb
        return self.M[a * nb:min((a + 1) * nb, self.m), b * nb:min((b + 1) * nb, self.n)]

    def otile(self, lq, a, b):
        """Oriented tile: actual (a, b) for QR steps, transpose of actual (b, a) for LQ steps."""
        return self.tile(b, a).T if lq else self.tile(a, b)


def _record(kind, phase, k, i, piv, V, tau, top_rows, ib):
    Y = K.reflector_matrix(kind, V, len(tau), top_rows)
    return {"kind": kind, "phase": phase, "k": k, "i": i, "piv": piv,
            "V": V.copy(), "tau": tau.copy(), "T": K.build_t(Y, tau, ib), "top_rows": top_rows}


def run_tasks(state, tasks):
    """Execute tasks (program order) on ``state``; used whole by ``bidiag_band`` and in part for timing."""
    ib = state["ib"]
    variant = state["variant"]
    refl = state["refl"]
    for idx, (typ, phase, k, i, piv, j) in tasks:
        if typ == T.COPY:
            src = state["A"].tile(i, j)
            dst = state["R"].tile(i, j)
            src = src[:dst.shape[0], :]    # a ragged last tile of R keeps only its n - (q-1) nb rows
            dst[...] = np.triu(src) if i == j else src
            continue
        mat = state["R"] if T.task_buffer(phase, k, variant) == 1 else state["A"]
        lq = phase == T.LQ
        if typ == T.GEQRT:
            X = mat.otile(lq, i, k)
            tau = K.geqrt(X)
            refl[idx] = _record("GE", phase, k, i, piv, X, tau, 0, ib)
            state["owner"][(T.GEQRT, phase, k, i)] = idx
        elif typ == T.UNMQR:
            r = refl[state["owner"][(T.GEQRT, phase, k, i)]]
            K.unmqr(r["V"], r["tau"], mat.otile(lq, i, j))
        elif typ == T.TSQRT:
            P = mat.otile(lq, piv, k)
            X = mat.otile(lq, i, k)
            assert P.shape[0] >= X.shape[1], "pivot tile must hold a full triangle"
            tau = K.tsqrt(P, X)
            refl[idx] = _record("TS", phase, k, i, piv, X, tau, X.shape[1], ib)
            state["owner"][(T.TSQRT, phase, k, i)] = idx
        elif typ == T.TSMQR:
            r = refl[state["owner"][(T.TSQRT, phase, k, i)]]
            K.tsmqr(r["V"], r["tau"], mat.otile(lq, piv, j), mat.otile(lq, i, j))
        elif typ == T.TTQRT:
            P = mat.otile(lq, piv, k)
            X = mat.otile(lq, i, k)
            assert P.shape[0] >= X.shape[1], "pivot tile must hold a full triangle"
            tau = K.ttqrt(P, X)
            refl[idx] = _record("TT", phase, k, i, piv, X, tau, X.shape[1], ib)
            state["owner"][(T.TTQRT, phase, k, i)] = idx
        elif typ == T.TTMQR:
            r = refl[state["owner"][(T.TTQRT, phase, k, i)]]
            K.ttmqr(r["V"], r["tau"], mat.otile(lq, piv, j), mat.otile(lq, i, j))
        else:
            raise ValueError(typ)


def new_state(A, nb, ib, tree, variant, resources=None, gamma=2):
    A = np.array(A, dtype=np.float64, copy=True)
    m, n = A.shape
    if m < n or n < 1:
        raise ValueError("need m >= n >= 1")
    if not (1 <= ib <= nb and nb % ib == 0):
        raise ValueError("need 1 <= ib <= nb and nb % ib == 0")
    p, q = -(-m // nb), -(-n // nb)
    tasks = T.task_list(p, q, tree, variant, resources, gamma)
    return {"A": Tiles(A, nb), "R": Tiles(np.zeros((n, n)), nb) if T.split_of(variant) is not None else None,
            "nb": nb, "ib": ib, "tree": tree, "variant": variant, "m": m, "n": n, "p": p, "q": q,
            "tasks": tasks, "refl": {}, "owner": {}}


def band_of(M, nb):
    """Band of the n x n leading block of M in LAPACK upper-band storage; entries outside are exact zeros."""
    n = M.shape[1]
    ab = np.zeros((nb + 1, n))
    for jj in range(n):
        for ii in range(max(0, jj - nb), jj + 1):
            ab[nb + ii - jj, jj] = M[ii, jj]
    return ab


def band_to_dense(ab, n):
    nb = ab.shape[0] - 1
    B = np.zeros((n, n))
    for jj in range(n):
        for ii in range(max(0, jj - nb), jj + 1):
            B[ii, jj] = ab[nb + ii - jj, jj]
    return B


def bidiag_band(A, nb, ib, tree, variant, resources=None, gamma=2):
    """Reduce A (m x n, m >= n) to band bidiagonal form.  Returns a result dict (see module doc)."""
    st = new_state(A, nb, ib, tree, variant, resources, gamma)
    run_tasks(st, list(enumerate(st["tasks"])))
    s = T.split_of(variant)
    if s is None:
        final = st["A"].M
    else:
        # rows of the first s tile rows come from the BiDiag steps on A, the rest from the R copy
        final = st["R"].M.copy()
        final[:s * nb, :] = st["A"].M[:s * nb, :]
    st["ab"] = band_of(final, nb)
    st["work"] = st["A"].M
    st["work2"] = st["R"].M if s is not None else None
    return st


def _apply_record_left(r, nb, C, trans):
    """Apply one panel task's reflectors (QR side) to the rows of C."""
    i0 = r["i"] * nb
    tau = r["tau"]
    Kr = len(tau)
    order = range(Kr) if trans else range(Kr - 1, -1, -1)
    V = r["V"]
    for jj in order:
        t = tau[jj]
        if t == 0.0:
            continue
        if r["kind"] == "GE":
            idx = np.arange(i0 + jj, i0 + V.shape[0])
            v = np.concatenate(([1.0], V[jj + 1:, jj]))
        else:
            p0 = r["piv"] * nb
            l = V.shape[0] if r["kind"] == "TS" else min(jj + 1, V.shape[0])
            idx = np.concatenate(([p0 + jj], np.arange(i0, i0 + l)))
            v = np.concatenate(([1.0], V[0:l, jj]))
        w = v @ C[idx, :]
        C[idx, :] -= t * np.outer(v, w)


def apply_q(res, C, trans):
    """Q C (trans = 0) or Q^T C (trans = 1) for C with m rows (R-BiDiag: Q = Q_preQR diag(Q_2, I))."""
    C = np.array(C, dtype=np.float64, copy=True)
    recs = [res["refl"][i] for i in sorted(res["refl"]) if res["refl"][i]["phase"] != T.LQ]
    seq = recs if trans else recs[::-1]
    for r in seq:
        _apply_record_left(r, res["nb"], C, trans)
    return C


def apply_p(res, C, trans):
    """C P (trans = 0) or C P^T (trans = 1) for C with n columns."""
    Ct = np.array(C, dtype=np.float64, copy=True).T.copy()
    # C P = (P^T C^T)^T, and P_t = H_0 ... H_{K-1} as for Q, so C P uses the "Q^T" order on C^T.
    recs = [res["refl"][i] for i in sorted(res["refl"]) if res["refl"][i]["phase"] == T.LQ]
    seq = recs if not trans else recs[::-1]
    for r in seq:
        _apply_record_left(r, res["nb"], Ct, not trans)
    return Ct.T.copy()


def dense_q(res):
    return apply_q(res, np.eye(res["m"]), 0)


def dense_p(res):
    return apply_p(res, np.eye(res["n"]), 0)
