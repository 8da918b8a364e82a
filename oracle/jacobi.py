"""One-sided Jacobi SVD (Hestenes 1958; Demmel and Veselic 1992): singular values of a small matrix.

ORACLE - test infrastructure only.  Used as an independent check that the singular values of the band
matrix B equal those of A (B = Q^T A P with Q, P orthogonal), next to numpy's LAPACK SVD.
"""
from __future__ import annotations

import numpy as np


def singular_values(M, tol=1e-15, max_sweeps=60):
    """Singular values of M (rows >= cols after an internal transpose), in decreasing order.

    Columns are orthogonalised pairwise by plane rotations until every pair satisfies
    |c_i . c_j| <= tol * ||c_i|| ||c_j||; the singular values are then the column norms.
    """
    U = np.array(M, dtype=np.float64, copy=True)
    if U.shape[0] < U.shape[1]:
        U = U.T.copy()
    n = U.shape[1]
    for _ in range(max_sweeps):
        rotated = False
        for i in range(n - 1):
            for j in range(i + 1, n):
                a = U[:, i] @ U[:, i]
                b = U[:, j] @ U[:, j]
                g = U[:, i] @ U[:, j]
                if g == 0.0 or abs(g) <= tol * np.sqrt(a * b):
                    continue
                rotated = True
                zeta = (b - a) / (2.0 * g)
                t = np.copysign(1.0, zeta) / (abs(zeta) + np.sqrt(1.0 + zeta * zeta))
                c = 1.0 / np.sqrt(1.0 + t * t)
                s = c * t
                ui = U[:, i].copy()
                U[:, i] = c * ui - s * U[:, j]
                U[:, j] = s * ui + c * U[:, j]
        if not rotated:
            break
    return np.sort(np.linalg.norm(U, axis=0))[::-1]
